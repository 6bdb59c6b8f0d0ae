"""CPU-only checks of the C-ABI library: it builds, loads, exports every
symbol that include/gridff.h declares with the signature the binding gives
it, and rejects use without a GPU."""
import os
import re

import pytest

from conftest import ROOT


def _declared():
    txt = open(os.path.join(ROOT, "include", "gridff.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gridff_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_2508_15522_gb300 import gridff
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(gridff.lib, n)]
    assert not missing, missing
    assert set(declared) == set(gridff.EXPORTED)


def test_binding_fails_loudly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2508_15522_gb300 import gridff
    with pytest.raises(gridff.GridffError):
        gridff.Context(0)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2508_15522_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", txt, flags=re.M), f


def _prototypes():
    txt = open(os.path.join(ROOT, "include", "gridff.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \t\*]*?)\s*\b(gridff_\w+)\s*\(([^;{]*?)\)\s*;", txt,
                                        flags=re.S):
        ps = [p.strip() for p in params.split(",")] if params.strip() not in ("", "void") else []
        out[name] = (" ".join(ret.split()), ps)
    return out


def test_binding_signatures_match_the_header():
    """Every ctypes signature of the binding has the header's argument count,
    a pointer where the header has one, the header's scalar width elsewhere,
    and the header's return type (a mismatch would corrupt a call at run
    time, which only a GPU run would otherwise show)."""
    import ctypes as C
    import __graft_entry__ as g
    g.build()
    from paper_2508_15522_gb300 import gridff
    protos = _prototypes()
    assert set(protos) == set(_declared())
    scalar = {"int": C.c_int, "int32_t": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64,
              "size_t": C.c_size_t, "double": C.c_double, "float": C.c_float}
    ret_of = {"gridff_status": C.c_int32, "void": None, "double": C.c_double, "int64_t": C.c_int64,
              "const char*": C.c_char_p, "void*": C.c_void_p}
    bad = []
    for name, (ret, params) in protos.items():
        f = getattr(gridff.lib, name)
        if ret.replace(" *", "*") not in ret_of or f.restype is not ret_of[ret.replace(" *", "*")]:
            bad.append((name, "return", ret, f.restype))
        if len(params) != len(f.argtypes):
            bad.append((name, "count", len(params), len(f.argtypes)))
            continue
        for p, a in zip(params, f.argtypes):
            if "*" in p or "[" in p:
                ok = a in (C.c_void_p, C.c_char_p) or issubclass(a, C._Pointer)
            else:
                t = re.sub(r"\bconst\b", "", p).split()[0]
                ok = t in scalar and C.sizeof(a) == C.sizeof(scalar[t]) and \
                    issubclass(a, C._SimpleCData) and a._type_ == scalar[t]._type_
            if not ok:
                bad.append((name, p, a))
    assert not bad, bad


STRUCTS = {"Substrate": "gridff_substrate", "GridOpts": "gridff_grid_opts", "Molecule": "gridff_molecule",
           "FireParams": "gridff_fire_params", "RelaxResult": "gridff_relax_result", "MDParams": "gridff_md_params",
           "LangevinParams": "gridff_langevin_params", "LaunchConfig": "gridff_launch_config",
           "TuneTrial": "gridff_tune_trial", "TrainParams": "gridff_train_params"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of the header's parameter structs have the C
    compiler's size and field offsets (a C program built from the header
    prints them)."""
    import ctypes as C
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import __graft_entry__ as g
    g.build()
    from paper_2508_15522_gb300 import gridff
    lines = ['#include <stdio.h>', '#include "gridff.h"', "int main(void) {"]
    want = {}
    for py, cname in STRUCTS.items():
        cls = getattr(gridff, py)
        want[cname] = C.sizeof(cls)
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            want[f"{cname}.{f[0]}"] = getattr(cls, f[0]).offset
            lines.append(f'  printf("{cname}.{f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert {k: int(v) for k, v in got.items()} == want


def test_parameter_defaults_match_the_oracle_and_the_header():
    """FIRE defaults of the library (Bitzek et al. 2006 constants, the
    displacement cap and the convergence threshold) equal the oracle's,
    stated independently; grid defaults are those the header documents
    (alpha 1.5 1/A and the 17 A Morse cutoff of Sec. 6)."""
    import ctypes as C
    import dataclasses
    import __graft_entry__ as g
    g.build()
    from oracle import dynamics as odyn
    from paper_2508_15522_gb300 import gridff
    p = gridff.FireParams()
    gridff.lib.gridff_fire_params_default(C.byref(p))
    for f in dataclasses.fields(odyn.FireParams):
        assert getattr(p, f.name) == pytest.approx(getattr(odyn.FireParams(), f.name), rel=1e-7), f.name
    assert p.clock_budget_s == 0.0
    o = gridff.GridOpts()
    gridff.lib.gridff_grid_opts_default(C.byref(o))
    assert (o.alpha, o.rcut, o.ewald_tol, o.ewald_rcut) == (1.5, 17.0, 1e-10, 12.0)
    assert o.channels == gridff.CH_C | gridff.CH_P | gridff.CH_L and o.storage == gridff.STORE_F32
    assert o.keep_f64 == 0 and o.spacing == 0.0 and list(o.origin) == [0.0] * 3 and list(o.length) == [0.0] * 3
