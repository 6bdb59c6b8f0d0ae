"""CPU-only checks of the C-ABI library: it builds, loads, exports every
symbol that include/gridff.h declares, and rejects use without a GPU."""
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
