"""Thin Python binding of libgridff (ctypes; argument marshalling only).

Every computation runs in the CUDA library behind the C ABI declared in
``include/gridff.h``; this module converts numpy arrays / torch tensors to
pointers and raises on non-OK statuses.  Importing it loads the library and
fails loudly if it has not been built (no CPU fallback exists).

Arrays: numpy arrays are host memory; torch CUDA tensors are passed as
device pointers (``GRIDFF_DEVICE_PTRS``) and used in place.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgridff.so")

# status codes and flags (mirror gridff.h)
OK, EINVAL, ENOMEM, ECUDA, EABORTED, ESTEPLIMIT, ENOTSUP, ETIMEOUT = range(8)
REP_CONVERGED, REP_BELOW, REP_NONFINITE, REP_ABORTED, REP_STEPLIMIT = 1, 2, 4, 8, 16
DEVICE_PTRS, ASYNC, CONTINUE, NO_GRID, NO_INTRA = 1, 2, 4, 8, 16
POINTS_BINNED = 32
TEST_NO_HANDOFF = 256
CH_C, CH_P, CH_L = 1, 2, 4
STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EABORTED", 5: "ESTEPLIMIT",
                6: "ENOTSUP", 7: "ETIMEOUT"}


class GridffError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Substrate(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.POINTER(C.c_double)), ("q", C.POINTER(C.c_double)),
                ("R", C.POINTER(C.c_double)), ("eps", C.POINTER(C.c_double)), ("cell", C.c_double * 9)]


class GridOpts(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("length", C.c_double * 3), ("spacing", C.c_double),
                ("alpha", C.c_double), ("rcut", C.c_double), ("ewald_tol", C.c_double),
                ("ewald_rcut", C.c_double), ("channels", C.c_int32), ("storage", C.c_int32),
                ("keep_f64", C.c_int32), ("ghost_below", C.c_int32)]


class Molecule(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.c_void_p), ("q", C.c_void_p), ("R", C.c_void_p),
                ("eps", C.c_void_p), ("mass", C.c_void_p),
                ("n_bonds", C.c_int32), ("bonds", C.c_void_p), ("bond_k", C.c_void_p),
                ("bond_r0", C.c_void_p),
                ("n_angles", C.c_int32), ("angles", C.c_void_p), ("angle_k", C.c_void_p),
                ("angle_cos0", C.c_void_p),
                ("n_torsions", C.c_int32), ("torsions", C.c_void_p), ("torsion_V", C.c_void_p),
                ("torsion_n", C.c_void_p), ("torsion_cos_nphi0", C.c_void_p)]


class FireParams(C.Structure):
    _fields_ = [("dt_start", C.c_float), ("dt_max", C.c_float), ("n_min", C.c_int32),
                ("f_inc", C.c_float), ("f_dec", C.c_float), ("alpha_start", C.c_float),
                ("f_alpha", C.c_float), ("d_max", C.c_float), ("f_conv", C.c_float),
                ("clock_budget_s", C.c_double)]


class RelaxResult(C.Structure):
    _fields_ = [("atom_evals", C.c_int64), ("n_converged", C.c_int32), ("max_steps", C.c_int32)]


class MDParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("record_every", C.c_int32), ("clock_budget_s", C.c_double)]


class LangevinParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("temperature", C.c_float), ("gamma", C.c_float), ("seed", C.c_uint64),
                ("step0", C.c_int64), ("clock_budget_s", C.c_double)]


class LaunchConfig(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("lanes_per_replica", C.c_int32), ("warps_per_block", C.c_int32),
                ("cache_slots", C.c_int32), ("queue", C.c_int32), ("l2_window", C.c_int32),
                ("blocks", C.c_int32), ("cache_global", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneTrial(C.Structure):
    _fields_ = [("cfg", LaunchConfig), ("atom_evals_per_s", C.c_double), ("ms", C.c_double)]


class TrainParams(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("w_q", C.c_float), ("w_t", C.c_float), ("tile", C.c_double * 2)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    P, I32, F64 = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "gridff_create": (I32, [C.c_int, P, C.POINTER(P)]),
        "gridff_destroy": (None, [P]),
        "gridff_last_error": (C.c_char_p, [P]),
        "gridff_stream": (P, [P]),
        "gridff_set_abort": (None, [P, C.c_int]),
        "gridff_grid_opts_default": (None, [C.POINTER(GridOpts)]),
        "gridff_build_grid": (I32, [P, C.POINTER(Substrate), C.POINTER(GridOpts), C.POINTER(P)]),
        "gridff_grid_from_coefs": (I32, [P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int32), I32, C.POINTER(C.c_double), I32,
                                         C.POINTER(P)]),
        "gridff_fit_coefs_noalloc": (I32, [P, P, P, C.POINTER(C.c_int32), I32, C.c_int]),
        "gridff_grid_info": (I32, [P, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_size_t)]),
        "gridff_grid_download_f64": (I32, [P, C.c_int, C.POINTER(C.c_double)]),
        "gridff_grid_storage": (I32, [P, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
        "gridff_grid_floor": (I32, [P, C.POINTER(C.c_double)]),
        "gridff_grid_save": (I32, [P, C.c_char_p]),
        "gridff_grid_load": (I32, [P, C.c_char_p, C.POINTER(P)]),
        "gridff_langevin": (I32, [P, P, P, I32, C.POINTER(LangevinParams), C.c_int]),
        "gridff_mlp_set_targets": (I32, [P, I32, P, P]),
        "gridff_mlp_train": (I32, [P, I32, I32, I32, P, I32, C.c_uint64, C.POINTER(TrainParams), P]),
        "gridff_rmsd_unique_xyz": (I32, [P, I32, I32, P, C.POINTER(C.c_double), F64, P, C.c_int]),
        "gridff_grid_destroy": (None, [P]),
        "gridff_replicas_create": (I32, [P, I32, C.POINTER(Molecule), I32, C.POINTER(C.c_int32), I32,
                                         F64, C.POINTER(P)]),
        "gridff_replicas_destroy": (None, [P]),
        "gridff_replicas_info": (I32, [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "gridff_set_state": (I32, [P, P, P, C.c_int]),
        "gridff_get_state": (I32, [P, P, P, C.c_int]),
        "gridff_get_positions": (I32, [P, P, C.c_int]),
        "gridff_get_fire_state": (I32, [P, P, P, P, P, P, P, C.c_int]),
        "gridff_get_last_eval": (I32, [P, P, P, C.c_int]),
        "gridff_eval": (I32, [P, P, P, C.c_int, P, P, P, P]),
        "gridff_fire_params_default": (None, [C.POINTER(FireParams)]),
        "gridff_relax": (I32, [P, P, P, I32, C.POINTER(FireParams), C.c_int, C.POINTER(RelaxResult)]),
        "gridff_run": (I32, [P, P, P, I32, C.POINTER(MDParams), C.c_int, P]),
        "gridff_probe_read_bandwidth": (I32, [P, P, C.c_size_t, I32, C.POINTER(C.c_double)]),
        "gridff_last_kernel_ms": (F64, [P]),
        "gridff_mlp_create": (I32, [P, I32, C.POINTER(C.c_int32), C.POINTER(P)]),
        "gridff_mlp_destroy": (None, [P]),
        "gridff_mlp_num_params": (C.c_int64, [P]),
        "gridff_mlp_set_params": (I32, [P, P]),
        "gridff_mlp_get_params": (I32, [P, P, P]),
        "gridff_mlp_forward": (I32, [P, I32, P, P]),
        "gridff_mlp_train_step": (I32, [P, I32, I32, P, P, P, C.POINTER(TrainParams), C.POINTER(C.c_float),
                                        C.c_int]),
        "gridff_mlp_propose": (I32, [P, P, P, I32, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "gridff_molecule_descriptor": (I32, [C.POINTER(Molecule), P]),
        "gridff_random_poses": (I32, [P, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double), F64, F64,
                                      F64]),
        "gridff_rmsd_unique": (I32, [P, I32, I32, P, C.POINTER(C.c_double), F64, P, C.c_int]),
        "gridff_set_launch_config": (I32, [P, C.POINTER(LaunchConfig)]),
        "gridff_get_launch_config": (I32, [P, C.c_int, C.POINTER(LaunchConfig)]),
        "gridff_tune": (I32, [P, P, P, C.POINTER(FireParams), I32, C.c_int, C.POINTER(LaunchConfig),
                              C.POINTER(TuneTrial), I32, C.POINTER(C.c_int32)]),
        "gridff_relax_graph_create": (I32, [P, P, P, I32, C.POINTER(FireParams), C.c_int, C.POINTER(P)]),
        "gridff_graph_launch": (I32, [P, C.POINTER(RelaxResult)]),
        "gridff_graph_destroy": (None, [P]),
        "gridff_template_rotors": (I32, [P, I32, C.POINTER(C.c_int32), P]),
        "gridff_build_poses": (I32, [P, P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int]),
        "gridff_pose_targets": (I32, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), P, P, C.c_int]),
        "gridff_lift": (I32, [P, C.c_double, C.c_int]),
        "gridff_eval_points": (I32, [P, P, C.c_int64, P, P, P, P, P, C.c_int]),
        "gridff_template_factors": (I32, [P, I32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()
EXPORTED = (
    "gridff_create", "gridff_destroy", "gridff_last_error", "gridff_stream", "gridff_set_abort",
    "gridff_grid_opts_default", "gridff_build_grid", "gridff_grid_from_coefs", "gridff_grid_info",
    "gridff_fit_coefs_noalloc",
    "gridff_grid_download_f64", "gridff_grid_destroy", "gridff_replicas_create",
    "gridff_replicas_destroy", "gridff_replicas_info", "gridff_set_state", "gridff_get_state",
    "gridff_get_positions", "gridff_get_fire_state", "gridff_get_last_eval", "gridff_eval", "gridff_fire_params_default",
    "gridff_relax", "gridff_run", "gridff_probe_read_bandwidth", "gridff_last_kernel_ms",
    "gridff_mlp_create", "gridff_mlp_destroy", "gridff_mlp_num_params", "gridff_mlp_set_params",
    "gridff_mlp_get_params", "gridff_mlp_forward", "gridff_mlp_train_step", "gridff_mlp_propose",
    "gridff_molecule_descriptor", "gridff_random_poses", "gridff_rmsd_unique",
    "gridff_set_launch_config", "gridff_get_launch_config", "gridff_tune", "gridff_relax_graph_create",
    "gridff_grid_storage", "gridff_grid_floor", "gridff_grid_save", "gridff_grid_load", "gridff_langevin", "gridff_rmsd_unique_xyz", "gridff_mlp_set_targets",
    "gridff_mlp_train",
    "gridff_graph_launch", "gridff_graph_destroy", "gridff_template_rotors", "gridff_build_poses",
    "gridff_pose_targets", "gridff_eval_points", "gridff_template_factors", "gridff_lift",
)
MAX_ROTORS = 12

KERNEL_RIGID_SUBWARP, KERNEL_RIGID_QUAD, KERNEL_FLEX_QUAD, KERNEL_FLEX_TERMS = 0, 1, 2, 3


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, is_device, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, False, None
    if _is_torch(a):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return C.c_void_p(a.data_ptr()), a.is_cuda, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), False, arr


class Context:
    """CUDA context of the library: device, stream, abort flag."""

    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        st = lib.gridff_create(int(device), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != OK:
            raise GridffError(st, f"gridff_create(device={device}) failed")
        self.h = h

    def check(self, st):
        if st != OK:
            raise GridffError(st, lib.gridff_last_error(self.h).decode())
        return st

    @property
    def stream(self):
        return lib.gridff_stream(self.h)

    def set_abort(self, value=True):
        lib.gridff_set_abort(self.h, int(bool(value)))

    def last_kernel_ms(self):
        return float(lib.gridff_last_kernel_ms(self.h))

    def probe_read_bandwidth(self, tensor, iters=50):
        out = C.c_double()
        self.check(lib.gridff_probe_read_bandwidth(self.h, C.c_void_p(tensor.data_ptr()),
                                                   tensor.numel() * tensor.element_size(), iters,
                                                   C.byref(out)))
        return out.value

    def close(self):
        if getattr(self, "h", None):
            lib.gridff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    def __init__(self, ctx: Context, handle):
        self.ctx, self.h = ctx, handle
        dims = (C.c_int32 * 3)(); org = (C.c_double * 3)(); sp = (C.c_double * 3)()
        ch = C.c_int32(); nb = C.c_size_t()
        ctx.check(lib.gridff_grid_info(handle, dims, org, sp, C.byref(ch), C.byref(nb)))
        self.dims, self.origin, self.spacing = tuple(dims), tuple(org), tuple(sp)
        self.channels, self.device_bytes = ch.value, nb.value
        st = C.c_int32(); sc = (C.c_float * 3)()
        ctx.check(lib.gridff_grid_storage(handle, C.byref(st), sc))
        self.storage, self.scales = st.value, tuple(sc)
        fl = C.c_double()
        ctx.check(lib.gridff_grid_floor(handle, C.byref(fl)))
        self.floor = fl.value
        # node planes below the floor
        self.ghost = int(round((self.floor - self.origin[2]) / self.spacing[2]))

    @property
    def n_channels(self):
        return bin(self.channels).count("1")

    def download_f64(self, what="coefs"):
        out = np.empty((self.n_channels,) + self.dims, np.float64)
        self.ctx.check(lib.gridff_grid_download_f64(self.h, 1 if what == "coefs" else 0,
                                                     out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def save(self, path):
        """gridff_grid_save: write the grid to a file."""
        self.ctx.check(lib.gridff_grid_save(self.h, os.fsencode(path)))

    def close(self):
        if getattr(self, "h", None):
            lib.gridff_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_grid(ctx: Context, sub, origin, length, spacing, channels=CH_C | CH_P | CH_L,
               alpha=1.5, rcut=17.0, ewald_tol=1e-10, ewald_rcut=12.0, keep_f64=False,
               storage=STORE_F32, ghost_below=0) -> Grid:
    """gridff_build_grid: substrate (object with xyz, q, R, eps, cell) -> Grid.
    `origin` is the floor; `ghost_below` node planes are added under it."""
    xyz = np.ascontiguousarray(sub.xyz, np.float64).ravel()
    q = np.ascontiguousarray(sub.q, np.float64)
    R = np.ascontiguousarray(sub.R, np.float64)
    eps = np.ascontiguousarray(sub.eps, np.float64)
    s = Substrate(len(q), xyz.ctypes.data_as(C.POINTER(C.c_double)), q.ctypes.data_as(C.POINTER(C.c_double)),
                  R.ctypes.data_as(C.POINTER(C.c_double)), eps.ctypes.data_as(C.POINTER(C.c_double)),
                  (C.c_double * 9)(*np.asarray(sub.cell, np.float64).ravel()))
    o = GridOpts()
    lib.gridff_grid_opts_default(C.byref(o))
    o.origin = (C.c_double * 3)(*origin)
    o.length = (C.c_double * 3)(*length)
    o.spacing, o.alpha, o.rcut = spacing, alpha, rcut
    o.ewald_tol, o.ewald_rcut, o.channels, o.keep_f64 = ewald_tol, ewald_rcut, channels, int(keep_f64)
    o.storage, o.ghost_below = storage, int(ghost_below)
    h = C.c_void_p()
    ctx.check(lib.gridff_build_grid(ctx.h, C.byref(s), C.byref(o), C.byref(h)))
    return Grid(ctx, h)


def load_grid(ctx: Context, path) -> Grid:
    """gridff_grid_load: a grid file written by Grid.save."""
    h = C.c_void_p()
    ctx.check(lib.gridff_grid_load(ctx.h, os.fsencode(path), C.byref(h)))
    return Grid(ctx, h)


def grid_from_coefs(ctx: Context, coefs, origin, spacing, channels, storage=STORE_F32) -> Grid:
    """gridff_grid_from_coefs: FP64 coefficients (C, nx, ny, nz) -> Grid."""
    c = np.ascontiguousarray(coefs, np.float64)
    dims = (C.c_int32 * 3)(*c.shape[1:])
    h = C.c_void_p()
    ctx.check(lib.gridff_grid_from_coefs(ctx.h, (C.c_double * 3)(*origin), (C.c_double * 3)(*spacing), dims,
                                         channels, c.ctypes.data_as(C.POINTER(C.c_double)), storage,
                                         C.byref(h)))
    return Grid(ctx, h)


def fit_coefs_noalloc(ctx: Context, values, coefs, flags: int = 0):
    """gridff_fit_coefs_noalloc on CUDA tensors: contiguous float64 of one
    shape (C, nx, ny, nz); returns the library's status."""
    for name, t in (("values", values), ("coefs", coefs)):
        if not _is_torch(t) or not t.is_cuda or t.ndim != 4:
            raise TypeError(f"{name} must be a 4-d CUDA tensor (C, nx, ny, nz)")
    if tuple(coefs.shape) != tuple(values.shape):
        raise TypeError("coefs must have the shape of values")
    pv, _, _ = _ptr(values, np.float64)
    pc, _, _ = _ptr(coefs, np.float64)
    dims = (C.c_int32 * 3)(*values.shape[1:])
    return lib.gridff_fit_coefs_noalloc(ctx.h, pv, pc, dims, int(values.shape[0]), flags)


def _mol_struct(m, keep):
    def f32(a):
        arr = np.ascontiguousarray(np.asarray(a, np.float32).ravel())
        keep.append(arr)
        return arr.ctypes.data_as(C.c_void_p)

    def i32(a):
        arr = np.ascontiguousarray(np.asarray(a, np.int32).ravel())
        keep.append(arr)
        return arr.ctypes.data_as(C.c_void_p)

    return Molecule(m.n, f32(m.xyz), f32(m.q), f32(m.R), f32(m.eps), f32(m.mass),
                    len(m.bonds), i32(m.bonds), f32(m.bond_k), f32(m.bond_r0),
                    len(m.angles), i32(m.angles), f32(m.angle_k), f32(m.angle_cos0),
                    len(m.torsions), i32(m.torsions), f32(m.torsion_V), i32(m.torsion_n),
                    f32(m.torsion_cos_nphi0))


class Replicas:
    """gridff_replicas: n_rep replicas of molecule templates (rigid or flexible)."""

    def __init__(self, ctx: Context, templates, template_of, rigid=False, alpha=1.5):
        keep = []
        mols = (Molecule * len(templates))(*[_mol_struct(m, keep) for m in templates])
        tof = np.ascontiguousarray(template_of, np.int32)
        h = C.c_void_p()
        ctx.check(lib.gridff_replicas_create(ctx.h, len(templates), mols, len(tof),
                                             tof.ctypes.data_as(C.POINTER(C.c_int32)), int(bool(rigid)),
                                             float(alpha), C.byref(h)))
        self.ctx, self.h, self.rigid = ctx, h, bool(rigid)
        self.template_atoms = np.array([m.n for m in templates], np.int32)
        n_rep = C.c_int32(); n_at = C.c_int32()
        ctx.check(lib.gridff_replicas_info(h, C.byref(n_rep), C.byref(n_at), None))
        self.n_rep, self.n_atoms = n_rep.value, n_at.value
        off = np.empty(self.n_rep + 1, np.int32)
        ctx.check(lib.gridff_replicas_info(h, None, None, off.ctypes.data_as(C.POINTER(C.c_int32))))
        self.atom_offset = off

    @property
    def state_sizes(self):
        if self.rigid:
            return 7 * self.n_rep, 6 * self.n_rep
        return 3 * self.n_atoms, 3 * self.n_atoms

    def set_state(self, x, v=None, flags=0):
        px, dx, kx = _ptr(x, np.float32)
        pv, dv, kv = _ptr(v, np.float32)
        nx, nv = self.state_sizes
        if not dx and np.asarray(kx).size != nx:
            raise ValueError(f"x must have {nx} floats")
        if v is not None and not dv and np.asarray(kv).size != nv:
            raise ValueError(f"v must have {nv} floats")
        flags |= DEVICE_PTRS if dx else 0
        self.ctx.check(lib.gridff_set_state(self.h, px, pv, flags))

    def get_state(self):
        nx, nv = self.state_sizes
        x = np.empty(nx, np.float32); v = np.empty(nv, np.float32)
        self.ctx.check(lib.gridff_get_state(self.h, x.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p), 0))
        return x, v

    def positions(self):
        x = np.empty(3 * self.n_atoms, np.float32)
        self.ctx.check(lib.gridff_get_positions(self.h, x.ctypes.data_as(C.c_void_p), 0))
        return x.reshape(-1, 3)

    def fire_state(self):
        n = self.n_rep
        out = dict(dt=np.empty(n, np.float32), alpha=np.empty(n, np.float32), nplus=np.empty(n, np.int32),
                   status=np.empty(n, np.int32), steps=np.empty(n, np.int32), energy=np.empty(n, np.float64))
        p = {k: v.ctypes.data_as(C.c_void_p) for k, v in out.items()}
        self.ctx.check(lib.gridff_get_fire_state(self.h, p["dt"], p["alpha"], p["nplus"], p["status"],
                                                 p["steps"], p["energy"], 0))
        return out

    def last_eval(self):
        """(state, forces) of every replica's final evaluation in the last
        relaxation (gridff_get_last_eval): rigid (n_rep, 7) poses and
        (n_rep, 6) total force + body torque; flexible (n_atoms, 3) each."""
        nx, nf = self.state_sizes
        x = np.empty(nx, np.float32); f = np.empty(nf, np.float32)
        self.ctx.check(lib.gridff_get_last_eval(self.h, x.ctypes.data_as(C.c_void_p),
                                                f.ctypes.data_as(C.c_void_p), 0))
        if self.rigid:
            return x.reshape(-1, 7), f.reshape(-1, 6)
        return x.reshape(-1, 3), f.reshape(-1, 3)

    def set_launch_config(self, cfg=None, **kw):
        """Fix the relaxation layout (None: the library's heuristic).  Keyword
        fields are set over the current layout; a layout given shared-memory
        slots or another kernel this way drops the global stencil cache unless
        cache_global is among the keywords."""
        if cfg is None and not kw:
            self.ctx.check(lib.gridff_set_launch_config(self.h, None))
            return
        c = self.launch_config() if cfg is None else cfg
        for k, v in kw.items():
            setattr(c, k, v)
        if "cache_global" not in kw and (kw.get("cache_slots", 0) > 0 or kw.get("kernel", KERNEL_FLEX_TERMS)
                                          != KERNEL_FLEX_TERMS):
            c.cache_global = 0
        self.ctx.check(lib.gridff_set_launch_config(self.h, C.byref(c)))

    def launch_config(self, use_grid=True) -> LaunchConfig:
        c = LaunchConfig()
        self.ctx.check(lib.gridff_get_launch_config(self.h, int(bool(use_grid)), C.byref(c)))
        return c

    def random_poses(self, seed, origin_xy, tile_xy, z_lo, z_hi, z_floor):
        """Random rigid starting poses drawn on the device (gridff_random_poses)."""
        o = (C.c_double * 2)(*origin_xy); t = (C.c_double * 2)(*tile_xy)
        self.ctx.check(lib.gridff_random_poses(self.h, C.c_uint64(seed), o, t, float(z_lo), float(z_hi),
                                               float(z_floor)))

    def template_factors(self, t=0) -> np.ndarray:
        """(n_atoms, 3) grid factors (Q, P, L) of template t as the kernels
        use them (gridff_template_factors)."""
        n = int(self.template_atoms[t])
        out = np.empty(3 * n, np.float32)
        st = lib.gridff_template_factors(self.h, int(t), out.ctypes.data_as(C.c_void_p))
        if st != OK:
            raise GridffError(st, "gridff_template_factors")
        return out.reshape(n, 3)

    def template_rotors(self, t=0) -> np.ndarray:
        """(n_rot, 4) reference quadruples (a, b, c, d) of template t's
        rotatable bonds in build order (gridff_template_rotors)."""
        n = C.c_int32(0)
        q = np.zeros(4 * MAX_ROTORS, np.int32)
        st = lib.gridff_template_rotors(self.h, int(t), C.byref(n), q.ctypes.data_as(C.c_void_p))
        if st != OK:
            raise GridffError(st, "gridff_template_rotors")
        return q[:4 * n.value].reshape(-1, 4)

    def build_poses(self, poses, origin_xy=None, tile_xy=None):
        """Set the state from (n_rep, 19) poses: centre, quaternion, torsions
        (gridff_build_poses; flexible replicas through the pose builder)."""
        o = (C.c_double * 2)(*origin_xy) if origin_xy is not None else None
        t = (C.c_double * 2)(*tile_xy) if tile_xy is not None else None
        if getattr(poses, "is_cuda", False):
            self.ctx.check(lib.gridff_build_poses(self.h, C.c_void_p(poses.contiguous().data_ptr()), o, t,
                                                  DEVICE_PTRS))
            return
        if hasattr(poses, "numpy"):
            poses = poses.numpy()
        p = np.ascontiguousarray(poses, np.float32).reshape(self.n_rep, MLP_OUT)
        self.ctx.check(lib.gridff_build_poses(self.h, p.ctypes.data_as(C.c_void_p), o, t, 0))

    def lift(self, z_floor):
        """gridff_lift: raise replicas whose lowest atom is below z_floor."""
        self.ctx.check(lib.gridff_lift(self.h, float(z_floor), 0))

    def pose_targets(self, origin_xy=None, tile_xy=None):
        """(targets (n_rep, 19), torsion masks (n_rep, 12)) of the current
        state (gridff_pose_targets)."""
        o = (C.c_double * 2)(*origin_xy) if origin_xy is not None else None
        t = (C.c_double * 2)(*tile_xy) if tile_xy is not None else None
        T = np.empty((self.n_rep, MLP_OUT), np.float32)
        M = np.empty((self.n_rep, MAX_ROTORS), np.float32)
        self.ctx.check(lib.gridff_pose_targets(self.h, o, t, T.ctypes.data_as(C.c_void_p),
                                               M.ctypes.data_as(C.c_void_p), 0))
        return T, M

    def rmsd_unique(self, poses, tile_xy, threshold=0.1, tmpl=0):
        """dup_of[i]: first earlier pose within `threshold` RMSD, else -1."""
        p = np.ascontiguousarray(poses, np.float32).reshape(-1, 7)
        out = np.empty(len(p), np.int32)
        t = (C.c_double * 2)(*tile_xy)
        self.ctx.check(lib.gridff_rmsd_unique(self.h, tmpl, len(p), p.ctypes.data_as(C.c_void_p), t,
                                              float(threshold), out.ctypes.data_as(C.c_void_p), 0))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib.gridff_replicas_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval(ctx: Context, grid, reps: Replicas, flags=0, out=None):
    """gridff_eval -> (E per replica, F (n_atoms, 3), per-atom grid energy, status)."""
    if out is not None:                    # device tensors: (E, F, Eatom, status)
        E, F, Ea, S = out
        ctx.check(lib.gridff_eval(ctx.h, grid.h if grid else None, reps.h, flags | DEVICE_PTRS,
                                  C.c_void_p(E.data_ptr()), C.c_void_p(F.data_ptr()),
                                  C.c_void_p(Ea.data_ptr()) if Ea is not None else None,
                                  C.c_void_p(S.data_ptr()) if S is not None else None))
        return out
    E = np.empty(reps.n_rep, np.float64)
    F = np.empty(3 * reps.n_atoms, np.float32)
    Ea = np.empty(reps.n_atoms, np.float32)
    S = np.empty(reps.n_rep, np.int32)
    ctx.check(lib.gridff_eval(ctx.h, grid.h if grid else None, reps.h, flags,
                              E.ctypes.data_as(C.c_void_p), F.ctypes.data_as(C.c_void_p),
                              Ea.ctypes.data_as(C.c_void_p), S.ctypes.data_as(C.c_void_p)))
    return E, F.reshape(-1, 3), Ea, S


def eval_points(ctx: Context, grid, xyz, qpl, out=None, flags=0):
    """gridff_eval_points -> (E (n,), F (n, 3), status (n,)).  With `out`
    = (E, F, status) device tensors and device-tensor inputs, nothing is
    copied (status may be None)."""
    if out is not None:
        E, F, S = out
        ctx.check(lib.gridff_eval_points(ctx.h, grid.h, int(E.numel()), C.c_void_p(xyz.data_ptr()),
                                         C.c_void_p(qpl.data_ptr()), C.c_void_p(E.data_ptr()),
                                         C.c_void_p(F.data_ptr()), C.c_void_p(S.data_ptr()) if S is not None else None,
                                         flags | DEVICE_PTRS))
        return out
    x = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    q = np.ascontiguousarray(qpl, np.float32).reshape(-1, 3)
    n = len(x)
    E = np.empty(n, np.float32)
    F = np.empty((n, 3), np.float32)
    S = np.empty(n, np.int32)
    ctx.check(lib.gridff_eval_points(ctx.h, grid.h, n, x.ctypes.data_as(C.c_void_p), q.ctypes.data_as(C.c_void_p),
                                     E.ctypes.data_as(C.c_void_p), F.ctypes.data_as(C.c_void_p),
                                     S.ctypes.data_as(C.c_void_p), flags))
    return E, F, S


def fire_params(**kw) -> FireParams:
    p = FireParams()
    lib.gridff_fire_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def relax(ctx: Context, grid, reps: Replicas, nsteps: int, params: FireParams | None = None,
          flags: int = 0, check: bool = True):
    """gridff_relax -> (status, RelaxResult)."""
    res = RelaxResult()
    st = lib.gridff_relax(ctx.h, grid.h if grid else None, reps.h, int(nsteps),
                          C.byref(params) if params is not None else None, flags, C.byref(res))
    if check and st not in (OK,):
        ctx.check(st)
    return st, res


def run(ctx: Context, grid, reps: Replicas, nsteps: int, dt: float, record_every: int = 0,
        flags: int = 0, clock_budget_s: float = 0.0, check: bool = True):
    """gridff_run -> (status, energy trace (n_records, n_rep) or None)."""
    p = MDParams(float(dt), int(record_every), float(clock_budget_s))
    trace = None
    tp = None
    if record_every > 0:
        trace = np.empty((nsteps // record_every + 1, reps.n_rep), np.float64)
        tp = trace.ctypes.data_as(C.c_void_p)
    st = lib.gridff_run(ctx.h, grid.h if grid else None, reps.h, int(nsteps), C.byref(p), flags, tp)
    if check and st != OK:
        ctx.check(st)
    return st, trace


MLP_OUT = 19
MLP_NO_UPDATE = 1


def train_params(lr=1e-3, tile=(1.0, 1.0), **kw) -> TrainParams:
    """gridff_train_params with the library defaults (Adam 0.9/0.999/1e-8,
    w_q = 1, w_t = 0.25) and the given learning rate and tile."""
    p = TrainParams(lr, 0.9, 0.999, 1e-8, 1.0, 0.25, (C.c_double * 2)(*tile))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def molecule_descriptor(mol) -> np.ndarray:
    """64-float descriptor of a molecule template (gridff_molecule_descriptor)."""
    keep = []
    m = _mol_struct(mol, keep)
    out = np.zeros(64, np.float32)
    st = lib.gridff_molecule_descriptor(C.byref(m), out.ctypes.data_as(C.c_void_p))
    if st != 0:
        raise GridffError(st, "gridff_molecule_descriptor: bad molecule")
    return out


class MLP:
    """gridff_mlp: the pose-proposal network (FP32 master parameters,
    bfloat16 tensor-core GEMMs)."""

    def __init__(self, ctx: Context, sizes):
        sz = np.ascontiguousarray(sizes, np.int32)
        h = C.c_void_p()
        ctx.check(lib.gridff_mlp_create(ctx.h, len(sz) - 1, sz.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(h)))
        self.ctx, self.h, self.sizes = ctx, h, tuple(int(s) for s in sz)
        self.n_params = int(lib.gridff_mlp_num_params(h))

    @staticmethod
    def flatten(Ws, bs) -> np.ndarray:
        return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in zip(Ws, bs)]).astype(np.float32)

    def unflatten(self, flat):
        Ws, bs, o = [], [], 0
        for i, j in zip(self.sizes[:-1], self.sizes[1:]):
            Ws.append(flat[o:o + i * j].reshape(j, i)); o += i * j
            bs.append(flat[o:o + j]); o += j
        return Ws, bs

    def set_params(self, Ws, bs):
        flat = self.flatten(Ws, bs)
        if flat.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {flat.size}")
        self.ctx.check(lib.gridff_mlp_set_params(self.h, flat.ctypes.data_as(C.c_void_p)))

    def get_params(self):
        p = np.empty(self.n_params, np.float32); g = np.empty(self.n_params, np.float32)
        self.ctx.check(lib.gridff_mlp_get_params(self.h, p.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p)))
        return p, g

    def forward(self, x):
        x = np.ascontiguousarray(x, np.float32)
        if x.ndim != 2 or x.shape[1] != self.sizes[0]:
            raise ValueError(f"x must be (rows, {self.sizes[0]})")
        y = np.empty((x.shape[0], MLP_OUT), np.float32)
        self.ctx.check(lib.gridff_mlp_forward(self.h, x.shape[0], x.ctypes.data_as(C.c_void_p),
                                              y.ctypes.data_as(C.c_void_p)))
        return y

    def train_step(self, x, targets, K, params: TrainParams, tors_mask=None, update=True):
        x = np.ascontiguousarray(x, np.float32)
        t = np.ascontiguousarray(targets, np.float32)
        B = t.shape[0]
        if x.shape != (B * K, self.sizes[0]) or t.shape != (B, MLP_OUT):
            raise ValueError("x must be (n_targets*K, n_in) and targets (n_targets, 19)")
        m = None if tors_mask is None else np.ascontiguousarray(tors_mask, np.float32)
        loss = C.c_float()
        self.ctx.check(lib.gridff_mlp_train_step(
            self.h, B, K, x.ctypes.data_as(C.c_void_p), t.ctypes.data_as(C.c_void_p),
            None if m is None else m.ctypes.data_as(C.c_void_p), C.byref(params), C.byref(loss),
            0 if update else MLP_NO_UPDATE))
        return loss.value

    def set_targets(self, targets, tors_mask=None):
        t = np.ascontiguousarray(targets, np.float32)
        if t.ndim != 2 or t.shape[1] != MLP_OUT:
            raise ValueError("targets must be (n, 19)")
        m = None if tors_mask is None else np.ascontiguousarray(tors_mask, np.float32)
        self.ctx.check(lib.gridff_mlp_set_targets(self.h, len(t), t.ctypes.data_as(C.c_void_p),
                                                  None if m is None else m.ctypes.data_as(C.c_void_p)))

    def train(self, steps, n_targets, K, descriptor, seed, params: TrainParams):
        """gridff_mlp_train: `steps` device-side steps; returns the losses."""
        d = np.ascontiguousarray(descriptor, np.float32)
        out = np.empty(steps, np.float32)
        self.ctx.check(lib.gridff_mlp_train(self.h, int(steps), int(n_targets), int(K), d.ctypes.data_as(C.c_void_p),
                                            d.size, C.c_uint64(seed), C.byref(params),
                                            out.ctypes.data_as(C.c_void_p)))
        return out

    def propose(self, reps: Replicas, descriptor, seed, origin_xy, tile_xy):
        d = np.ascontiguousarray(descriptor, np.float32)
        o = (C.c_double * 2)(*origin_xy); t = (C.c_double * 2)(*tile_xy)
        self.ctx.check(lib.gridff_mlp_propose(self.h, reps.h, d.ctypes.data_as(C.c_void_p), d.size,
                                              C.c_uint64(seed), o, t))

    def close(self):
        if getattr(self, "h", None):
            lib.gridff_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune(ctx: Context, grid, reps: Replicas, params: FireParams | None = None, trial_steps: int = 20,
         flags: int = 0, max_trials: int = 64):
    """gridff_tune -> (best LaunchConfig, [trial dicts])."""
    best = LaunchConfig()
    trials = (TuneTrial * max_trials)()
    n = C.c_int32()
    ctx.check(lib.gridff_tune(ctx.h, grid.h if grid else None, reps.h,
                              C.byref(params) if params is not None else None, int(trial_steps), flags,
                              C.byref(best), trials, max_trials, C.byref(n)))
    log = [dict(t.cfg.as_dict(), atom_evals_per_s=t.atom_evals_per_s, ms=t.ms)
           for t in trials[:min(n.value, max_trials)]]
    return best, log


class RelaxGraph:
    """gridff_relax_graph_create: one relaxation captured in a CUDA graph."""

    def __init__(self, ctx: Context, grid, reps: Replicas, nsteps: int, params: FireParams | None = None,
                 flags: int = 0):
        h = C.c_void_p()
        ctx.check(lib.gridff_relax_graph_create(ctx.h, grid.h if grid else None, reps.h, int(nsteps),
                                                C.byref(params) if params is not None else None, flags,
                                                C.byref(h)))
        self.ctx, self.h = ctx, h

    def launch(self, wait: bool = True, check: bool = True):
        if not wait:
            self.ctx.check(lib.gridff_graph_launch(self.h, None))
            return OK, None
        res = RelaxResult()
        st = lib.gridff_graph_launch(self.h, C.byref(res))
        if check and st != OK:
            self.ctx.check(st)
        return st, res

    def close(self):
        if getattr(self, "h", None):
            lib.gridff_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def langevin(ctx: Context, grid, reps: Replicas, nsteps: int, dt: float, temperature: float, gamma: float,
             seed: int, step0: int = 0, flags: int = 0, clock_budget_s: float = 0.0, check: bool = True):
    """gridff_langevin (BAOAB) -> status."""
    p = LangevinParams(dt, temperature, gamma, C.c_uint64(seed), step0, clock_budget_s)
    st = lib.gridff_langevin(ctx.h, grid.h if grid else None, reps.h, int(nsteps), C.byref(p), flags)
    if check and st != OK:
        ctx.check(st)
    return st


def rmsd_unique_xyz(ctx: Context, xyz, tile_xy, threshold=0.1):
    """dup_of for n structures of one molecule, xyz (n, n_atoms, 3)."""
    x = np.ascontiguousarray(xyz, np.float32)
    n, na = x.shape[0], x.shape[1]
    out = np.empty(n, np.int32)
    t = (C.c_double * 2)(*tile_xy)
    ctx.check(lib.gridff_rmsd_unique_xyz(ctx.h, na, n, x.ctypes.data_as(C.c_void_p), t, float(threshold),
                                         out.ctypes.data_as(C.c_void_p), 0))
    return out
