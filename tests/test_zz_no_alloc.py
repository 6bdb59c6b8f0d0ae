"""The allocation-free coefficient fit (gridff_fit_coefs_noalloc).

Callers that cannot allocate device memory at fit time (memory reserved by
another allocator, or loops that cannot afford cudaFree's synchronisation)
use this entry point.  It must give the same coefficients as the fit inside
gridff_build_grid, call after call, although all calls share one fixed
device table.  This file is collected last so that a failure here does not
stop the other GPU tests in a run that stops at the first failure.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import bspline as obs
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_COEF = 1e-7    # relative to the largest coefficient, as for the grid-build parity


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2508_15522_gb300 import gridff
    ctx = gridff.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    return gridff, ctx, torch


def _reference(G, ctx, spacing, height):
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, spacing, height=height)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True)
    return grid.download_f64("values"), grid.download_f64("coefs")


def test_noalloc_fit_matches_build_grid_on_two_calls_in_a_row(env):
    G, ctx, torch = env
    cases = [_reference(G, ctx, 0.6, 3.0), _reference(G, ctx, 0.45, 4.2)]
    assert cases[0][0].shape != cases[1][0].shape      # the shared table is rebuilt per call
    for vals, ref in cases:
        dv = torch.from_numpy(vals).cuda()
        dc = torch.full_like(dv, float("nan"))
        st = G.fit_coefs_noalloc(ctx, dv, dc)
        assert st == G.OK, G.lib.gridff_last_error(ctx.h).decode()
        got = dc.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL_COEF * np.abs(ref).max()
        # and against the oracle's exact fit of the same node values (dense
        # 1D solves of the collocation system, independent of the GPU fit)
        exact = obs.fit_exact(vals)
        assert np.abs(got - exact).max() <= TOL_COEF * np.abs(exact).max()
    # in place (values == coefs) gives the same result
    vals, ref = cases[0]
    d = torch.from_numpy(vals.copy()).cuda()
    assert G.fit_coefs_noalloc(ctx, d, d) == G.OK
    assert np.abs(d.cpu().numpy() - ref).max() <= TOL_COEF * np.abs(ref).max()


def test_noalloc_fit_rejects_sizes_beyond_its_table(env):
    G, ctx, torch = env
    dims = (C.c_int32 * 3)(8, 8, 5000)
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = G.lib.gridff_fit_coefs_noalloc(ctx.h, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), dims, 1, 0)
    assert st == G.EINVAL
    assert "4..4096" in G.lib.gridff_last_error(ctx.h).decode()


def test_noalloc_fit_rejects_host_and_overlapping_arrays(env):
    """Arguments that would make the line solves touch memory outside the
    caller's device arrays are refused before any kernel runs."""
    G, ctx, torch = env
    dims = (C.c_int32 * 3)(4, 4, 4)
    host = np.zeros(64, np.float64)
    dev = torch.zeros(64 + 8, dtype=torch.float64, device="cuda")
    hp = C.c_void_p(host.ctypes.data)
    st = G.lib.gridff_fit_coefs_noalloc(ctx.h, hp, C.c_void_p(dev.data_ptr()), dims, 1, 0)
    assert st == G.EINVAL and "not memory of device" in G.lib.gridff_last_error(ctx.h).decode()
    a, b = C.c_void_p(dev.data_ptr()), C.c_void_p(dev.data_ptr() + 8 * 8)   # ranges overlap by 56 values
    st = G.lib.gridff_fit_coefs_noalloc(ctx.h, a, b, dims, 1, 0)
    assert st == G.EINVAL and "overlap" in G.lib.gridff_last_error(ctx.h).decode()
    with pytest.raises(TypeError):
        G.fit_coefs_noalloc(ctx, torch.zeros(1, 4, 4, 4, dtype=torch.float64), dev[:64].view(1, 4, 4, 4))
    with pytest.raises(TypeError):
        G.fit_coefs_noalloc(ctx, dev[:64].view(1, 4, 4, 4), dev[:64].view(1, 4, 4, 4).float())
