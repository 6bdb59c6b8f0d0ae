"""Precision tiers of the stored coefficients (FP32, FP16, BF16 with
per-channel scales) on a neutral fcc(111) slab (Pauli and London channels
only): every tier's interpolated energy differs from the FP32 tier by at
most the tier's rounding bound, and each tier's error against the FP64
pairwise reference is reported."""
import numpy as np
import pytest

from oracle import bspline as obs
from oracle import precision as oprec
from oracle import substrate as osub
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as ge
    ge.build()
    from paper_2508_15522_gb300 import gridff
    return gridff


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


@pytest.fixture(scope="module")
def setup(G, ctx):
    sub = synth.fcc111_slab(ncell=4, layers=3, grid_height=8.0)
    box = synth.grid_box_for(sub, 0.1, height=8.0)
    grids = {t: G.build_grid(ctx, sub, box.origin, box.length, box.spacing, channels=G.CH_P | G.CH_L,
                             keep_f64=(t == "f32"), storage=oprec.STORAGE[t]) for t in ("f32", "f16", "bf16")}
    mol = synth.random_flexible_molecule(24, 4, 17)
    n_rep = 40
    x = synth.flexible_positions(mol, sub, n_rep, seed=18, h_lo=2.5, h_hi=4.0, min_clear=2.0)
    return sub, box, grids, mol, n_rep, x.reshape(-1, 3).astype(np.float32)


def test_tier_records_and_scales(G, setup):
    sub, box, grids, mol, n_rep, pts = setup
    coefs = grids["f32"].download_f64("coefs")
    n_rec = np.prod(np.array(grids["f32"].dims) + [3, 3, 2])
    for t, width in (("f32", 8), ("f16", 4), ("bf16", 4)):
        g = grids[t]
        assert g.storage == oprec.STORAGE[t]
        assert g.device_bytes == n_rec * width           # two slots {P, L}
        _, scales = oprec.quantize(coefs, t)
        assert np.array_equal(np.array(g.scales[1:], np.float64), scales)
        assert g.scales[0] == 1.0


def test_tier_error_bounds_and_pairwise_error(G, ctx, setup):
    sub, box, grids, mol, n_rep, pts = setup
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    reps.set_state(pts.ravel())
    out = {t: G.eval(ctx, grids[t], reps, flags=G.NO_INTRA) for t in grids}
    coefs = grids["f32"].download_f64("coefs")
    Q = np.tile(mol.q, n_rep); R = np.tile(mol.R, n_rep); eps = np.tile(mol.eps, n_rep)
    P_, L_ = osub.factor_params(R, eps, 1.5)
    # |factor| x sum |c| w per atom: the scale of the rounding error
    fa, _, _ = obs.eval_grid(np.abs(coefs), box.origin, grids["f32"].spacing, pts.astype(np.float64))
    e_abs = np.abs(P_) * fa[:, 0] + np.abs(L_) * fa[:, 1]
    E_ref, F_ref = osub.pairwise_reference(pts.astype(np.float64), Q, R, eps, sub)
    Ea32 = out["f32"][2].astype(np.float64)
    report = {}
    for t in ("f16", "bf16"):
        Ea = out[t][2].astype(np.float64)
        _, scales = oprec.quantize(coefs, t)
        floor = (np.abs(P_) * scales[0] + np.abs(L_) * scales[1]) * 2.0 ** (oprec.TIERS[t][1] - 1)
        bound = oprec.unit_roundoff(t) * e_abs + floor + 2e-6 * (1 + np.abs(Ea32))
        assert np.all(np.abs(Ea - Ea32) <= bound), t
    for t in grids:
        Ea, F = out[t][2].astype(np.float64), out[t][1].astype(np.float64)
        report[t] = (np.abs(Ea - E_ref).max(), np.abs(F - F_ref).max())
    print("tier: max |dE| per atom (eV), max |dF| (eV/A) vs FP64 pairwise:", report)
    # ordering of the tiers' errors against the reference
    assert report["f32"][0] <= report["f16"][0] <= report["bf16"][0] + 1e-12
    reps.close()


def test_rigid_relaxation_runs_on_every_tier(G, ctx, setup):
    """The sub-warp relaxation kernel reads every record kind: the relaxed
    energies of the three tiers agree to the BF16 bound."""
    sub, box, grids, mol0, n_rep, pts = setup
    mol = synth.c24h8o6_core()
    com, quat = synth.rigid_poses(mol, sub, 64, seed=19)
    pose = np.concatenate([com, quat], 1).astype(np.float32).ravel()
    E = {}
    for t, g in grids.items():
        reps = G.Replicas(ctx, [mol], [0] * 64, rigid=True)
        reps.set_state(pose)
        G.relax(ctx, g, reps, 20, G.fire_params(f_conv=0.0))
        E[t] = reps.fire_state()["energy"]
        reps.close()
    assert np.all(np.isfinite(E["f16"])) and np.all(np.isfinite(E["bf16"]))
    assert np.abs(E["f16"] - E["f32"]).max() < 1e-2
    assert np.abs(E["bf16"] - E["f32"]).max() < 5e-2
