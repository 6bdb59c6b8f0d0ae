"""GPU parity of gridff_relax (FIRE) and gridff_run (NVE) against the oracle,
plus host-side failure detection (abort flag, clock budget, bad inputs)."""
import numpy as np
import pytest

from oracle import dynamics as odyn
from oracle import grid as ogrid
from oracle import intra as ointra
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
def small_field(G, ctx):
    """A smooth synthetic field over a 2a x 2a tile (random coefficients,
    small amplitude) shared by the parity tests."""
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, 0.25, height=8.0)
    n, h = ogrid.grid_dims(box.length, box.spacing)
    coefs = synth.random_coefficients(n, 3, seed=31, scale=(0.02, 0.01, 0.03))
    grid = G.grid_from_coefs(ctx, coefs, box.origin, h, 7)
    return sub, box, h, coefs.astype(np.float32).astype(np.float64), grid


def test_fire_flexible_first_steps_match_oracle(G, ctx, small_field):
    sub, box, h, c32, grid = small_field
    mol = synth.chain_molecule()
    n_rep = 37                                      # a ragged last block of warps
    x0 = synth.flexible_positions(mol, sub, n_rep, seed=32).astype(np.float32)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol)
    for nsteps, tol in ((1, 2e-6), (5, 2e-5), (20, 2e-4)):
        reps = G.Replicas(ctx, [mol], [0] * n_rep)
        reps.set_state(x0.ravel())
        st, res = G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0))
        assert res.atom_evals == n_rep * mol.n * nsteps
        x, v = reps.get_state()
        fs = reps.fire_state()
        ref = odyn.fire_flexible(x0.astype(np.float64), np.zeros(x0.shape), mol.mass, fn, nsteps,
                                 odyn.FireParams(f_conv=0.0))
        assert np.abs(x.reshape(ref["x"].shape) - ref["x"]).max() <= tol, nsteps
        assert np.allclose(fs["dt"], ref["dt"], rtol=1e-5)
        assert np.array_equal(fs["nplus"], ref["nplus"])
        assert (fs["steps"] == nsteps).all()


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_fire_rigid_first_steps_match_oracle(G, ctx, small_field, storage):
    from oracle import precision as oprec
    sub, box, h, c32, grid0 = small_field
    grid = G.grid_from_coefs(ctx, c32, box.origin, h, 7, storage=storage)
    c32 = oprec.quantize(c32, {0: "f32", 1: "f16", 2: "bf16"}[storage])[0]
    mol = synth.c24h8o6_core()
    n_rep = 33
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=33)
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    body = mol.xyz.astype(np.float32).astype(np.float64)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol, intra=False)
    for nsteps, tol in ((1, 2e-6), (10, 1e-4)):
        reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
        reps.set_state(pose.ravel())
        G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0))
        x, v = reps.get_state()
        x = x.reshape(n_rep, 7)
        ref = odyn.fire_rigid(pose[:, :3].astype(np.float64), pose[:, 3:].astype(np.float64),
                              np.zeros((n_rep, 3)), np.zeros((n_rep, 3)), body, mol.mass, fn, nsteps,
                              odyn.FireParams(f_conv=0.0))
        xg = odyn.rigid_positions(x[:, :3].astype(np.float64), x[:, 3:].astype(np.float64), body)
        xo = odyn.rigid_positions(ref["com"], ref["quat"], body)
        assert np.abs(xg - xo).max() <= tol, nsteps


def test_fire_relaxation_reaches_minima_by_oracle_forces(G, ctx):
    """Relax chains on a grid built from a real substrate; every replica the
    GPU reports converged has an oracle (FP64) force norm below the
    threshold plus the FP32 tolerance."""
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, 0.4, height=10.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True)
    coefs = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    mol = synth.chain_molecule()
    n_rep = 16
    x0 = synth.flexible_positions(mol, sub, n_rep, seed=34).astype(np.float32)
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    reps.set_state(x0.ravel())
    st, res = G.relax(ctx, grid, reps, 4000, G.fire_params(f_conv=1e-3))
    fs = reps.fire_state()
    conv = (fs["status"] & G.REP_CONVERGED) != 0
    assert conv.sum() >= n_rep // 2
    x, _ = reps.get_state()
    fn = odyn.make_force_fn(coefs, ("C", "P", "L"), grid.origin, grid.spacing, mol)
    E, F, _ = fn(x.reshape(n_rep, mol.n, 3).astype(np.float64))
    fnorm = np.sqrt((F * F).sum((1, 2)))
    assert (fnorm[conv] < 1e-3 + 5e-4).all(), fnorm[conv]
    assert np.allclose(fs["energy"][conv], E[conv], atol=1e-4 * mol.n)


def test_nve_flexible_steps_match_oracle(G, ctx, small_field):
    sub, box, h, c32, grid = small_field
    mol = synth.chain_molecule()
    n_rep = 12
    x0 = synth.flexible_positions(mol, sub, n_rep, seed=35).astype(np.float32)
    g = synth.rng(36)
    v0 = (0.002 * g.standard_normal(x0.shape)).astype(np.float32)
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    reps.set_state(x0.ravel(), v0.ravel())
    st, trace = G.run(ctx, grid, reps, 10, dt=0.5, record_every=5)
    x, v = reps.get_state()
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol)
    xr, vr, tr = odyn.nve_flexible(x0.astype(np.float64), v0.astype(np.float64), mol.mass, fn, 10, 0.5,
                                   record_every=5)
    assert np.abs(x.reshape(xr.shape) - xr).max() < 5e-5
    assert np.abs(trace - tr).max() < 1e-4 * mol.n


def test_nve_rigid_no_squish_matches_oracle_and_conserves_energy(G, ctx):
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, 0.2, height=10.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True)
    coefs = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    mol = synth.c24h8o6_core()
    n_rep = 8
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=37, h_lo=3.5, h_hi=4.5, min_clear=2.5)
    g = synth.rng(38)
    vel = np.concatenate([1e-3 * g.standard_normal((n_rep, 3)), 2e-4 * g.standard_normal((n_rep, 3))], 1)
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    reps.set_state(pose.ravel(), vel.astype(np.float32).ravel())
    st, trace = G.run(ctx, grid, reps, 20, dt=1.0, record_every=10)
    body = mol.xyz.astype(np.float32).astype(np.float64)
    fn = odyn.make_force_fn(coefs, ("C", "P", "L"), grid.origin, grid.spacing, mol, intra=False)
    c, q, v, w, tr = odyn.nve_rigid(pose[:, :3].astype(np.float64), pose[:, 3:].astype(np.float64),
                                    vel[:, :3].astype(np.float32).astype(np.float64),
                                    vel[:, 3:].astype(np.float32).astype(np.float64), body, mol.mass, fn,
                                    20, 1.0, record_every=10)
    x, _ = reps.get_state()
    x = x.reshape(n_rep, 7)
    xg = odyn.rigid_positions(x[:, :3].astype(np.float64), x[:, 3:].astype(np.float64), body)
    assert np.abs(xg - odyn.rigid_positions(c, q, body)).max() < 1e-4
    assert np.abs(trace - tr).max() < 1e-4
    # longer run: energy fluctuation stays small (symplectic, no drift)
    st, trace = G.run(ctx, grid, reps, 2000, dt=1.0, record_every=100)
    drift = np.abs(trace - trace[0]).max(0)
    assert drift.max() < 2e-3, drift


def test_abort_flag_stops_relax_with_status(G, ctx, small_field):
    sub, box, h, c32, grid = small_field
    mol = synth.chain_molecule()
    reps = G.Replicas(ctx, [mol], [0] * 8)
    reps.set_state(synth.flexible_positions(mol, sub, 8, seed=39).astype(np.float32).ravel())
    ctx.set_abort(True)
    try:
        st, res = G.relax(ctx, grid, reps, 100, G.fire_params(f_conv=0.0), check=False)
    finally:
        ctx.set_abort(False)
    assert st == G.EABORTED
    fs = reps.fire_state()
    assert ((fs["status"] & G.REP_ABORTED) != 0).all()
    assert (fs["steps"] == 0).all()
    # the context stays usable
    st, res = G.relax(ctx, grid, reps, 3, G.fire_params(f_conv=0.0))
    assert st == G.OK and res.atom_evals == 8 * mol.n * 3


def test_clock_budget_stops_long_run(G, ctx, small_field):
    sub, box, h, c32, grid = small_field
    mol = synth.chain_molecule()
    reps = G.Replicas(ctx, [mol], [0] * 4)
    reps.set_state(synth.flexible_positions(mol, sub, 4, seed=40).astype(np.float32).ravel())
    st, res = G.relax(ctx, grid, reps, 10_000_000, G.fire_params(f_conv=0.0, clock_budget_s=0.05), check=False)
    assert st == G.ESTEPLIMIT
    fs = reps.fire_state()
    assert ((fs["status"] & G.REP_STEPLIMIT) != 0).all()
    assert (fs["steps"] > 0).all() and (fs["steps"] < 10_000_000).all()


def test_nonfinite_and_invalid_inputs_are_reported(G, ctx, small_field):
    sub, box, h, c32, grid = small_field
    mol = synth.chain_molecule()
    reps = G.Replicas(ctx, [mol], [0] * 4)
    x = synth.flexible_positions(mol, sub, 4, seed=41).astype(np.float32)
    x[1, 2, 0] = np.nan
    x[2, :, 2] = sub.z_top - 3.0                      # below the grid
    b0, b1 = mol.bonds[0]
    x[3, b1] = x[3, b0]                               # a zero-length bond: its angles are undefined
    reps.set_state(x.ravel())
    E, F, Ea, S = G.eval(ctx, grid, reps)
    assert S[0] == 0
    assert S[1] & G.REP_NONFINITE
    assert S[2] & G.REP_BELOW
    assert S[3] & G.REP_NONFINITE
    st, res = G.relax(ctx, grid, reps, 10, G.fire_params(f_conv=0.0))
    fs = reps.fire_state()
    assert fs["status"][1] & G.REP_NONFINITE and fs["steps"][1] == 1
    assert fs["status"][3] & G.REP_NONFINITE and fs["steps"][3] == 1
    assert fs["steps"][0] == 10 and not fs["status"][0] & G.REP_NONFINITE   # the others go on
    bad = synth.chain_molecule()
    bad.bonds = bad.bonds.copy()
    bad.bonds[0] = (0, 0)                            # self bond
    with pytest.raises(G.GridffError) as e:
        G.Replicas(ctx, [bad], [0])
    assert e.value.status == G.EINVAL
