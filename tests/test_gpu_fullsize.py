"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times: the 113 x 113 x 200 NaCl grid with 4096 rigid C24H8O6
replicas (sampled replicas against the oracle), and the oracle-size
configuration (57 x 57 x 100 grid at 0.2 A, 64 flexible 10-atom chains,
500 FIRE iterations)."""
import numpy as np
import pytest

from oracle import dynamics as odyn
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


def test_rigid_4096_replicas_full_grid_sampled(G, ctx):
    sub = synth.rocksalt_slab(a=5.64, ncell=8, layers=3, charge=0.7)
    box = synth.grid_box_for(sub, 0.1, height=20.0)
    mol = synth.c24h8o6_core()
    com, quat = synth.rigid_poses(mol, sub, 4096, seed=1002)
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True)
    assert grid.dims == (113, 113, 200)
    c32 = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    reps = G.Replicas(ctx, [mol], [0] * 4096, rigid=True)
    cfg = reps.launch_config()
    assert cfg.kernel == G.KERNEL_RIGID_SUBWARP and cfg.lanes_per_replica == 16
    body = mol.xyz.astype(np.float32).astype(np.float64)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), grid.origin, grid.spacing, mol, intra=False)
    sample = np.r_[0:8, 2040:2048, 4088:4096]          # first, middle and last waves
    for nsteps, tol in ((1, 2e-6), (10, 1e-4)):
        reps.set_state(pose.ravel())
        st, res = G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0))
        assert res.atom_evals == 4096 * mol.n * nsteps
        x, _ = reps.get_state()
        x = x.reshape(4096, 7)[sample]
        ref = odyn.fire_rigid(pose[sample, :3].astype(np.float64), pose[sample, 3:].astype(np.float64),
                              np.zeros((len(sample), 3)), np.zeros((len(sample), 3)), body, mol.mass, fn, nsteps,
                              odyn.FireParams(f_conv=0.0))
        xg = odyn.rigid_positions(x[:, :3].astype(np.float64), x[:, 3:].astype(np.float64), body)
        xo = odyn.rigid_positions(ref["com"], ref["quat"], body)
        assert np.abs(xg - xo).max() <= tol, nsteps
    reps.close()


def test_oracle_size_configuration(G, ctx):
    sub = synth.rocksalt_slab(a=5.64, ncell=4, layers=2, charge=0.7)
    box = synth.grid_box_for(sub, 0.2, height=20.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True)
    assert grid.dims == (57, 57, 100)
    c32 = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    mol = synth.chain_molecule()
    x0 = synth.flexible_positions(mol, sub, 64, seed=1001).astype(np.float32)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), grid.origin, grid.spacing, mol)
    reps = G.Replicas(ctx, [mol], [0] * 64)
    reps.set_state(x0.ravel())
    G.relax(ctx, grid, reps, 20, G.fire_params(f_conv=0.0))
    x, _ = reps.get_state()
    ref = odyn.fire_flexible(x0.astype(np.float64), np.zeros(x0.shape), mol.mass, fn, 20, odyn.FireParams(f_conv=0.0))
    assert np.abs(x.reshape(ref["x"].shape) - ref["x"]).max() <= 2e-4
    # 500 FIRE iterations: every converged replica is an oracle minimum with the reported energy
    reps.set_state(x0.ravel())
    st, res = G.relax(ctx, grid, reps, 500, G.fire_params(f_conv=1e-3))
    fs = reps.fire_state()
    conv = (fs["status"] & G.REP_CONVERGED) != 0
    assert conv.sum() > 0
    x, _ = reps.get_state()
    E, F, _ = fn(x.reshape(64, mol.n, 3).astype(np.float64))
    assert (np.sqrt((F[conv] ** 2).sum((1, 2))) < 1e-3 + 5e-4).all()
    assert np.allclose(fs["energy"][conv], E[conv], atol=1e-4 * mol.n)
    reps.close()
