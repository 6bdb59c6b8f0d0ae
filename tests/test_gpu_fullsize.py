"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times: the 113 x 113 x 200 NaCl grid with 4096 rigid C24H8O6
replicas (sampled replicas against the oracle; the time-sliced and queued
schedules of a long launch bit for bit), the uneven batch of 16384 flexible
replicas (sampled), the fcc(111) precision workload with 65536 rigid
replicas on its 231 x 200 x 400 grid in FP32 and FP16 (sampled), and the
oracle-size configuration (57 x 57 x 100 grid at 0.2 A, 64 flexible 10-atom
chains, 500 FIRE iterations)."""
import numpy as np
import pytest

from oracle import dynamics as odyn
from oracle import precision as oprec
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
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True, ghost_below=8)
    assert grid.dims == (113, 113, 208)
    c32 = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    reps = G.Replicas(ctx, [mol], [0] * 4096, rigid=True)
    cfg = reps.launch_config()
    assert cfg.kernel == G.KERNEL_RIGID_SUBWARP and cfg.lanes_per_replica == 16
    body = mol.xyz.astype(np.float32).astype(np.float64)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), grid.origin, grid.spacing, mol, intra=False, ghost=grid.ghost)
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
    # a launch long enough for the time-sliced schedule (2048 warp tasks on
    # fewer resident warps): equal bit for bit to the whole-task queue
    out = []
    for mode in (0, 1):
        reps.set_launch_config(G.LaunchConfig(kernel=cfg.kernel, lanes_per_replica=cfg.lanes_per_replica,
                                              warps_per_block=cfg.warps_per_block, cache_slots=cfg.cache_slots,
                                              queue=mode))
        reps.set_state(pose.ravel())
        st, res = G.relax(ctx, grid, reps, 200, G.fire_params(f_conv=0.0))
        assert res.atom_evals == 4096 * mol.n * 200
        x, v = reps.get_state()
        out.append((x, v, reps.fire_state()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    for k in ("dt", "alpha", "nplus", "status", "steps", "energy"):
        assert np.array_equal(out[0][2][k], out[1][2][k]), k
    reps.close()


def test_uneven_batch_full_size_sampled(G, ctx):
    sub = synth.rocksalt_slab(a=5.64, ncell=8, layers=3, charge=0.7)
    box = synth.grid_box_for(sub, 0.1, height=20.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True, ghost_below=8)
    c32 = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    mols, tof = synth.uneven_batch(16384, 256, 77)
    reps = G.Replicas(ctx, mols, tof)
    x0 = np.zeros((reps.n_atoms, 3), np.float32)
    off = reps.atom_offset
    for k, m in enumerate(mols):
        idx = np.where(tof == k)[0]
        if len(idx):
            P = synth.flexible_positions(m, sub, len(idx), seed=5000 + k)
            for j, r in enumerate(idx):
                x0[off[r]:off[r + 1]] = P[j]
    sizes = np.array([m.n for m in mols])
    # sampled replicas: the largest and smallest templates, first and last replicas
    sample = sorted({int(np.argmax(sizes[tof])), int(np.argmin(sizes[tof])), 0, 1, 8191, 16383})
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=2, cache_slots=0, queue=1)
    reps.set_state(x0.ravel())
    G.relax(ctx, grid, reps, 20, G.fire_params(f_conv=0.0), check=False)
    x, _ = reps.get_state()
    x = x.reshape(-1, 3)
    for r in sample:
        m = mols[tof[r]]
        fn = odyn.make_force_fn(c32, ("C", "P", "L"), grid.origin, grid.spacing, m, ghost=grid.ghost)
        ref = odyn.fire_flexible(x0[off[r]:off[r + 1]][None].astype(np.float64), np.zeros((1, m.n, 3)), m.mass,
                                 fn, 20, odyn.FireParams(f_conv=0.0))
        assert np.abs(x[off[r]:off[r + 1]] - ref["x"][0]).max() <= 2e-4, (r, m.n)
    reps.close(); grid.close()


@pytest.mark.parametrize("tier", ["f32", "f16"])
def test_fcc111_precision_workload_full_size_sampled(G, ctx, tier):
    sub = synth.fcc111_slab(a=4.08, ncell=12, layers=4)
    box = synth.grid_box_for(sub, 0.05, height=20.0)
    mol = synth.rigid_molecule(24, 2024)
    n_rep = 65536
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=2025)
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    grid32 = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, channels=G.CH_P | G.CH_L, keep_f64=True,
                          ghost_below=8)
    coefs = grid32.download_f64("coefs")
    grid = grid32 if tier == "f32" else G.grid_from_coefs(ctx, coefs, grid32.origin, grid32.spacing,
                                                          G.CH_P | G.CH_L, storage=oprec.STORAGE[tier])
    cq, _ = oprec.quantize(coefs, tier)
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    reps.set_state(pose.ravel())
    st, res = G.relax(ctx, grid, reps, 10, G.fire_params(f_conv=0.0))
    assert res.atom_evals == n_rep * mol.n * 10
    x, _ = reps.get_state()
    sample = np.r_[0:4, 32766:32770, 65532:65536]
    x = x.reshape(n_rep, 7)[sample]
    body = mol.xyz.astype(np.float32).astype(np.float64)
    fn = odyn.make_force_fn(cq, ("P", "L"), grid32.origin, grid32.spacing, mol, intra=False, ghost=grid32.ghost)
    ref = odyn.fire_rigid(pose[sample, :3].astype(np.float64), pose[sample, 3:].astype(np.float64),
                          np.zeros((len(sample), 3)), np.zeros((len(sample), 3)), body, mol.mass, fn, 10,
                          odyn.FireParams(f_conv=0.0))
    xg = odyn.rigid_positions(x[:, :3].astype(np.float64), x[:, 3:].astype(np.float64), body)
    assert np.abs(xg - odyn.rigid_positions(ref["com"], ref["quat"], body)).max() <= 1e-4
    reps.close()
    if grid is not grid32:
        grid.close()
    grid32.close()


def test_oracle_size_configuration(G, ctx):
    sub = synth.rocksalt_slab(a=5.64, ncell=4, layers=2, charge=0.7)
    box = synth.grid_box_for(sub, 0.2, height=20.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True, ghost_below=4)
    assert grid.dims == (57, 57, 104)
    c32 = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    mol = synth.chain_molecule()
    x0 = synth.flexible_positions(mol, sub, 64, seed=1001).astype(np.float32)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), grid.origin, grid.spacing, mol, ghost=grid.ghost)
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
