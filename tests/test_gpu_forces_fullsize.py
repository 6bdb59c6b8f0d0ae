"""Energies and forces of the relaxation kernels, element by element, at the
workloads' full sizes and in the launch configurations the benchmark times,
against the FP32 oracle mirror at the absolute gates |dF| <= 1e-4 eV/A per
atom and |dE| <= 1e-5 eV per atom.

The kernels keep, for every replica, the state and forces of the final
evaluation of a relaxation (gridff_get_last_eval); the energy of that
evaluation is the one gridff_get_fire_state reports.  Rigid replicas give
the total force and the body-frame torque, so their tolerances are the
per-atom gates summed over the molecule (triangle inequality):
|dF_tot| <= n 1e-4 eV/A, |dtau| <= 1e-4 sum_i |b_i| eV, |dE| <= n 1e-5 eV.
Flexible replicas give every atom's force (grid + intramolecular terms).

Relaxation lengths: 1 iteration (the record is the start state), 200 (the
stencil cache serves most evaluations; the rigid launch runs on the
time-sliced schedule, whose replicas are split between two warps) and, for
the rigid workload, the 2000 iterations of one benchmark step.  The same
grid and poses also pin gridff_eval and gridff_eval_points on the real
0.1 A grid at the absolute gates.
"""
import numpy as np
import pytest

from oracle import dynamics as odyn
from oracle import grid as ogrid
from oracle import intra as ointra
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F = 1e-4     # eV/A per atom
TOL_E = 1e-5     # eV per atom
CHUNK = 8192     # points per oracle call (bounds the oracle's memory)


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
def nacl(G, ctx):
    """The 113 x 113 x 200 FP32 grid of the 8 x 8 x 3 NaCl(001) slab with
    8 ghost planes below its floor, as the benchmark builds it, and its
    coefficients rounded to FP32 (what the kernels read)."""
    sub = synth.rocksalt_slab(a=5.64, ncell=8, layers=3, charge=0.7)
    box = synth.grid_box_for(sub, 0.1, height=20.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, keep_f64=True, ghost_below=8)
    assert grid.dims == (113, 113, 208) and grid.ghost == 8
    c32 = grid.download_f64("coefs").astype(np.float32).astype(np.float64)
    yield sub, box, grid, c32
    grid.close()


def oracle_grid_ef(c32, grid, pts, Q, R, eps):
    """Per-point FP32-mirror energy and force, in chunks."""
    E = np.empty(len(pts)); F = np.empty((len(pts), 3)); below = np.empty(len(pts), bool)
    for a in range(0, len(pts), CHUNK):
        b = min(a + CHUNK, len(pts))
        e, f, bl = ogrid.grid_energy_forces(c32, ("C", "P", "L"), grid.origin, grid.spacing, pts[a:b], Q[a:b],
                                            R[a:b], eps[a:b], dtype=np.float32, ghost=grid.ghost)
        E[a:b], F[a:b], below[a:b] = e, f, bl
    return E, F, below


def oracle_rigid(c32, grid, mol, pose):
    """Energy, total force and body torque of rigid poses (n_rep, 7) from
    the oracle's per-atom FP32-mirror values at R(q) b + c."""
    body = mol.xyz.astype(np.float32).astype(np.float64)
    n_rep = len(pose)
    x = odyn.rigid_positions(pose[:, :3].astype(np.float64), pose[:, 3:].astype(np.float64), body)
    E, F, _ = oracle_grid_ef(c32, grid, x.reshape(-1, 3), np.tile(mol.q, n_rep), np.tile(mol.R, n_rep),
                             np.tile(mol.eps, n_rep))
    Ft, tau = odyn.rigid_reduce(F.reshape(n_rep, mol.n, 3), pose[:, 3:].astype(np.float64), body)
    return E.reshape(n_rep, mol.n).sum(1), Ft, tau


def test_rigid_bench_workload_energy_force_torque(G, ctx, nacl):
    """All 4096 replicas of the benchmark workload (38-atom C24H8O6 core),
    in the benchmark's launch configuration: energy, total force and torque
    of the final evaluation after 1, 200 and 2000 FIRE iterations."""
    sub, box, grid, c32 = nacl
    mol = synth.c24h8o6_core()
    n_rep = 4096
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=1002)
    pose0 = np.concatenate([com, quat], 1).astype(np.float32)
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    cfg = reps.launch_config()
    assert cfg.kernel == G.KERNEL_RIGID_SUBWARP and cfg.lanes_per_replica == 16
    body = mol.xyz.astype(np.float32).astype(np.float64)
    tol_tau = TOL_F * np.linalg.norm(body, axis=1).sum()
    for nsteps in (1, 200, 2000):
        reps.set_state(pose0.ravel())
        st, res = G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0))
        assert res.atom_evals == n_rep * mol.n * nsteps
        xl, fl = reps.last_eval()
        E = reps.fire_state()["energy"]
        if nsteps == 1:
            assert np.array_equal(xl, pose0)          # the first evaluation is at the start pose
        assert np.isfinite(xl).all() and np.isfinite(fl).all()
        Eo, Fo, To = oracle_rigid(c32, grid, mol, xl)
        dE, dF, dT = np.abs(E - Eo).max(), np.abs(fl[:, :3] - Fo).max(), np.abs(fl[:, 3:] - To).max()
        print(f"rigid, {nsteps} iterations: max|dE| {dE:.2e} eV, max|dF_tot| {dF:.2e} eV/A, "
              f"max|dtau| {dT:.2e} eV; max|F_tot| {np.abs(Fo).max():.2f} eV/A")
        assert dE <= TOL_E * mol.n, nsteps
        assert dF <= TOL_F * mol.n, nsteps
        assert dT <= tol_tau, nsteps
    reps.close()


def test_rigid_eval_on_real_grid_per_atom(G, ctx, nacl):
    """gridff_eval of 512 benchmark poses: every atom's grid energy and force
    against the oracle at the absolute gates."""
    sub, box, grid, c32 = nacl
    mol = synth.c24h8o6_core()
    n_rep = 512
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=1002)
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    reps.set_state(pose.ravel())
    E, F, Ea, S = G.eval(ctx, grid, reps)
    x = reps.positions().astype(np.float64)
    Eo, Fo, _ = oracle_grid_ef(c32, grid, x, np.tile(mol.q, n_rep), np.tile(mol.R, n_rep),
                               np.tile(mol.eps, n_rep))
    print("eval per atom: max|dF|", np.abs(F - Fo).max(), "max|dE|", np.abs(Ea - Eo).max())
    assert np.abs(F - Fo).max() <= TOL_F
    assert np.abs(Ea - Eo).max() <= TOL_E
    reps.close()


def test_eval_points_on_real_grid(G, ctx, nacl):
    """gridff_eval_points at 200 000 uniform points of the interpolation
    workload (tile x [z0 + 2, z0 + 8] A, i.e. 3-9 A above the top ions)
    against the oracle at the absolute gates; and 4 000 points in the first
    five cells above the grid floor (1.0-1.5 A above the top ions), where
    the Pauli wall puts |E| up to about 40 eV and |F| up to about 120 eV/A
    on an atom.  FP32 carries about 7 significant digits, so there the gates
    are applied relative to the magnitude (|dF| <= 1e-4 max(1, |F|), the
    same for E), and the absolute figures are printed."""
    sub, box, grid, c32 = nacl
    mol = synth.c24h8o6_core()
    reps = G.Replicas(ctx, [mol], [0], rigid=True)
    qpl = reps.template_factors(0)
    for zband, n, absolute in (((2.0, 8.0), 200_000, True), ((0.0, 0.5), 4000, False)):
        pts = synth.uniform_points(n, box, 31, zband=zband).astype(np.float32)
        k = np.arange(len(pts)) % mol.n
        Eo, Fo, below = oracle_grid_ef(c32, grid, pts.astype(np.float64), mol.q[k], mol.R[k], mol.eps[k])
        for flags, name in ((0, "direct"), (G.POINTS_BINNED, "binned")):
            E, F, S = G.eval_points(ctx, grid, pts, qpl[k], flags=flags)
            dF, dE = np.abs(F - Fo).max(), np.abs(E - Eo).max()
            print(f"eval_points ({name}), z0 + {zband} A: max|dF| {dF:.2e} eV/A (max|F| {np.abs(Fo).max():.2f}), "
                  f"max|dE| {dE:.2e} eV (max|E| {np.abs(Eo).max():.2f})")
            if absolute:
                assert dF <= TOL_F and dE <= TOL_E
            else:
                assert (np.abs(F - Fo) <= TOL_F * np.maximum(1.0, np.abs(Fo))).all()
                assert (np.abs(E - Eo) <= TOL_E * np.maximum(1.0, np.abs(Eo))).all()
            assert not below.any() and not (S & G.REP_BELOW).any()
    reps.close()


def _uneven(G, ctx, sub):
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
    return mols, tof, reps, x0


@pytest.mark.parametrize("wpb,gcache", [(8, 0), (2, 0), (8, 1)])
def test_uneven_batch_per_atom_forces(G, ctx, nacl, wpb, gcache):
    """The uneven batch (16384 flexible replicas of 10-120 atoms) in the
    unique-term layout with the work queue: per-atom forces (grid +
    intramolecular) and per-replica energies of the final evaluation after
    1 and 200 iterations, on 64 replicas that span the sizes (the largest
    and smallest templates, both ends of the batch).  Atoms that a
    relaxation has pushed below the grid floor (flagged BELOW: the field
    there is the clamped continuation of the lowest cells, with forces of
    tens of eV/A) are held to the gate relative to the force's magnitude,
    as the eval test holds points in the first cells above the floor; every
    other atom to the absolute gate."""
    sub, box, grid, c32 = nacl
    mols, tof, reps, x0 = _uneven(G, ctx, sub)
    off = reps.atom_offset
    sizes = np.array([m.n for m in mols])[tof]
    order = np.argsort(sizes, kind="stable")
    sample = sorted(set(order[np.linspace(0, len(order) - 1, 60).astype(int)].tolist()) | {0, 1, 16382, 16383})
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=wpb, cache_slots=0, queue=1,
                           cache_global=gcache)
    for nsteps in (1, 200):
        reps.set_state(x0.ravel())
        G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0), check=False)
        xl, fl = reps.last_eval()
        E = reps.fire_state()["energy"]
        if nsteps == 1:
            assert np.array_equal(xl, x0)
        worst_f = worst_e = worst_below = 0.0
        n_below = 0
        for r in sample:
            m = mols[tof[r]]
            x = xl[off[r]:off[r + 1]].astype(np.float64)
            Eg, Fg, _ = oracle_grid_ef(c32, grid, x, m.q, m.R, m.eps)
            Ei, Fi = ointra.energy_forces(x[None], m)
            Fo = Fg + Fi[0]
            below = x[:, 2] < grid.floor
            gate = np.where(below, TOL_F * np.maximum(1.0, np.abs(Fo).max(1)), TOL_F)
            dFa = np.abs(fl[off[r]:off[r + 1]] - Fo).max(1)
            dF = dFa[~below].max(initial=0.0)
            Eo = Eg.sum() + Ei[0]
            dE = abs(E[r] - Eo)
            gate_e = TOL_E * (max(m.n, abs(Eo)) if below.any() else m.n)
            worst_f, worst_e = max(worst_f, dF), max(worst_e, dE / m.n)
            if below.any():
                n_below += int(below.sum())
                worst_below = max(worst_below, float((dFa[below] / np.maximum(1.0, np.abs(Fo[below]).max(1))).max()))
            if (dFa > gate).any():
                import torch
                a = int(np.argmax(dFa / gate))
                xt = torch.tensor(x, dtype=torch.float32, requires_grad=True)
                (g32,) = torch.autograd.grad(ointra.energy(xt[None], m).sum(), xt)
                print(f"replica {r} atom {a}: |dF| {dFa[a]:.2e}, z - floor {x[a, 2] - grid.floor:.3f} A, "
                      f"|F_grid| {np.linalg.norm(Fg[a]):.2f}, |F_intra| {np.linalg.norm(Fi[0, a]):.2f}, "
                      f"FP32 autograd intra vs FP64 {np.abs(-g32.numpy()[a] - Fi[0, a]).max():.2e}")
                for t in ("bond", "angle", "torsion", "nonbonded"):
                    print("  ", t, np.linalg.norm(ointra.energy_forces(x[None], m, terms=(t,))[1][0, a]))
            assert (dFa <= gate).all(), (r, m.n, nsteps, dF)
            assert dE <= gate_e, (r, m.n, nsteps, dE)
        print(f"uneven batch, {wpb} warps per block, global stencil cache {gcache}, {nsteps} iterations: max|dF| {worst_f:.2e} eV/A "
              f"(atoms above the floor), max|dE|/atom {worst_e:.2e} eV; {n_below} sampled atoms below the floor, "
              f"max |dF|/max(1, |F|) there {worst_below:.2e}")
    reps.close()


@pytest.fixture(scope="module")
def fcc(G, ctx):
    sub = synth.fcc111_slab(a=4.08, ncell=12, layers=4)
    box = synth.grid_box_for(sub, 0.05, height=20.0)
    grid32 = G.build_grid(ctx, sub, box.origin, box.length, box.spacing, channels=G.CH_P | G.CH_L, keep_f64=True,
                          ghost_below=8)
    yield sub, grid32, grid32.download_f64("coefs")
    grid32.close()


@pytest.mark.parametrize("tier", ["f32", "f16", "bf16"])
def test_fcc111_workload_energy_force_torque(G, ctx, fcc, tier):
    """The fcc(111) precision workload (231 x 200 x 400 grid, P and L
    channels, 65536 rigid 24-atom replicas): energy, total force and torque
    of the final evaluation after 1 and 200 iterations on 2048 replicas from
    both ends and the middle, against the oracle on the tier's own
    (quantised) coefficients."""
    from oracle import precision as oprec
    sub, grid32, coefs = fcc
    mol = synth.rigid_molecule(24, 2024)
    n_rep = 65536
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=2025)
    pose0 = np.concatenate([com, quat], 1).astype(np.float32)
    grid = grid32 if tier == "f32" else G.grid_from_coefs(ctx, coefs, grid32.origin, grid32.spacing,
                                                          G.CH_P | G.CH_L, storage=oprec.STORAGE[tier])
    cq, _ = oprec.quantize(coefs, tier)
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    body = mol.xyz.astype(np.float32).astype(np.float64)
    sample = np.r_[0:512, 32512:33536, 65024:65536]
    for nsteps in (1, 200):
        reps.set_state(pose0.ravel())
        st, res = G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0))
        xl, fl = reps.last_eval()
        E = reps.fire_state()["energy"]
        p = xl[sample]
        x = odyn.rigid_positions(p[:, :3].astype(np.float64), p[:, 3:].astype(np.float64), body)
        ns = len(sample)
        Eo, Fo, _ = ogrid.grid_energy_forces(cq, ("P", "L"), grid32.origin, grid32.spacing, x.reshape(-1, 3),
                                             np.tile(mol.q, ns), np.tile(mol.R, ns), np.tile(mol.eps, ns),
                                             dtype=np.float32, ghost=grid32.ghost)
        Ft, tau = odyn.rigid_reduce(Fo.astype(np.float64).reshape(ns, mol.n, 3), p[:, 3:].astype(np.float64), body)
        Eo = Eo.astype(np.float64).reshape(ns, mol.n).sum(1)
        dE, dF, dT = np.abs(E[sample] - Eo).max(), np.abs(fl[sample, :3] - Ft).max(), np.abs(fl[sample, 3:] - tau).max()
        print(f"fcc(111) {tier}, {nsteps} iterations: max|dE| {dE:.2e}, max|dF_tot| {dF:.2e}, max|dtau| {dT:.2e}")
        assert dE <= TOL_E * mol.n
        assert dF <= TOL_F * mol.n
        assert dT <= TOL_F * np.linalg.norm(body, axis=1).sum()
    reps.close()
    if grid is not grid32:
        grid.close()
