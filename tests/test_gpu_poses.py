"""GPU parity of the flexible-pose builder and its inverse
(gridff_template_rotors, gridff_build_poses, gridff_pose_targets, and
gridff_mlp_propose on flexible replicas) against oracle/poses.py."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import poses as P
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu

TILE = (11.28, 11.28)


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as ge
    ge.build()
    from paper_2508_15522_gb300 import gridff
    return gridff


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


def ring_molecule():
    """Five-ring with a three-atom tail and a hydrogen (the oracle pin's
    topology), generated geometry."""
    ring = [np.array([1.2 * math.cos(2 * math.pi * k / 5), 1.2 * math.sin(2 * math.pi * k / 5), 0.0])
            for k in range(5)]
    xyz = np.array(ring + [[2.6, 0.6, 0.3], [3.9, 0.2, -0.4], [5.2, 0.7, 0.2], [-0.4, 1.9, 0.8]])
    xyz[5:8] += ring[4] - ring[0]
    bonds = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (4, 5), (5, 6), (6, 7), (0, 8)]
    m = synth._finish(["C", "C", "C", "C", "C", "C", "C", "O", "H"], xyz, np.zeros(9), bonds)
    return m


@pytest.fixture(scope="module")
def mols():
    return [synth.chain_molecule(), synth.random_flexible_molecule(60, 10, 5),
            synth.random_flexible_molecule(120, 12, 7), ring_molecule(), synth.random_flexible_molecule(33, 12, 9)]


def test_rotors_match_oracle(G, ctx, mols):
    reps = G.Replicas(ctx, mols, list(range(len(mols))))
    for t, m in enumerate(mols):
        want = [r["quad"] for r in P.rotors(m.n, m.bonds, m.torsions)]
        got = [tuple(int(v) for v in q) for q in reps.template_rotors(t)]
        assert got == want, t
    assert len(reps.template_rotors(2)) == G.MAX_ROTORS
    reps.close()


def _random_poses(g, n, com_scale=5.0):
    P0 = np.zeros((n, 19), np.float32)
    P0[:, :3] = g.uniform(-com_scale, com_scale, (n, 3))
    P0[:, 3:7] = g.standard_normal((n, 4))
    P0[:, 7:] = g.uniform(-math.pi, math.pi, (n, 12))
    return P0


def test_builder_matches_oracle(G, ctx, mols):
    g = np.random.default_rng(11)
    tof = np.repeat(np.arange(len(mols)), 7).astype(np.int32)
    reps = G.Replicas(ctx, mols, tof)
    poses = _random_poses(g, len(tof))
    poses[3, 3:7] = 0.0                                  # zero quaternion: no rotation
    origin = (-1.0, 2.0)
    reps.build_poses(poses, origin, TILE)
    x, v = reps.get_state()
    assert np.all(v == 0)
    off = reps.atom_offset
    for r, t in enumerate(tof):
        m = mols[t]
        rot = P.rotors(m.n, m.bonds, m.torsions)
        com = poses[r, :3].astype(np.float64).copy()
        for a in range(2):
            com[a] = origin[a] + np.mod(com[a] - origin[a], TILE[a])
        ref = P.build(m.xyz, m.mass, rot, com, poses[r, 3:7].astype(np.float64),
                      poses[r, 7:7 + len(rot)].astype(np.float64))
        xr = x[3 * off[r]:3 * off[r + 1]].reshape(-1, 3)
        assert np.abs(xr - ref).max() < 2e-4, (r, np.abs(xr - ref).max())
        d = np.array([P.dihedral(*(xr[i].astype(np.float64) for i in q["quad"])) for q in rot])
        if len(rot):
            assert np.abs(np.angle(np.exp(1j * (d - poses[r, 7:7 + len(rot)])))).max() < 2e-4
    reps.close()


def test_targets_match_oracle_and_invert_the_builder(G, ctx, mols):
    g = np.random.default_rng(12)
    tof = np.repeat(np.arange(len(mols)), 5).astype(np.int32)
    reps = G.Replicas(ctx, mols, tof)
    poses = _random_poses(g, len(tof))
    reps.build_poses(poses)
    x, _ = reps.get_state()
    T, M = reps.pose_targets()
    off = reps.atom_offset
    for r, t in enumerate(tof):
        m = mols[t]
        rot = P.rotors(m.n, m.bonds, m.torsions)
        xr = x[3 * off[r]:3 * off[r + 1]].reshape(-1, 3).astype(np.float64)
        com, q, th = P.targets(m.xyz, m.mass, rot, xr)
        assert np.abs(T[r, :3] - com).max() < 1e-4
        assert np.abs(T[r, 3:7] - q).max() < 2e-4, (r, T[r, 3:7], q)
        k = len(rot)
        assert np.abs(np.angle(np.exp(1j * (T[r, 7:7 + k] - th)))).max() < 2e-4
        assert np.all(T[r, 7 + k:] == 0) and np.all(M[r, :k] == 1) and np.all(M[r, k:] == 0)
        # the inverse of the builder: the input pose up to the quaternion sign
        qin = poses[r, 3:7] / np.linalg.norm(poses[r, 3:7])
        assert abs(abs(float(np.dot(T[r, 3:7], qin))) - 1) < 1e-4
        assert np.abs(np.angle(np.exp(1j * (T[r, 7:7 + k] - poses[r, 7:7 + k])))).max() < 2e-4
    # rebuilding from the targets gives the same positions
    reps.build_poses(T)
    x2, _ = reps.get_state()
    assert np.abs(x2 - x).max() < 5e-4
    reps.close()


def test_rigid_poses_and_targets(G, ctx):
    mol = synth.c24h8o6_core()
    g = np.random.default_rng(13)
    reps = G.Replicas(ctx, [mol], [0] * 9, rigid=True)
    poses = _random_poses(g, 9)
    reps.build_poses(poses, (0.0, 0.0), TILE)
    x, v = reps.get_state()
    x = x.reshape(9, 7)
    assert np.all(v == 0)
    q = poses[:, 3:7] / np.linalg.norm(poses[:, 3:7], axis=1, keepdims=True)
    assert np.abs(x[:, 3:7] - q).max() < 1e-6
    assert np.all((x[:, :2] >= 0) & (x[:, :2] < np.array(TILE)))
    T, M = reps.pose_targets()
    assert np.abs(T[:, 3:7] - q * np.sign(q[:, :1])).max() < 1e-6
    assert np.all(M == 0) and np.all(T[:, 7:] == 0)
    assert len(reps.template_rotors(0)) == 0
    reps.close()


def test_propose_places_flexible_replicas_by_the_builder(G, ctx):
    mol = synth.random_flexible_molecule(40, 8, 21)
    n_rep = 64
    sizes = (80, 64, 64, 19)
    Ws, bs = synth.mlp_weights(sizes, 71)
    bs[-1][2] = 4.0
    net = G.MLP(ctx, sizes)
    net.set_params([W.astype(np.float32).astype(np.float64) for W in Ws], bs)
    desc = G.molecule_descriptor(mol)
    seed, origin = 0xABCDEF, (0.5, -0.5)
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    net.propose(reps, desc, seed, origin, TILE)
    x1, v1 = reps.get_state()
    assert np.all(v1 == 0)
    # the same network outputs through gridff_build_poses
    X = np.concatenate([np.tile(desc.astype(np.float64), (n_rep, 1)), omlp.counter_normal(seed, n_rep, 16)], 1)
    Y = net.forward(X.astype(np.float32))
    reps.build_poses(Y, origin, TILE)
    x2, _ = reps.get_state()
    assert np.abs(x1 - x2).max() < 1e-3
    net.close(); reps.close()


def test_flexible_learned_proposal_loop(G, ctx):
    """The learned-proposal loop on a flexible molecule, every step on the
    device: relax random starts, take the relaxed poses (with their torsions)
    as targets, train the network on them, propose and relax again."""
    from paper_2508_15522_gb300 import sampling as S
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, 0.2, height=10.0)
    grid = G.build_grid(ctx, sub, box.origin, box.length, box.spacing)
    mol = synth.random_flexible_molecule(24, 6, 31)
    n_rep = 256
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    reps.set_state(synth.flexible_positions(mol, sub, n_rep, seed=32).astype(np.float32).ravel())
    G.relax(ctx, grid, reps, 300, G.fire_params(f_conv=1e-3), check=False)
    tile = sub.tile
    T, M = reps.pose_targets((0.0, 0.0), tile)
    k = len(reps.template_rotors(0))
    assert k >= 3 and np.all(M[:, :k] == 1) and np.isfinite(T).all()
    net = S.new_network(ctx, T, seed=3)
    net.set_targets(T, M)
    desc = G.molecule_descriptor(mol)
    losses = net.train(300, 64, 4, desc, 5, G.train_params(lr=1e-3, tile=tile))
    assert np.isfinite(losses).all() and losses[-20:].mean() < losses[:20].mean()
    net.propose(reps, desc, 77, (0.0, 0.0), tile)
    x, _ = reps.get_state()
    assert np.isfinite(x).all()
    st, res = G.relax(ctx, grid, reps, 100, G.fire_params(f_conv=1e-3), check=False)
    assert st in (G.OK,) and res.atom_evals > 0
    net.close(); reps.close(); grid.close()


def test_lift_raises_only_replicas_below_the_floor(G, ctx):
    """gridff_lift: flexible replicas lowered below z_floor come back with
    their lowest atom at z_floor, shifted as a whole; rigid replicas move
    their centre so that the oracle's lowest atom of R(q) b + c is at z_floor;
    replicas above it are left bit for bit."""
    from oracle import dynamics as odyn
    mol = synth.random_flexible_molecule(20, 3, 31)
    sub = synth.rocksalt_slab(ncell=2)
    x = synth.flexible_positions(mol, sub, 6, seed=32).astype(np.float32)
    zf = float(sub.z_top + 1.8)                  # the starts keep 2 A: the odd replicas lie above it
    x[::2, :, 2] -= x[::2, :, 2].min(1, keepdims=True) - (zf - 1.3)    # replicas 0, 2, 4 start 1.3 A too low
    reps = G.Replicas(ctx, [mol], [0] * 6)
    reps.set_state(x.ravel())
    reps.lift(zf)
    y = reps.get_state()[0].reshape(x.shape)
    for r in range(6):
        if r % 2:
            assert np.array_equal(y[r], x[r])
        else:
            assert abs(y[r, :, 2].min() - zf) < 1e-5
            d = y[r] - x[r]
            assert np.abs(d[:, :2]).max() == 0 and np.ptp(d[:, 2]) < 1e-5
    core = synth.c24h8o6_core()
    com, quat = synth.rigid_poses(core, sub, 5, seed=33)
    com[:3, 2] = sub.z_top - 1.0                                      # three centres inside the slab
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    rig = G.Replicas(ctx, [core], [0] * 5, rigid=True)
    rig.set_state(pose.ravel())
    rig.lift(zf)
    p = rig.get_state()[0].reshape(5, 7)
    low = odyn.rigid_positions(p[:, :3].astype(np.float64), p[:, 3:].astype(np.float64),
                               core.xyz.astype(np.float32).astype(np.float64))[..., 2].min(1)
    assert np.abs(low[:3] - zf).max() < 1e-4 and np.array_equal(p[3:], pose[3:])
    assert np.array_equal(p[:3, [0, 1, 3, 4, 5, 6]], pose[:3, [0, 1, 3, 4, 5, 6]])
    rig.close(); reps.close()
