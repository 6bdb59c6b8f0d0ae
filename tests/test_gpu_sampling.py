"""GPU parity of the random starting poses and the RMSD uniqueness filter."""
import numpy as np
import pytest

from oracle import sampling
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu

TILE = (11.28, 11.28)


@pytest.fixture(scope="module")
def gf():
    from paper_2508_15522_gb300 import gridff
    return gridff


@pytest.fixture(scope="module")
def ctx(gf):
    c = gf.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n_rep", [1, 333])
def test_random_poses_match_oracle(gf, ctx, n_rep):
    mol = synth.c24h8o6_core()
    reps = gf.Replicas(ctx, [mol], np.zeros(n_rep, np.int32), rigid=True)
    seed = 0xDEADBEEF12345
    reps.random_poses(seed, (-1.0, 2.0), TILE, 4.0, 6.0, 1.5)
    x, v = reps.get_state()
    ref = sampling.random_poses(mol.xyz.astype(np.float64), n_rep, seed, (-1.0, 2.0), TILE, 4.0, 6.0, 1.5)
    # FP32 trigonometry and products against FP64: a few ulps of 10 A
    assert np.max(np.abs(x.reshape(n_rep, 7) - ref)) < 2e-5
    assert np.all(v == 0)
    reps.close()


def _cluster_set(mol, seed):
    """Relaxed-like poses with near copies (RMSD 0.02 A), far variants
    (RMSD >= 0.3 A) and tile images, shuffled."""
    g = synth.rng(seed)
    com, quat = synth.rigid_poses(mol, synth.rocksalt_slab(a=5.64, ncell=8, layers=3, charge=0.7), 60, seed)
    base = np.concatenate([com, quat], 1)
    out = [base]
    near = base.copy(); near[:, :3] += g.normal(0, 0.02 / np.sqrt(3), (60, 3)); out.append(near)
    far = base.copy(); far[:, :3] += g.normal(0, 0.5, (60, 3)); out.append(far)
    img = base.copy(); img[:, 0] += TILE[0] * g.integers(-2, 3, 60); img[:, 1] -= TILE[1]; out.append(img)
    P = np.concatenate(out)
    P = P[g.permutation(len(P))]
    return P.astype(np.float32)


def test_rmsd_unique_matches_oracle(gf, ctx):
    mol = synth.c24h8o6_core()
    body = mol.xyz.astype(np.float64)
    reps = gf.Replicas(ctx, [mol], [0], rigid=True)
    P = _cluster_set(mol, 91)
    ref = sampling.dup_of(body, P.astype(np.float64), TILE, 0.1)
    # no pair sits within 10 % of the threshold, so FP32 cannot flip a decision
    for i in range(len(P)):
        for j in range(i):
            assert abs(sampling.rmsd(body, P[i], P[j], TILE) - 0.1) > 0.01
    got = reps.rmsd_unique(P, TILE, 0.1)
    assert got.tolist() == ref.tolist()
    assert 60 <= np.sum(ref == -1) < len(P)
    assert reps.rmsd_unique(P[:1], TILE, 0.1).tolist() == [-1]
    assert reps.rmsd_unique(np.zeros((0, 7), np.float32), TILE, 0.1).size == 0
    reps.close()


def test_mlp_proposals_beat_random_starts(gf, ctx):
    """Ablation: relaxations started from the trained proposal network land in
    the best-known minimum far more often than random starts, and still
    cover most of its symmetry-equivalent copies."""
    from paper_2508_15522_gb300 import sampling as S
    sub = synth.rocksalt_slab(a=5.64, ncell=8, layers=3, charge=0.7)
    box = synth.grid_box_for(sub, 0.1, height=20.0)
    grid = gf.build_grid(ctx, sub, box.origin, box.length, box.spacing)
    mol = synth.c24h8o6_core()
    surf = S.Surface((0.0, 0.0), (5.64, 5.64), sub.z_top + 3.0, sub.z_top + 5.0, sub.z_top + 2.0)
    sp = S.Sampler(ctx, grid, mol, surf, n_rep=2048, nsteps=2000)
    runs, targets = [], []
    for k in range(8):
        runs.append(sp.random_batch(100 + k))
        targets.append(sp.targets())
    E = np.concatenate([b.energy for b in runs]); P = np.concatenate([b.poses for b in runs])
    C = np.concatenate([b.converged for b in runs])
    T = np.concatenate(targets)
    e_best = E[C].min()
    h = C & (E <= e_best + 0.01)
    n_unique = len(sp.unique(P[h], E[h]))
    net = S.new_network(ctx, T[h], seed=3)
    S.train_on_device(net, sp.desc, T[h], surf, 3000, batch=256, K=8, lr=1e-3, seed=4)
    rnd = [sp.random_batch(200 + k) for k in range(2)]
    mlp = [sp.proposal_batch(net, 300 + k) for k in range(2)]
    frac_r = np.mean([S.hits(b, e_best).mean() for b in rnd])
    frac_m = np.mean([S.hits(b, e_best).mean() for b in mlp])
    Pm = np.concatenate([b.poses[S.hits(b, e_best)] for b in mlp])
    Em = np.concatenate([b.energy[S.hits(b, e_best)] for b in mlp])
    assert frac_m > 3 * frac_r > 0
    assert len(sp.unique(Pm, Em)) >= n_unique // 2
    net.close(); sp.close(); grid.close()


def test_one_network_learns_two_molecules_by_their_descriptors(gf, ctx):
    """The descriptor input across molecules: one network is trained on the
    best-known poses of two different rigid molecules, every training row
    carrying its own molecule's descriptor.  For each molecule, proposals
    made with its descriptor relax into its best-known minimum far more often
    than random starts, and more often than proposals made with the other
    molecule's descriptor."""
    import time
    from paper_2508_15522_gb300 import sampling as S
    sub = synth.rocksalt_slab(a=5.64, ncell=8, layers=3, charge=0.7)
    box = synth.grid_box_for(sub, 0.1, height=20.0)
    grid = gf.build_grid(ctx, sub, box.origin, box.length, box.spacing, ghost_below=8)
    surf = S.Surface((0.0, 0.0), (5.64, 5.64), sub.z_top + 3.0, sub.z_top + 5.0, sub.z_top + 2.0)
    mols = [synth.c24h8o6_core(), synth.rigid_molecule(24, 2024)]
    sps = [S.Sampler(ctx, grid, m, surf, n_rep=2048, nsteps=2000) for m in mols]
    e_best, T = [], []
    for sp in sps:
        runs, tg = [], []
        for k in range(8):
            runs.append(sp.random_batch(500 + k))
            tg.append(sp.targets())
        E = np.concatenate([b.energy for b in runs])
        C = np.concatenate([b.converged for b in runs])
        e_best.append(E[C].min())
        T.append(np.concatenate(tg)[C & (E <= E[C].min() + 0.01)])
    assert min(len(t) for t in T) > 20
    descs = [sp.desc for sp in sps]
    assert np.abs(descs[0] - descs[1]).max() > 0.1
    net = S.new_network(ctx, np.concatenate(T), seed=3)
    g = np.random.default_rng(4)
    tp = gf.train_params(lr=1e-3, tile=surf.tile_xy)
    B, K = 256, 8
    for _ in range(3000):
        m = g.integers(0, 2, B)
        targets = np.stack([T[j][g.integers(0, len(T[j]))] for j in m])
        x = np.concatenate([np.repeat(np.stack([descs[j] for j in m]), K, 0),
                            g.standard_normal((B * K, S.N_NOISE)).astype(np.float32)], 1)
        net.train_step(x, targets, K, tp)

    def hit_fraction(j, how, seed):
        sp = sps[j]
        if how == "random":
            b = sp.random_batch(seed)
        else:
            net.propose(sp.reps, descs[j if how == "own" else 1 - j], seed, surf.origin_xy, surf.tile_xy)
            b = sp._relax(time.perf_counter())
        return S.hits(b, e_best[j]).mean()

    for j in range(2):
        own = np.mean([hit_fraction(j, "own", 900 + k) for k in range(2)])
        other = np.mean([hit_fraction(j, "other", 910 + k) for k in range(2)])
        rnd = np.mean([hit_fraction(j, "random", 920 + k) for k in range(2)])
        print(f"molecule {j}: hit fraction own descriptor {own:.3f}, other {other:.3f}, random {rnd:.3f}")
        assert own > 3 * rnd and own > 1.5 * other
    net.close()
    for sp in sps:
        sp.close()
    grid.close()
