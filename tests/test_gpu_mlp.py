"""GPU parity of the pose-proposal MLP (tensor-core forward, winner-takes-all
backward, Adam, on-device proposal) against the float64 oracle with the
bfloat16 operand rounding mirrored."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = (80, 256, 256, 256, 19)
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


def _inputs(rows, seed):
    X = np.concatenate([np.tile(synth.rng(seed).random(64) * 0.5, (rows, 1)),
                        synth.noise(rows, 16, seed + 1)], 1)
    return X.astype(np.float32)


def _targets(B, seed):
    g = synth.rng(seed)
    T = np.zeros((B, 19))
    T[:, :2] = g.random((B, 2)) * TILE
    T[:, 2] = 3.0 + g.random(B)
    q = g.standard_normal((B, 4))
    T[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    T[:, 7:] = g.uniform(-np.pi, np.pi, (B, 12))
    mask = (g.random((B, 12)) < 0.5).astype(np.float64)
    return T.astype(np.float32), mask.astype(np.float32)


def _close(a, b, rel):
    """max |a - b| <= rel * max |b| (error relative to the tensor's scale)."""
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return np.max(np.abs(a - b)) <= rel * max(np.max(np.abs(b)), 1e-30)


# Tolerance: operands are bfloat16 on both sides, so the products agree
# exactly; what differs is the FP32 accumulation order (~1e-6 relative) and,
# through it, an occasional different bfloat16 rounding of a hidden
# activation (2^-8 relative on one of 256 terms of the next layer).  2e-3 of
# the tensor's scale bounds both with a wide margin and is below the 4e-3
# gap between the mirrored and the unrounded float64 network, so a missing
# rounding step fails it, as does a transposed operand or a dropped bias.
REL = 2e-3


@pytest.mark.parametrize("rows", [1, 37, 300])
def test_forward_matches_oracle(gf, ctx, rows):
    Ws, bs = synth.mlp_weights(SIZES, 21)
    net = gf.MLP(ctx, SIZES)
    net.set_params(Ws, bs)
    X = _inputs(rows, 22)
    y = net.forward(X)
    ref, _ = omlp.forward([W.astype(np.float32) for W in Ws], bs, X.astype(np.float64), mirror=True)
    assert y.shape == (rows, 19)
    assert _close(y, ref, REL)
    net.close()


@pytest.mark.parametrize("B,K", [(1, 1), (40, 3), (130, 4)])
def test_gradients_match_oracle(gf, ctx, B, K):
    Ws, bs = synth.mlp_weights(SIZES, 31)
    Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]
    net = gf.MLP(ctx, SIZES)
    net.set_params(Ws, bs)
    X = _inputs(B * K, 32)
    T, mask = _targets(B, 33)
    tp = gf.train_params(lr=1e-3, tile=TILE)
    loss = net.train_step(X, T, K, tp, tors_mask=mask, update=False)
    out, cache = omlp.forward(Ws, bs, X.astype(np.float64), mirror=True)
    # the winner is an argmin: check that the oracle's choice is not a near tie
    d, _ = omlp.pose_distance(out, np.repeat(T, K, 0), np.repeat(mask, K, 0), TILE)
    d = np.sort(d.reshape(B, K), 1)
    if K > 1:
        assert np.min(d[:, 1] - d[:, 0]) > 1e-3
    L, dout, _ = omlp.wta_loss(out, T.astype(np.float64), mask.astype(np.float64), K, TILE)
    dWs, dbs = omlp.backward(Ws, cache, dout, mirror=True)
    assert loss == pytest.approx(L, rel=1e-3)
    _, g = net.get_params()
    gW, gb = net.unflatten(g)
    for l in range(len(Ws)):
        assert _close(gW[l], dWs[l], REL), l
        assert _close(gb[l], dbs[l], REL), l
    net.close()


def test_adam_step_matches_oracle(gf, ctx):
    Ws, bs = synth.mlp_weights(SIZES, 41)
    Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]
    net = gf.MLP(ctx, SIZES)
    net.set_params(Ws, bs)
    B, K = 64, 2
    X = _inputs(B * K, 42)
    T, mask = _targets(B, 43)
    lr = 1e-3
    net.train_step(X, T, K, gf.train_params(lr=lr, tile=TILE), tors_mask=mask)
    p, _ = net.get_params()
    out, cache = omlp.forward(Ws, bs, X.astype(np.float64), mirror=True)
    _, dout, _ = omlp.wta_loss(out, T.astype(np.float64), mask.astype(np.float64), K, TILE)
    dWs, dbs = omlp.backward(Ws, cache, dout, mirror=True)
    params = [a.copy() for pair in zip(Ws, bs) for a in pair]
    grads = [a for pair in zip(dWs, dbs) for a in pair]
    omlp.adam(params, grads, {}, lr=lr, t=1)
    ref = np.concatenate([a.ravel() for a in params])
    g = np.concatenate([a.ravel() for a in grads])
    p0 = np.concatenate([a.ravel() for pair in zip(Ws, bs) for a in pair])
    # first Adam step moves each parameter by lr * g / (|g| + eps): compare
    # where the gradient is clearly resolved (sign and size agree on both sides)
    scale = np.concatenate([np.full(a.size, np.max(np.abs(a))) for a in grads])
    sure = np.abs(g) > 0.05 * scale
    assert sure.sum() > 1000
    assert np.max(np.abs(p[sure] - ref[sure])) < 1e-6
    assert np.max(np.abs(p - p0)) <= lr * (1 + 1e-5)
    net.close()


def test_training_reduces_the_loss(gf, ctx):
    """A few hundred Adam steps on a fixed set of poses lower the WTA loss."""
    Ws, bs = synth.mlp_weights(SIZES, 51)
    net = gf.MLP(ctx, SIZES)
    net.set_params(Ws, bs)
    B, K = 256, 4
    T, mask = _targets(B, 53)
    tp = gf.train_params(lr=1e-3, tile=TILE)
    first = None
    for it in range(300):
        X = _inputs(B * K, 1000 + it)
        loss = net.train_step(X, T, K, tp, tors_mask=mask)
        first = loss if first is None else first
    assert np.isfinite(loss) and loss < 0.5 * first
    net.close()


def test_propose_writes_oracle_poses(gf, ctx):
    mol = synth.c24h8o6_core()
    n_rep = 200
    reps = gf.Replicas(ctx, [mol], np.zeros(n_rep, np.int32), rigid=True)
    Ws, bs = synth.mlp_weights(SIZES, 61)
    Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]
    bs[-1][2] = 3.0                                  # push the COM above the surface
    net = gf.MLP(ctx, SIZES)
    net.set_params(Ws, bs)
    desc = gf.molecule_descriptor(mol)
    origin = (-1.0, 2.0)
    seed = 0x1234_5678_9ABC
    net.propose(reps, desc, seed, origin, TILE)
    x, v = reps.get_state()
    x = x.reshape(n_rep, 7)
    X = np.concatenate([np.tile(desc.astype(np.float64), (n_rep, 1)), omlp.counter_normal(seed, n_rep, 16)], 1)
    out, _ = omlp.forward(Ws, bs, X, mirror=True)
    scale = np.max(np.abs(out))
    d = x[:, :3] - out[:, :3]
    for a in range(2):
        d[:, a] -= TILE[a] * np.round(d[:, a] / TILE[a])
        assert np.all((x[:, a] >= origin[a] - 1e-4) & (x[:, a] < origin[a] + TILE[a] + 1e-4))
    assert np.max(np.abs(d)) <= REL * scale
    nu = np.linalg.norm(out[:, 3:7], axis=1, keepdims=True)
    assert np.allclose(np.linalg.norm(x[:, 3:7], axis=1), 1, atol=1e-5)
    # normalisation divides the output error by |u|
    assert np.all(np.abs(x[:, 3:7] - out[:, 3:7] / nu) <= 2 * REL * scale / nu)
    assert np.all(v == 0)
    net.close(); reps.close()


def test_descriptor_values(gf):
    mol = synth.c24h8o6_core()
    d = gf.molecule_descriptor(mol)
    assert d.shape == (64,)
    assert d[0] == pytest.approx(mol.n / 128)
    assert d[1:6].sum() == pytest.approx(1.0)
    assert np.all(d[20:] == 0)
    # inertia roots ascending, all positive for a planar but not linear core
    assert 0 < d[8] <= d[9] <= d[10]


def test_bad_arguments_are_rejected(gf, ctx):
    with pytest.raises(gf.GridffError):
        gf.MLP(ctx, (80, 256, 18))                  # output must be 19 wide
    net = gf.MLP(ctx, (200, 32, 19))
    mol = synth.c24h8o6_core()
    reps = gf.Replicas(ctx, [mol], np.zeros(4, np.int32), rigid=True)
    with pytest.raises(gf.GridffError):
        net.propose(reps, np.zeros(64, np.float32), 1, (0, 0), TILE)   # 136 noise inputs
    with pytest.raises(gf.GridffError):
        net.propose(reps, np.zeros(136, np.float32), 1, (0, 0), (0.0, TILE[1]))   # empty tile
    net.close(); reps.close()


def test_device_training_step_matches_oracle(gf, ctx):
    """gridff_mlp_train draws its batch on the device; the oracle rebuilds the
    same batch from the counters and takes the same Adam step."""
    Ws, bs = synth.mlp_weights(SIZES, 71)
    Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]
    net = gf.MLP(ctx, SIZES)
    net.set_params(Ws, bs)
    T_all, mask_all = _targets(500, 72)
    net.set_targets(T_all, mask_all)
    desc = (synth.rng(73).random(64) * 0.5).astype(np.float32)
    B, K, seed, lr = 48, 3, 0x5EED, 1e-3
    losses = net.train(1, B, K, desc, seed, gf.train_params(lr=lr, tile=TILE))
    p, _ = net.get_params()
    rows, X = omlp.train_batch(seed, 0, len(T_all), B, K, desc.astype(np.float64), 16)
    T = T_all[rows].astype(np.float64); M = mask_all[rows].astype(np.float64)
    out, cache = omlp.forward(Ws, bs, X, mirror=True)
    L, dout, _ = omlp.wta_loss(out, T, M, K, TILE)
    assert losses[0] == pytest.approx(L, rel=2e-3)
    dWs, dbs = omlp.backward(Ws, cache, dout, mirror=True)
    params = [a.copy() for pair in zip(Ws, bs) for a in pair]
    grads = [a for pair in zip(dWs, dbs) for a in pair]
    omlp.adam(params, grads, {}, lr=lr, t=1)
    ref = np.concatenate([a.ravel() for a in params])
    g = np.concatenate([a.ravel() for a in grads])
    scale = np.concatenate([np.full(a.size, np.max(np.abs(a))) for a in grads])
    sure = np.abs(g) > 0.05 * scale
    assert sure.sum() > 1000 and np.max(np.abs(p[sure] - ref[sure])) < 1e-6
    # further steps continue the counter stream and lower the loss
    more = net.train(300, 256, 4, desc, seed, gf.train_params(lr=1e-3, tile=TILE))
    assert np.all(np.isfinite(more)) and more[-20:].mean() < more[:20].mean()
    net.close()


def test_training_loop_split_over_calls_equals_one_call(gf, ctx):
    """The training loop replays one captured step whose counters (random
    stream step, loss slot, Adam t) advance on the device: 2 x 25 steps in
    two calls give the same parameters and losses, bit for bit, as 50 steps
    in one call."""
    Ws, bs = synth.mlp_weights(SIZES, 81)
    T_all, mask_all = _targets(300, 82)
    desc = (synth.rng(83).random(64) * 0.5).astype(np.float32)
    out = []
    for split in ((50,), (25, 25)):
        net = gf.MLP(ctx, SIZES)
        net.set_params(Ws, bs)
        net.set_targets(T_all, mask_all)
        ls = np.concatenate([net.train(n, 64, 4, desc, 9, gf.train_params(lr=1e-3, tile=TILE)) for n in split])
        out.append((net.get_params()[0], ls))
        net.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
