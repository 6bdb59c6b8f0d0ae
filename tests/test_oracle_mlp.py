"""Pins of the oracle's pose-proposal MLP (forward, WTA loss, backward, Adam)."""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2508_15522_gb300 import synth


def _net(seed=1, sizes=(80, 32, 32, 19)):
    return synth.mlp_weights(sizes, seed)


def test_bf16_rounding_known_values():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(1 + 2 ** -8) == 1.0
    assert mlp.bf16(1 + 3 * 2 ** -9) == 1 + 2 ** -7
    assert mlp.bf16(-2.0) == -2.0
    x = np.random.default_rng(0).standard_normal(1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2 ** -8)


def test_relu_network_special_case():
    """One hidden unit: out = w2 * max(w1 . x + b1, 0) + b2."""
    W1 = np.array([[1.0, -2.0]]); b1 = np.array([0.5])
    W2 = np.array([[3.0]]); b2 = np.array([-1.0])
    X = np.array([[1.0, 1.0], [2.0, 0.0]])
    out, _ = mlp.forward([W1, W2], [b1, b2], X, mirror=False)
    assert out[:, 0].tolist() == [-1.0, 3.0 * 2.5 - 1.0]


def test_pose_distance_invariances():
    g = synth.rng(3)
    t = np.zeros((1, 19)); t[0, 3] = 1.0
    o = t.copy()
    o[0, 3:7] = [-2.0, 0, 0, 0]                     # -q (scaled): same orientation
    o[0, 0] = 11.28                                  # one tile over in x
    d, _ = mlp.pose_distance(o, t, np.zeros((1, 12)), (11.28, 11.28))
    assert d[0] == pytest.approx(0.0, abs=1e-12)
    o[0, 3:7] = [0, 1, 0, 0]                         # 180 deg rotation: 1 - (q.q*)^2 = 1
    d, _ = mlp.pose_distance(o, t, np.zeros((1, 12)), (11.28, 11.28))
    assert d[0] == pytest.approx(1.0)


def test_backward_matches_finite_differences():
    Ws, bs = _net(5, (16, 8, 8, 19))
    g = synth.rng(6)
    X = g.standard_normal((12, 16))
    T = g.standard_normal((4, 19)); T[:, 3:7] /= np.linalg.norm(T[:, 3:7], axis=1, keepdims=True)
    mask = (g.random((4, 12)) < 0.5).astype(float)
    tile = (11.28, 9.99)

    def loss_of():
        out, _ = mlp.forward(Ws, bs, X, mirror=False)
        return mlp.wta_loss(out, T, mask, 3, tile)[0]

    out, cache = mlp.forward(Ws, bs, X, mirror=False)
    L, dout, win = mlp.wta_loss(out, T, mask, 3, tile)
    dWs, dbs = mlp.backward(Ws, cache, dout, mirror=False)
    h = 1e-6
    for l in range(len(Ws)):
        for (i, j) in [(0, 0), (1, 2), (Ws[l].shape[0] - 1, Ws[l].shape[1] - 1)]:
            Ws[l][i, j] += h; lp = loss_of()
            Ws[l][i, j] -= 2 * h; lm = loss_of()
            Ws[l][i, j] += h
            assert (lp - lm) / (2 * h) == pytest.approx(dWs[l][i, j], abs=1e-6, rel=1e-4)
        bs[l][0] += h; lp = loss_of(); bs[l][0] -= 2 * h; lm = loss_of(); bs[l][0] += h
        assert (lp - lm) / (2 * h) == pytest.approx(dbs[l][0], abs=1e-6, rel=1e-4)


def test_adam_first_step_is_signed_learning_rate():
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-3])]
    mlp.adam(p, g, {}, lr=0.01, t=1)
    assert np.allclose(p[0], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], atol=1e-6)


def test_adam_constant_gradient_moves_by_the_learning_rate_every_step():
    # with a constant gradient the bias-corrected moments are exactly g and
    # g^2 at every step t, so each step moves lr * g / (|g| + eps)
    p = [np.array([1.0, -2.0, 0.5, 3.0])]
    g = np.array([0.3, -4.0, 1e-3, -1e-6])
    state = {}
    for t in range(1, 8):
        mlp.adam(p, [g], state, lr=0.01, t=t)
    want = np.array([1.0, -2.0, 0.5, 3.0]) - 7 * 0.01 * g / (np.abs(g) + 1e-8)
    assert np.abs(p[0] - want).max() < 1e-12


def test_wta_gradient_only_on_the_winner():
    T = np.zeros((2, 19)); T[:, 3] = 1.0
    out = np.zeros((6, 19)); out[:, 3] = 1.0
    out[[0, 1, 2], 0] = [3.0, 0.1, 2.0]          # target 0: proposal 1 wins
    out[[3, 4, 5], 1] = [0.2, 5.0, 6.0]          # target 1: proposal 0 wins
    L, g, win = mlp.wta_loss(out, T, np.zeros((2, 12)), 3, (100.0, 100.0))
    assert win.tolist() == [1, 0]
    assert np.count_nonzero(np.abs(g).sum(1)) == 2
    assert L == pytest.approx((0.01 + 0.04) / 2)


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0 (state advances by the golden gamma each call)
    # starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F.
    gamma = 0x9E3779B97F4A7C15
    outs = [mlp.splitmix64((k * gamma) & ((1 << 64) - 1)) for k in range(3)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_normal_moments():
    z = mlp.counter_normal(12345, 200, 16).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * np.sqrt(2 / z.size)
    assert abs(np.mean(z ** 4) - 3) < 0.3
