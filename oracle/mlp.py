"""Pose-proposal MLP: forward, winner-takes-all pose loss, backward, Adam.

Oracle (test infrastructure).  The network is not in the paper; it is the
learned proposal of poses for GridFF relaxations (molecule descriptor and
noise in; centre of mass, orientation quaternion and torsions out).  This
module restates it in float64 with plain numpy matrix products, optionally
mirroring the GPU's bfloat16 rounding of GEMM operands (weights, layer
inputs, back-propagated gradients) so that parity can be checked.

Definitions
-----------
layer l: a_l = h_{l-1} W_l^T + b_l;  h_l = max(a_l, 0) (hidden), h_L = a_L
output o = [c (3), u (4), theta (12)];  q = u / |u|
pose distance to a target (c*, q*, theta*, torsion mask m):
    d = |c - c*|^2_min-image(xy) + w_q (1 - (q . q*)^2)
        + w_t sum_j m_j (1 - cos(theta_j - theta*_j))
(x, y of the centre use the minimum image on the periodic tile Lx, Ly.)
winner-takes-all loss over K proposals of one target: min_k d_k; the batch
loss is the mean over targets; only the winning proposal gets a gradient.
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
      w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

N_POS, N_QUAT, N_TORS = 3, 4, 12
N_OUT = N_POS + N_QUAT + N_TORS


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, np.float64).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(Ws, bs, X, mirror=True):
    """Returns (output, cache).  mirror: round GEMM operands to bfloat16."""
    r = bf16 if mirror else (lambda a: np.asarray(a, np.float64))
    h = np.asarray(X, np.float64)
    cache = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        hin = r(h)
        a = hin @ r(W).T + b
        cache.append((hin, a))
        h = np.maximum(a, 0.0) if l < len(Ws) - 1 else a
    return h, cache


def pose_distance(o, t, mask, tile, w_q=1.0, w_t=0.25):
    """Distance of outputs o (N, 19) to targets t (N, 19) and its gradient."""
    o = np.asarray(o, np.float64)
    t = np.asarray(t, np.float64)
    dc = o[:, :3] - t[:, :3]
    for a in range(2):
        dc[:, a] -= tile[a] * np.round(dc[:, a] / tile[a])
    u = o[:, 3:7]
    nu = np.linalg.norm(u, axis=1, keepdims=True)
    q = u / nu
    s = np.sum(q * t[:, 3:7], 1, keepdims=True)
    dth = o[:, 7:] - t[:, 7:]
    d = np.sum(dc * dc, 1) + w_q * (1 - s[:, 0] ** 2) + w_t * np.sum(mask * (1 - np.cos(dth)), 1)
    g = np.zeros_like(o)
    g[:, :3] = 2 * dc
    g[:, 3:7] = -2 * w_q * s * (t[:, 3:7] - s * q) / nu
    g[:, 7:] = w_t * mask * np.sin(dth)
    return d, g


def wta_loss(out, targets, mask, K, tile, w_q=1.0, w_t=0.25):
    """Winner-takes-all loss: out (B*K, 19) holds K proposals per target
    (proposal k of target b at row b*K + k).  Returns (loss, dL/dout, winners)."""
    B = len(targets)
    d, g = pose_distance(out, np.repeat(targets, K, 0), np.repeat(mask, K, 0), tile, w_q, w_t)
    d = d.reshape(B, K)
    win = np.argmin(d, 1)
    grad = np.zeros_like(out)
    rows = np.arange(B) * K + win
    grad[rows] = g[rows] / B
    return float(np.mean(d[np.arange(B), win])), grad, win


def backward(Ws, cache, dout, mirror=True):
    """Gradients (dW, db) of every layer for dL/doutput = dout."""
    r = bf16 if mirror else (lambda a: np.asarray(a, np.float64))
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    g = np.asarray(dout, np.float64)
    for l in range(len(Ws) - 1, -1, -1):
        hin, a = cache[l]
        if l < len(Ws) - 1:
            g = g * (a > 0)
        gr = r(g)
        dWs[l] = gr.T @ hin
        dbs[l] = g.sum(0)
        g = gr @ r(Ws[l])
    return dWs, dbs


def adam(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t starts at 1); updates params and state in place."""
    for k, (p, g) in enumerate(zip(params, grads)):
        m, v = state.setdefault(k, (np.zeros_like(p), np.zeros_like(p)))
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        state[k] = (m, v)
        p -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)


_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """Output of the SplitMix64 generator (Steele, Lea and Flood, 2014) whose
    state is x: advance by the golden gamma, then the variant-13 mix."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def counter_normal(seed: int, rows: int, dim: int) -> np.ndarray:
    """Standard normal draws of the proposal noise: entry (r, j) from the
    counter 64 r + j hashed with the seed, then Box-Muller (float64 here;
    the device evaluates the same formula in float32)."""
    out = np.empty((rows, dim))
    for r in range(rows):
        for j in range(dim):
            s = splitmix64(seed ^ splitmix64(64 * r + j))
            u1 = ((s >> 40) + 1) / 2.0 ** 24
            u2 = ((s >> 16) & 0xFFFFFF) / 2.0 ** 24
            out[r, j] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def train_batch(seed: int, step: int, n_all: int, B: int, K: int, desc, n_noise: int):
    """The library's device-side training batch of step `step`: target rows
    splitmix64(seed ^ splitmix64(2^20 step + b)) mod n_all, and inputs
    [descriptor, noise] with noise j of row m from the counter
    64 (2^20 step + m) + j (Box-Muller in float64 here)."""
    rows = [splitmix64(seed ^ splitmix64((step << 20) + b)) % n_all for b in range(B)]
    X = np.zeros((B * K, len(desc) + n_noise))
    X[:, :len(desc)] = np.asarray(desc, np.float64)
    for m in range(B * K):
        for j in range(n_noise):
            s = splitmix64(seed ^ splitmix64((((step << 20) + m) << 6) + j))
            u1 = ((s >> 40) + 1) / 2.0 ** 24
            u2 = ((s >> 16) & 0xFFFFFF) / 2.0 ** 24
            X[m, len(desc) + j] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return np.array(rows), X
