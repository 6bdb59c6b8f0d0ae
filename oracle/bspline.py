"""Cubic B-spline basis, coefficient fit and tricubic evaluation (Sec. 5).

Oracle (test infrastructure).  Conventions shared with the library by
*definition*, not by code:

* grid nodes along an axis: x_k = x0 + k*dx, k = 0..n-1;
* x and y are periodic with period n*dx; z is clamped: a coefficient index
  below 0 or above n-1 reads the end coefficient (reading: the paper does
  not state the z boundary);
* 1D interpolant (Eq. Bspline1D): f(x) = sum_{j=-1..2} B((x - x_{i+j})/dx)
  b_{i+j} with i = floor((x - x0)/dx);
* 3D interpolant: tensor product, evaluated as 16 1D passes along z, 4
  along y, 1 along x (Sec. 5); the gradient is the exact derivative of the
  interpolant (Sec. 5, forces as the analytic gradient);
* z outside the grid: below the first node the point is clamped to the first
  node and flagged; at or above the last node the field is taken as 0
  (reading: the substrate potentials have decayed to ~1e-13 there).
"""
from __future__ import annotations

import numpy as np


def B(t):
    """Cubic B-spline basis of Eq. Bspline (any float dtype, elementwise)."""
    t = np.asarray(t)
    one = t.dtype.type(1) if t.dtype.kind == "f" else 1.0
    a = np.abs(t)
    inner = one * 2 / 3 - t * t + a * a * a / 2
    outer = (2 - a) ** 3 / 6
    return np.where(a < 1, inner, np.where(a < 2, outer, 0 * t))


def dB(t):
    """Derivative dB/dt of Eq. Bspline, piece by piece."""
    t = np.asarray(t)
    a = np.abs(t)
    s = np.sign(t)
    inner = -2 * t + 3 * t * a / 2          # d/dt (2/3 - t^2 + |t|^3/2)
    outer = -s * (2 - a) ** 2 / 2           # d/dt ((2-|t|)^3/6)
    return np.where(a < 1, inner, np.where(a < 2, outer, 0 * t))


OFFSETS = np.array([-1, 0, 1, 2])


def weights(t):
    """Basis weights B(t - j) and derivatives B'(t - j), j = -1..2, for the
    fractional position t in [0, 1) (Eq. Bspline1D).  Shape (..., 4)."""
    t = np.asarray(t)
    s = t[..., None] - OFFSETS.astype(t.dtype)
    return B(s), dB(s)


def collocation_matrix(n: int, periodic: bool) -> np.ndarray:
    """Matrix M with (M b)_k = interpolant at node k (Eq. Bspline1D at t=0).

    Row k holds B(-j) at column idx(k + j), j = -1..2, where idx wraps
    (periodic) or clamps to [0, n-1].
    """
    M = np.zeros((n, n))
    for k in range(n):
        for j in OFFSETS:
            m = k + j
            m = m % n if periodic else min(max(m, 0), n - 1)
            M[k, m] += float(B(np.float64(-j)))
    return M


def _apply_along(M, arr, axis):
    return np.moveaxis(np.tensordot(M, np.moveaxis(arr, axis, 0), axes=(1, 0)), 0, axis)


def _solve_along(M, arr, axis):
    moved = np.moveaxis(arr, axis, 0)
    sol = np.linalg.solve(M, moved.reshape(moved.shape[0], -1)).reshape(moved.shape)
    return np.moveaxis(sol, 0, axis)


PERIODIC = (True, True, False)


def fit_exact(values: np.ndarray) -> np.ndarray:
    """Coefficients b with (Mx (x) My (x) Mz) b = values, for values of shape
    (nx, ny, nz) or (C, nx, ny, nz).

    The paper fits b so that the interpolant reproduces the node values
    (Sec. 5); the Kronecker-structured linear system has a unique solution,
    obtained here by one dense 1D solve per axis.
    """
    v = np.asarray(values, np.float64)
    lead = v.ndim - 3
    b = v
    for ax in range(3):
        M = collocation_matrix(v.shape[lead + ax], PERIODIC[ax])
        b = _solve_along(M, b, lead + ax)
    return b


def apply_collocation(b: np.ndarray) -> np.ndarray:
    """Node values of the interpolant with coefficients b."""
    lead = b.ndim - 3
    out = b
    for ax in range(3):
        M = collocation_matrix(b.shape[lead + ax], PERIODIC[ax])
        out = _apply_along(M, out, lead + ax)
    return out


def fit_gradient_descent(values: np.ndarray, iterations: int, step: float = 1.0,
                         b0: np.ndarray | None = None):
    """The paper's fit (Sec. 5): gradient descent on the squared node error.

    Minimises 0.5*||A b - v||^2 with A the tensor-product collocation
    operator; the gradient is A^T (A b - v).  Starts from b0 (default: the
    node values).  Returns (b, rms history).  The paper gives neither the
    start nor the step; the reading is b0 = v and a fixed step.
    """
    v = np.asarray(values, np.float64)
    b = v.copy() if b0 is None else np.asarray(b0, np.float64).copy()
    lead = v.ndim - 3
    mats = [collocation_matrix(v.shape[lead + ax], PERIODIC[ax]) for ax in range(3)]
    hist = []
    for _ in range(iterations):
        r = b
        for ax in range(3):
            r = _apply_along(mats[ax], r, lead + ax)
        r = r - v
        hist.append(float(np.sqrt(np.mean(r * r))))
        g = r
        for ax in range(3):
            g = _apply_along(mats[ax].T, g, lead + ax)
        b = b - step * g
    return b, np.array(hist)


def eval_grid(coefs: np.ndarray, origin, spacing, points: np.ndarray,
              dtype=np.float64, below_u: float = 0.0):
    """Tricubic B-spline value and gradient of every channel at the points.

    coefs: (C, nx, ny, nz); origin, spacing: 3-vectors; points: (N, 3).
    All arithmetic is done in ``dtype`` (float64, or float32 for the
    single-precision mirror, which also rounds the coefficients first).
    ``below_u``: the floor of the grid in units of the z spacing above the
    first node (the number of ghost node planes below the floor, see
    grid.py); a point is flagged below when its z coordinate in those units
    is smaller.  Below the first node the point is still clamped to it.
    Returns (f (N, C), grad (N, C, 3), below (N,) bool).
    """
    dt = np.dtype(dtype).type
    c = np.asarray(coefs).astype(dtype)
    C, nx, ny, nz = c.shape
    P = np.asarray(points).astype(dtype)
    o = np.asarray(origin, np.float64).astype(dtype)
    h = np.asarray(spacing, np.float64).astype(dtype)

    def axis_setup(u, n, periodic):
        i = np.floor(u)
        t = (u - i).astype(dtype)
        i = i.astype(np.int64)
        idx = i[:, None] + OFFSETS[None, :]
        idx = np.mod(idx, n) if periodic else np.clip(idx, 0, n - 1)
        w, dw = weights(t)
        return idx, w.astype(dtype), dw.astype(dtype)

    ux = (P[:, 0] - o[0]) / h[0]
    uy = (P[:, 1] - o[1]) / h[1]
    uz = (P[:, 2] - o[2]) / h[2]
    below = uz < dt(below_u)
    uz = np.where(uz < 0, dt(0), uz)
    above = uz >= nz - 1
    uz = np.where(above, dt(0), uz)
    ix, wx, dwx = axis_setup(ux, nx, True)
    iy, wy, dwy = axis_setup(uy, ny, True)
    iz, wz, dwz = axis_setup(uz, nz, False)

    # gather the 4x4x4 stencil of every channel: (C, N, 4, 4, 4)
    g = c[:, ix[:, :, None, None], iy[:, None, :, None], iz[:, None, None, :]]
    # 16 passes along z: value and z-derivative of each (x, y) column
    fz = np.zeros(g.shape[:4], dtype)
    fz_d = np.zeros(g.shape[:4], dtype)
    for k in range(4):
        fz = fz + wz[None, :, None, None, k] * g[..., k]
        fz_d = fz_d + dwz[None, :, None, None, k] * g[..., k]
    # 4 passes along y
    fy = np.zeros(g.shape[:3], dtype)
    fy_dy = np.zeros(g.shape[:3], dtype)
    fy_dz = np.zeros(g.shape[:3], dtype)
    for k in range(4):
        fy = fy + wy[None, :, None, k] * fz[..., k]
        fy_dy = fy_dy + dwy[None, :, None, k] * fz[..., k]
        fy_dz = fy_dz + wy[None, :, None, k] * fz_d[..., k]
    # 1 pass along x
    f = np.zeros(g.shape[:2], dtype)
    gx = np.zeros(g.shape[:2], dtype)
    gy = np.zeros(g.shape[:2], dtype)
    gz = np.zeros(g.shape[:2], dtype)
    for k in range(4):
        f = f + wx[None, :, k] * fy[..., k]
        gx = gx + dwx[None, :, k] * fy[..., k]
        gy = gy + wx[None, :, k] * fy_dy[..., k]
        gz = gz + wx[None, :, k] * fy_dz[..., k]
    grad = np.stack([gx / h[0], gy / h[1], gz / h[2]], -1)      # (C, N, 3)
    zero = above[None, :]
    f = np.where(zero, dt(0), f)
    grad = np.where(zero[..., None], dt(0), grad)
    return f.T.copy(), np.transpose(grad, (1, 0, 2)).copy(), below
