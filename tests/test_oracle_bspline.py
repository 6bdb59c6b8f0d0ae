"""Pins of the oracle's B-spline basis, fit and tricubic evaluation (Sec. 5)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import bspline
from paper_2508_15522_gb300 import synth


def test_basis_golden_knots():
    for t, val in read_golden("bspline_knots.txt"):
        assert bspline.B(np.float64(t)) == pytest.approx(val, abs=1e-15)


def test_partition_of_unity_and_derivative_sum():
    t = np.linspace(0, 1, 1001, endpoint=False)
    w, dw = bspline.weights(t)
    assert np.abs(w.sum(1) - 1).max() < 1e-14
    assert np.abs(dw.sum(1)).max() < 1e-14
    assert (w >= 0).all()


def test_derivative_matches_finite_difference_and_is_c2():
    t = np.linspace(-2.3, 2.3, 941)
    h = 1e-6
    fd = (bspline.B(t + h) - bspline.B(t - h)) / (2 * h)
    assert np.abs(fd - bspline.dB(t)).max() < 1e-8
    # second derivative continuous at the knots 0, +-1, +-2 (C2 spline)
    for k in (-2.0, -1.0, 0.0, 1.0, 2.0):
        e = 1e-5
        d2l = (bspline.dB(np.float64(k - e)) - bspline.dB(np.float64(k - 2 * e))) / e
        d2r = (bspline.dB(np.float64(k + 2 * e)) - bspline.dB(np.float64(k + e))) / e
        assert abs(d2l - d2r) < 1e-3


def test_collocation_rows():
    M = bspline.collocation_matrix(6, periodic=True)
    assert M[0, 0] == pytest.approx(2 / 3) and M[0, 1] == pytest.approx(1 / 6)
    assert M[0, 5] == pytest.approx(1 / 6)
    Mc = bspline.collocation_matrix(6, periodic=False)
    assert Mc[0, 0] == pytest.approx(5 / 6) and Mc[5, 5] == pytest.approx(5 / 6)
    assert np.allclose(Mc.sum(1), 1) and np.allclose(M.sum(1), 1)


def _nodes(shape, h, origin=(0.0, 0.0, 0.0)):
    ax = [origin[a] + np.arange(shape[a]) * h[a] for a in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


def test_fit_reproduces_node_values_through_evaluation():
    g = synth.rng(11)
    shape = (7, 6, 9)
    v = g.standard_normal((2,) + shape)
    b = bspline.fit_exact(v)
    h = (0.3, 0.25, 0.2)
    pts = _nodes(shape, h, (1.0, -2.0, 0.5))
    pts = pts[pts[:, 2] < 0.5 + (shape[2] - 1) * h[2] - 1e-9]   # last z node is 'above'
    f, _, below = bspline.eval_grid(b, (1.0, -2.0, 0.5), h, pts)
    idx = np.round((pts - np.array([1.0, -2.0, 0.5])) / np.array(h)).astype(int)
    ref = v[:, idx[:, 0], idx[:, 1], idx[:, 2]].T
    assert not below.any()
    assert np.abs(f - ref).max() < 1e-12


def test_constant_field_is_reproduced_everywhere():
    v = np.full((1, 5, 6, 7), 3.25)
    b = bspline.fit_exact(v)
    assert np.allclose(b, 3.25, atol=1e-13)
    pts = synth.rng(3).uniform(-5, 5, (200, 3))
    pts[:, 2] = synth.rng(4).uniform(0, 0.9 * 6 * 0.3, 200)
    f, gr, _ = bspline.eval_grid(b, (0, 0, 0), (0.3, 0.3, 0.3), pts)
    assert np.abs(f - 3.25).max() < 1e-12
    assert np.abs(gr).max() < 1e-10


def _cos_field_error(n):
    # periodic in x, y with period 2; z-dependence smooth, evaluated in the
    # middle of the z range so the clamped boundary does not matter
    L = 2.0
    h = L / n
    nz = int(round(3.0 / h)) + 1
    shape = (n, n, nz)
    pts = _nodes(shape, (h, h, h))
    fun = lambda p: np.cos(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1]) * np.cos(0.7 * p[:, 2])
    b = bspline.fit_exact(fun(pts).reshape((1,) + shape))
    q = synth.rng(5).uniform(0, 1, (400, 3)) * np.array([L, L, 1.0]) + np.array([0, 0, 1.0])
    f, _, _ = bspline.eval_grid(b, (0, 0, 0), (h, h, h), q)
    return np.abs(f[:, 0] - fun(q)).max()


def test_fourth_order_convergence():
    e1 = _cos_field_error(16)
    e2 = _cos_field_error(32)
    assert 12.0 < e1 / e2 < 20.0          # O(h^4): ratio ~16


def test_interpolation_error_within_classical_bound_for_exponential():
    # f(z) = exp(-k z): error <= (5/384) h^4 max|f''''| for cubic spline
    # interpolation (Hall & Meyer 1976), here along z only
    k, h = 3.0, 0.1
    nz = 80
    z = np.arange(nz) * h
    v = np.broadcast_to(np.exp(-k * z), (1, 4, 4, nz)).copy()
    b = bspline.fit_exact(v)
    zq = np.linspace(2.0, 5.0, 301)
    pts = np.stack([np.zeros_like(zq), np.zeros_like(zq), zq], 1)
    f, _, _ = bspline.eval_grid(b, (0, 0, 0), (1.0, 1.0, h), pts)
    err = np.abs(f[:, 0] - np.exp(-k * zq))
    bound = 5 / 384 * h ** 4 * k ** 4 * np.exp(-k * (zq - 2 * h))
    assert (err <= bound).all()


def test_clamped_z_end_closed_form_and_order():
    """Reading of the z ends: coefficients beyond the first and last node
    repeat the end coefficient.  Closed form at the floor node (t = 0, B
    weights 1/6, 4/6, 1/6 and slope weights -1/2, 0, 1/2 per h): value
    (5 b_0 + b_1) / 6 and z-slope (b_1 - b_0) / (2 h).  Consequence for a
    smooth field: fourth order in the interior, but in the first cell above
    the floor the value is first order and the slope error does not shrink
    with h (about 40 % of the slope of exp(-3 z) at the floor)."""
    g = np.random.default_rng(2)
    h = 0.1
    b = g.standard_normal((1, 4, 4, 12))
    f, grad, below = bspline.eval_grid(b, (0, 0, 0), (1.0, 1.0, h), np.array([[1.0, 2.0, 0.0]]))
    # at x, y nodes the x and y weights are (1/6, 4/6, 1/6) too
    col = lambda k: (b[0, 0:3, 1:4, k] * np.outer([1, 4, 1], [1, 4, 1]) / 36).sum()
    assert not below[0]
    assert f[0, 0] == pytest.approx((5 * col(0) + col(1)) / 6, abs=1e-13)
    assert grad[0, 0, 2] == pytest.approx((col(1) - col(0)) / (2 * h), abs=1e-12)

    def errors(h):
        nz = int(round(4.0 / h)) + 1
        v = np.broadcast_to(np.exp(-3.0 * np.arange(nz) * h), (1, 4, 4, nz)).copy()
        c = bspline.fit_exact(v)
        out = []
        for lo, hi in ((0.0, h), (1.5, 2.5)):
            zq = np.linspace(lo, hi, 201)
            pts = np.stack([np.full_like(zq, 0.3), np.full_like(zq, 0.7), zq], 1)
            fv, gv, _ = bspline.eval_grid(c, (0, 0, 0), (1.0, 1.0, h), pts)
            out.append((np.abs(fv[:, 0] - np.exp(-3 * zq)).max(), np.abs(gv[:, 0, 2] + 3 * np.exp(-3 * zq)).max()))
        return out

    (fe1, fs1), (ie1, _) = errors(0.1)
    (fe2, fs2), (ie2, _) = errors(0.05)
    assert 1.7 < fe1 / fe2 < 2.5               # first cell: O(h) in the value
    assert min(fs1, fs2) > 0.3 * 3.0           # ... and no convergence of the slope
    assert 12.0 < ie1 / ie2 < 20.0             # interior: O(h^4)


def test_ghost_nodes_make_the_floor_cell_interior_accurate():
    """Ghost nodes (reading of the z boundary): node values of exp(-3 z)
    also taken on G planes below the floor z = 0 and fitted with the rest.
    With G = 8 the floor cell [0, h] meets the interior bounds of cubic
    spline interpolation (Hall and Meyer 1976): |f - s| <= (5/384) h^4 M4
    and |f' - s'| <= (1/24) h^3 M4, M4 = max |4th derivative| = 81 on the
    cell; without them (G = 0) the value and the slope miss those bounds by
    two orders of magnitude and more."""
    def floor_cell_errors(h, G):
        nz = int(round(4.0 / h)) + 1 + G
        z = (np.arange(nz) - G) * h
        v = np.broadcast_to(np.exp(-3.0 * z), (1, 4, 4, nz)).copy()
        c = bspline.fit_exact(v)
        zq = np.linspace(0.0, h, 201)
        pts = np.stack([np.full_like(zq, 0.3), np.full_like(zq, 0.7), zq + G * h], 1)
        f, gr, below = bspline.eval_grid(c, (0, 0, 0), (1.0, 1.0, h), pts, below_u=G)
        assert not below.any()
        return np.abs(f[:, 0] - np.exp(-3 * zq)).max(), np.abs(gr[:, 0, 2] + 3 * np.exp(-3 * zq)).max()

    for h in (0.1, 0.05):
        hm_value, hm_slope = 5.0 / 384.0 * h ** 4 * 81.0, h ** 3 / 24.0 * 81.0
        ev, es = floor_cell_errors(h, 8)
        assert ev <= hm_value and es <= hm_slope, (h, ev, es)
        ev0, es0 = floor_cell_errors(h, 0)
        assert ev0 > 50 * hm_value and es0 > 200 * hm_slope


def test_ghost_floor_flags_points_but_evaluates_them():
    """With G ghost planes the floor is G spacings above the first node:
    a point between the first node and the floor is flagged below but
    evaluated on its own cell (not clamped); below the first node it is
    clamped to the first node plane."""
    g = np.random.default_rng(5)
    h, G = 0.2, 3
    b = g.standard_normal((1, 5, 5, 12))
    pts = np.array([[0.5, 0.5, 0.5 * h], [0.5, 0.5, (G + 0.01) * h], [0.5, 0.5, (G - 0.01) * h],
                    [0.5, 0.5, -0.7], [0.5, 0.5, 0.0]])
    f, _, below = bspline.eval_grid(b, (0, 0, 0), (1.0, 1.0, h), pts, below_u=G)
    assert below.tolist() == [True, False, True, True, True]
    f0, _, _ = bspline.eval_grid(b, (0, 0, 0), (1.0, 1.0, h), pts[:1])
    assert f[0, 0] == f0[0, 0]                       # evaluated where it is
    assert f[3, 0] == f[4, 0]                         # clamped to the first node plane


def test_gradient_matches_finite_difference():
    g = synth.rng(21)
    b = g.standard_normal((3, 6, 5, 9))
    h = (0.2, 0.3, 0.25)
    pts = g.uniform(0, 1, (50, 3)) * np.array([1.2, 1.5, 1.0]) + np.array([0, 0, 0.4])
    f, gr, _ = bspline.eval_grid(b, (0, 0, 0), h, pts)
    eps = 1e-6
    for a in range(3):
        d = np.zeros(3); d[a] = eps
        fp, _, _ = bspline.eval_grid(b, (0, 0, 0), h, pts + d)
        fm, _, _ = bspline.eval_grid(b, (0, 0, 0), h, pts - d)
        assert np.abs((fp - fm) / (2 * eps) - gr[:, :, a]).max() < 1e-6


def test_periodicity_in_x_and_y():
    g = synth.rng(22)
    b = g.standard_normal((1, 5, 7, 6))
    h = (0.4, 0.3, 0.2)
    pts = g.uniform(0, 1, (40, 3)) * np.array([2.0, 2.1, 0.8])
    f0, g0, _ = bspline.eval_grid(b, (0, 0, 0), h, pts)
    for shift in ((5 * 0.4, 0, 0), (0, 7 * 0.3, 0), (-3 * 5 * 0.4, 2 * 7 * 0.3, 0)):
        f1, g1, _ = bspline.eval_grid(b, (0, 0, 0), h, pts + np.array(shift))
        assert np.abs(f1 - f0).max() < 1e-12 and np.abs(g1 - g0).max() < 1e-11


def test_z_outside_grid():
    g = synth.rng(23)
    b = g.standard_normal((1, 4, 4, 6))
    h = (0.5, 0.5, 0.5)
    top = 5 * 0.5
    pts = np.array([[0.3, 0.3, top], [0.3, 0.3, top + 1.0], [0.3, 0.3, -0.2], [0.3, 0.3, 0.0]])
    f, gr, below = bspline.eval_grid(b, (0, 0, 0), h, pts)
    assert f[0, 0] == 0 and f[1, 0] == 0 and np.all(gr[:2] == 0)
    assert below.tolist() == [False, False, True, False]
    assert f[2, 0] == f[3, 0]


def test_float32_mirror_agrees_with_float64():
    g = synth.rng(24)
    b = g.standard_normal((3, 8, 8, 10))
    pts = g.uniform(0, 1, (300, 3)) * np.array([1.6, 1.6, 1.5]) + np.array([0, 0, 0.1])
    f64, g64, _ = bspline.eval_grid(b.astype(np.float32).astype(np.float64), (0, 0, 0), (0.2, 0.2, 0.2), pts)
    f32, g32, _ = bspline.eval_grid(b, (0, 0, 0), (0.2, 0.2, 0.2), pts, dtype=np.float32)
    assert f32.dtype == np.float32
    assert np.abs(f32 - f64).max() < 2e-6 and np.abs(g32 - g64).max() < 5e-5


def test_gradient_descent_fit_converges_to_exact_solution():
    # gradient descent on 0.5||A b - v||^2 contracts the error by at most
    # max |1 - step * lam^2| per iteration, lam over the eigenvalues of A
    # (products of the 1D collocation eigenvalues)
    g = synth.rng(25)
    v = g.standard_normal((5, 4, 6))
    b_exact = bspline.fit_exact(v)
    step, iters = 1.9, 3000
    b, hist = bspline.fit_gradient_descent(v, iters, step=step)
    lam = [np.linalg.eigvalsh(bspline.collocation_matrix(n, p))
           for n, p in zip(v.shape, bspline.PERIODIC)]
    lam3 = np.einsum("i,j,k->ijk", *lam).ravel()
    rho = np.max(np.abs(1 - step * lam3 ** 2))
    e0 = np.linalg.norm(v - b_exact)
    assert np.all(np.diff(hist) <= 1e-15)          # monotone
    assert np.linalg.norm(b - b_exact) <= rho ** iters * e0 * (1 + 1e-6) + 1e-12
    assert np.abs(b - b_exact).max() < 1e-4
