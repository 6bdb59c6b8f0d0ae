"""Pins of the oracle's rigid-body kinematics, FIRE and NVE integrators."""
import math

import numpy as np
import pytest

from oracle import dynamics as dyn
from paper_2508_15522_gb300 import synth


def test_quaternion_matrix_known_rotation_and_orthonormal():
    q = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])   # 90 deg about z
    R = dyn.quat_matrix(q)
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    qs = synth.random_quaternions(20, synth.rng(1))
    Rs = dyn.quat_matrix(qs)
    assert np.allclose(np.einsum("rij,rkj->rik", Rs, Rs), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(Rs), 1.0)
    # composition: R(a (x) b) = R(a) R(b)
    a, b = qs[:10], qs[10:]
    assert np.allclose(dyn.quat_matrix(dyn.quat_mul(a, b)), Rs[:10] @ Rs[10:], atol=1e-13)


def test_rigid_reduce_pure_couple():
    """Forces +f and -f at +-b along x in the body frame: zero net force,
    torque 2 b f about z (body frame)."""
    body = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    F = np.array([[[0, 0.5, 0], [0, -0.5, 0]]])
    Ft, tau = dyn.rigid_reduce(F, np.array([[1.0, 0, 0, 0]]), body)
    assert np.allclose(Ft, 0) and np.allclose(tau, [[0, 0, 1.0]])


def _harmonic(k, center):
    def fn(x):
        d = x - center
        return 0.5 * k * np.sum(d * d, (1, 2)), -k * d, np.zeros(len(x), int)
    return fn


def test_fire_flexible_harmonic_converges_to_minimum():
    g = synth.rng(2)
    center = g.uniform(-1, 1, (1, 5, 3))
    x0 = center + g.uniform(-0.5, 0.5, (3, 5, 3))
    st = dyn.fire_flexible(x0, np.zeros_like(x0), np.full(5, 12.0), _harmonic(2.0, center),
                           3000, dyn.FireParams(f_conv=1e-6))
    assert (st["status"] & dyn.CONVERGED).all()
    assert np.abs(st["x"] - center).max() < 1e-6 / 2.0


def test_fire_zero_force_nothing_moves():
    x0 = synth.rng(3).uniform(0, 1, (2, 4, 3))
    fn = lambda x: (np.zeros(len(x)), np.zeros_like(x), np.zeros(len(x), int))
    st = dyn.fire_flexible(x0, np.zeros_like(x0), np.ones(4), fn, 10)
    assert np.array_equal(st["x"], x0) and (st["status"] == dyn.CONVERGED).all()
    assert (st["steps"] == 1).all()


def test_fire_uphill_velocity_is_reset():
    """P = F.v <= 0 zeroes v and halves dt (Bitzek 2006)."""
    center = np.zeros((1, 1, 3))
    x0 = np.array([[[1.0, 0, 0]]])
    v0 = np.array([[[0.3, 0, 0]]])           # moving away from the minimum
    p = dyn.FireParams()
    st = dyn.fire_flexible(x0, v0, np.array([1.0]), _harmonic(1.0, center), 1, p)
    assert st["dt"][0] == pytest.approx(p.dt_start * p.f_dec)
    # velocity restarted from zero: v = ACC F/m dt
    assert st["v"][0, 0, 0] == pytest.approx(dyn.ACC * (-1.0) * p.dt_start * p.f_dec)


def test_fire_rigid_converges_to_target_pose():
    """Every atom tied by a spring to a rigidly moved copy of the body: the
    minimum is that pose (net force and torque vanish there)."""
    mol = synth.c24h8o6_core()
    g = synth.rng(4)
    q_t = synth.random_quaternions(2, g)
    c_t = g.uniform(-1, 1, (2, 3))
    target = dyn.rigid_positions(c_t, q_t, mol.xyz)
    fn = _harmonic(0.5, target)
    # start slightly off the target pose
    dq = np.concatenate([np.ones((2, 1)), 0.15 * g.standard_normal((2, 3))], 1)
    q0 = dyn.quat_mul(q_t, dq / np.linalg.norm(dq, axis=1, keepdims=True))
    c0 = c_t + g.uniform(-0.4, 0.4, (2, 3))
    st = dyn.fire_rigid(c0, q0, np.zeros((2, 3)), np.zeros((2, 3)), mol.xyz, mol.mass, fn, 5000,
                        dyn.FireParams(f_conv=1e-6))
    assert (st["status"] & dyn.CONVERGED).all()
    x = dyn.rigid_positions(st["com"], st["quat"], mol.xyz)
    assert np.abs(x - target).max() < 1e-5


def test_velocity_verlet_second_order_and_exact_solution():
    """Harmonic oscillator: x(t) = A cos(w t); the energy error of velocity
    Verlet scales as dt^2."""
    k, m, A = 2.0, 3.0, 0.7
    w = math.sqrt(k * dyn.ACC / m)
    fn = _harmonic(k, np.zeros((1, 1, 3)))
    errs = []
    for dt in (0.4, 0.2):
        n = int(round(200 / dt))
        x, v, tr = dyn.nve_flexible(np.array([[[A, 0, 0]]]), np.zeros((1, 1, 3)), np.array([m]), fn, n, dt)
        assert x[0, 0, 0] == pytest.approx(A * math.cos(w * n * dt), abs=5e-3)
        errs.append(np.abs(tr[:, 0] - tr[0, 0]).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_no_squish_torque_free_symmetric_top_precession():
    """Torque-free symmetric top (I1 = I2): the body angular velocity
    precesses about axis 3 at Omega = (I3 - I1)/I1 * w3; kinetic energy and
    |L| are conserved (Euler's equations, closed form)."""
    # symmetric body in its principal frame: 4 equal masses in a square + 2 on the axis
    body = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 0.5], [0, 0, -0.5]], float)
    mass = np.array([1.0, 1, 1, 1, 2, 2])
    M, I, _ = dyn.rigid_constants(body, mass)
    assert I[0] == pytest.approx(I[1])
    fn = lambda x: (np.zeros(len(x)), np.zeros_like(x), np.zeros(len(x), int))
    w0 = np.array([[0.02, 0.0, 0.05]])
    dt, n = 0.5, 400
    com, q, v, w, tr = dyn.nve_rigid(np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), np.zeros((1, 3)),
                                     w0, body, mass, fn, n, dt)
    Om = (I[2] - I[0]) / I[0] * w0[0, 2]
    t = n * dt
    want = np.array([0.02 * math.cos(Om * t), 0.02 * math.sin(Om * t), 0.05])
    # sign of the precession depends on the convention; compare both senses
    alt = np.array([0.02 * math.cos(Om * t), -0.02 * math.sin(Om * t), 0.05])
    assert min(np.abs(w[0] - want).max(), np.abs(w[0] - alt).max()) < 2e-4
    L = I * w[0]
    assert np.linalg.norm(L) == pytest.approx(np.linalg.norm(I * w0[0]), rel=1e-9)
    # the splitting does not conserve the kinetic energy exactly: the error
    # is a bounded oscillation of order dt^2 (symplectic), no drift
    errs = []
    for h in (0.5, 0.25):
        *_, tr = dyn.nve_rigid(np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), np.zeros((1, 3)),
                               w0, body, mass, fn, int(4000 / h), h, record_every=int(40 / h))
        rel = np.abs(tr[:, 0] - tr[0, 0]) / tr[0, 0]
        assert rel[-1] < 0.5 * rel.max()           # returns: oscillation, not drift
        errs.append(rel.max())
    assert errs[0] < 1e-4 and 3.5 < errs[0] / errs[1] < 4.5


def test_no_squish_energy_error_second_order():
    """Rigid molecule in a smooth external field: the NVE energy fluctuation
    falls ~4x when dt halves."""
    mol = synth.c24h8o6_core()
    center = dyn.rigid_positions(np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), mol.xyz)
    fn = _harmonic(0.05, center)
    dq = np.array([[1.0, 0.05, -0.03, 0.04]]); dq /= np.linalg.norm(dq)
    errs = []
    for dt in (1.0, 0.5):
        *_, tr = dyn.nve_rigid(np.array([[0.2, -0.1, 0.1]]), dq, np.zeros((1, 3)), np.zeros((1, 3)),
                               mol.xyz, mol.mass, fn, int(round(400 / dt)), dt)
        errs.append(np.abs(tr[:, 0] - tr[0, 0]).max())
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_langevin_without_friction_is_velocity_verlet():
    g = np.random.default_rng(41)
    k = 0.7
    x0 = g.standard_normal((3, 4, 3)); v0 = 0.01 * g.standard_normal((3, 4, 3)); mass = np.full(4, 12.0)
    fn = lambda x: (0.5 * k * np.sum(x * x, (1, 2)), -k * x, np.zeros(len(x), int))
    xl, vl, _ = dyn.langevin_baoab(x0, v0, mass, fn, 50, 0.7, 300.0, 0.0, lambda s: g.standard_normal((3, 12)))
    xv, vv, _ = dyn.nve_flexible(x0, v0, mass, fn, 50, 0.7)
    assert np.allclose(xl, xv, atol=1e-12) and np.allclose(vl, vv, atol=1e-12)


def test_langevin_free_particles_reach_maxwell_boltzmann():
    g = np.random.default_rng(42)
    R, n, T, m = 50, 20, 300.0, 12.0
    fn = lambda x: (np.zeros(len(x)), np.zeros_like(x), np.zeros(len(x), int))
    x, v, _ = dyn.langevin_baoab(np.zeros((R, n, 3)), np.zeros((R, n, 3)), np.full(n, m), fn, 30, 1.0, T, 1.0,
                                  lambda s: g.standard_normal((R, 3 * n)))
    var = dyn.KB * T * dyn.ACC / m
    N = v.size
    assert abs(np.mean(v * v) / var - 1.0) < 5 * np.sqrt(2.0 / N)


def test_langevin_harmonic_configurational_temperature():
    """BAOAB samples the harmonic oscillator's positions exactly:
    <x^2> = kB T / k."""
    g = np.random.default_rng(43)
    R, n, T, k = 40, 10, 300.0, 1.0
    fn = lambda x: (0.5 * k * np.sum(x * x, (1, 2)), -k * x, np.zeros(len(x), int))
    x = np.zeros((R, n, 3)); v = np.zeros((R, n, 3))
    acc = []
    for block in range(40):
        x, v, _ = dyn.langevin_baoab(x, v, np.full(n, 12.0), fn, 50, 2.0, T, 0.05,
                                      lambda s: g.standard_normal((R, 3 * n)))
        if block >= 10:
            acc.append(np.mean(x * x))
    assert abs(np.mean(acc) / (dyn.KB * T / k) - 1.0) < 0.05


def test_langevin_noise_stream_is_standard_normal():
    z = dyn.langevin_noise(99, range(20), 7, 60).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size) and abs(z.var() - 1) < 6 * np.sqrt(2 / z.size)
    assert not np.array_equal(dyn.langevin_noise(99, [0], 7, 5), dyn.langevin_noise(99, [0], 8, 5))
