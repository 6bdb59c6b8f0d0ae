"""Pins of the oracle's random starting poses and RMSD uniqueness filter."""
import numpy as np
import pytest

from oracle import sampling
from oracle.dynamics import quat_matrix
from paper_2508_15522_gb300 import synth

TILE = (11.28, 11.28)


@pytest.fixture(scope="module")
def body():
    return synth.c24h8o6_core().xyz.astype(np.float64)


def test_rmsd_translation_tile_and_sign(body):
    p = np.array([1.0, 2.0, 5.0, 0.5, 0.5, 0.5, 0.5])
    q = p.copy(); q[:3] += [0.3, -0.4, 0.0]
    assert sampling.rmsd(body, p, q, TILE) == pytest.approx(0.5)
    q = p.copy(); q[0] += TILE[0]; q[1] -= 2 * TILE[1]
    assert sampling.rmsd(body, p, q, TILE) == pytest.approx(0.0, abs=1e-12)
    q = p.copy(); q[3:] *= -3.0                        # -q, unnormalised: same rotation
    assert sampling.rmsd(body, p, q, TILE) == pytest.approx(0.0, abs=1e-12)
    q = p.copy(); q[2] += TILE[0]                      # z is not periodic
    assert sampling.rmsd(body, p, q, TILE) == pytest.approx(TILE[0])


def test_rmsd_rotation_closed_form(body):
    """Rotation by theta about z: |R b - b|^2 = 2 (1 - cos theta)(bx^2 + by^2)."""
    th = 0.3
    p = np.array([0, 0, 5.0, 1, 0, 0, 0])
    q = np.array([0, 0, 5.0, np.cos(th / 2), 0, 0, np.sin(th / 2)])
    ref = np.sqrt(np.mean(2 * (1 - np.cos(th)) * (body[:, 0] ** 2 + body[:, 1] ** 2)))
    assert sampling.rmsd(body, p, q, TILE) == pytest.approx(ref, rel=1e-12)


def test_dup_of_constructed_set(body):
    p0 = np.array([1.0, 2.0, 5.0, 1, 0, 0, 0])
    poses = [p0, p0 + [0.05, 0, 0, 0, 0, 0, 0], p0 + [1.0, 0, 0, 0, 0, 0, 0],
             p0 + [TILE[0], 0, 0, 0, 0, 0, 0], p0 + [1.02, 0.0, 0.03, 0, 0, 0, 0]]
    assert sampling.dup_of(body, poses, TILE, 0.1).tolist() == [-1, 0, -1, 0, 2]


def test_random_poses_ranges_and_uniform_orientation(body):
    n = 4000
    P = sampling.random_poses(body, n, 77, (-1.0, 2.0), TILE, 4.0, 6.0, 1.5)
    assert np.all((P[:, 0] >= -1.0) & (P[:, 0] < -1.0 + TILE[0]))
    assert np.all((P[:, 1] >= 2.0) & (P[:, 1] < 2.0 + TILE[1]))
    assert np.allclose(np.linalg.norm(P[:, 3:], axis=1), 1.0)
    low = np.array([sampling.positions(body, p)[:, 2].min() for p in P[:200]])
    assert np.all(low >= 1.5 - 1e-9)
    lifted = P[:200, 2] > 6.0
    assert lifted.any() and np.allclose(low[lifted], 1.5)
    # uniform on SO(3): E[R] = 0 and E[w^2] = 1/4
    R = quat_matrix(P[:, 3:])
    assert np.abs(R.mean(0)).max() < 4 / np.sqrt(n)
    assert np.mean(P[:, 3] ** 2) == pytest.approx(0.25, abs=4 * 0.15 / np.sqrt(n))


def test_rmsd_xyz_translation_tile_image_and_conformation():
    g = np.random.default_rng(12)
    a = g.standard_normal((9, 3)) + [3.0, 4.0, 8.0]
    b = a + [0.3, 0.0, -0.4]
    assert sampling.rmsd_xyz(a, b, TILE) == pytest.approx(0.5)
    assert sampling.rmsd_xyz(a, a + [2 * TILE[0], -TILE[1], 0.0], TILE) == pytest.approx(0.0, abs=1e-12)
    c = a.copy(); c[0] += [0.0, 0.0, 0.9]                       # one atom moved: conformation counts
    assert sampling.rmsd_xyz(a, c, TILE) == pytest.approx(0.3)
    # a rotation about the mean position is not aligned away
    ang = 0.2
    Rz = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1.0]])
    m = a.mean(0)
    r = (a - m) @ Rz.T + m
    ref = np.sqrt(np.mean(np.sum((a - r) ** 2, 1)))
    assert sampling.rmsd_xyz(a, r, TILE) == pytest.approx(ref) and ref > 0.1
    assert sampling.dup_of_xyz([a, b, a + [TILE[0], 0, 0], c, b + [0.01, 0, 0]], TILE, 0.1).tolist() == \
        [-1, -1, 0, -1, 1]
