"""Pins of the oracle's flexible-pose builder (oracle/poses.py): dihedral
sign and values against closed forms, Rodrigues rotation against known
rotations, the rotatable bonds of a hand-checked chain and of a ring,
builder invariants (every dihedral set exactly, bond lengths, bond angles
and the centre of mass kept, no torsion change = rigid placement), Horn's
quaternion against an SVD (Kabsch) solution, and the round trip pose ->
positions -> pose."""
import math

import numpy as np
import pytest

from oracle import dynamics as odyn
from oracle import poses as P
from paper_2508_15522_gb300 import synth


@pytest.mark.parametrize("phi", [0.0, 0.3, 1.2, -2.0, 3.1, -math.pi / 2])
def test_dihedral_closed_form(phi):
    # a on +x, b at the origin, c on +z, d turned by phi about +z: IUPAC sign
    a, b, c = np.array([1.0, 0, 0]), np.zeros(3), np.array([0, 0, 1.5])
    d = np.array([2 * math.cos(phi), 2 * math.sin(phi), 1.5])
    assert P.dihedral(a, b, c, d) == pytest.approx(phi, abs=1e-12)


def test_dihedral_staggered_butane_anti():
    # zig-zag planar chain: anti (180 deg); cis: 0
    a, b, c, d = (np.array(v, float) for v in ([0, 1, 0], [0, 0, 0], [1, 0, 0], [1, -1, 0]))
    assert abs(abs(P.dihedral(a, b, c, d)) - math.pi) < 1e-12
    assert P.dihedral(a, b, c, np.array([1.0, 1, 0])) == pytest.approx(0.0, abs=1e-12)


def test_rotate_about_known_rotations():
    x = np.array([[1.0, 0, 0], [0, 2.0, 0]])
    y = P.rotate_about(x, np.zeros(3), np.array([0, 0, 1.0]), math.pi / 2)
    assert np.allclose(y, [[0, 1, 0], [-2, 0, 0]], atol=1e-14)
    z = P.rotate_about(x, np.array([1.0, 1, 1]), np.array([0.6, 0, 0.8]), 2 * math.pi)
    assert np.allclose(z, x, atol=1e-13)


def test_rotors_of_the_chain_molecule():
    # bonds 0-1 0-5 0-6 1-2 1-7 2-3 3-4 3-8 4-9; root = 5 (lowest index of
    # degree 1); depths 5:0 0:1 1,6:2 2,7:3 3:4 4,8:5 9:6
    m = synth.chain_molecule()
    rot = P.rotors(m.n, m.bonds, m.torsions)
    assert [r["quad"] for r in rot] == [(5, 0, 1, 2), (0, 1, 2, 3), (1, 2, 3, 4), (2, 3, 4, 9)]
    assert rot[0]["move"] == [1, 2, 3, 4, 7, 8, 9]
    assert rot[3]["move"] == [4, 9]


def test_ring_bonds_are_not_rotatable():
    # cyclopentane-like ring 0..4 with a tail 4-5-6-7 and a hydrogen 8 on 0
    bonds = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (4, 5), (5, 6), (6, 7), (0, 8)]
    torsions = [(4, 0, 1, 2), (0, 4, 5, 6), (4, 5, 6, 7)]
    rot = P.rotors(9, bonds, torsions)
    # root = 7 (degree 1, lower than 8): the ring bond 0-1 is dropped; the
    # tail bonds 5-6 (depth of 6: 1) and 4-5 (depth of 5: 2) remain, oriented
    # away from the root, d the lowest-index other neighbour of c
    quads = [r["quad"] for r in rot]
    assert quads == [(7, 6, 5, 4), (6, 5, 4, 0)]
    assert rot[0]["move"] == [0, 1, 2, 3, 4, 5, 8]
    assert rot[1]["move"] == [0, 1, 2, 3, 4, 8]


@pytest.fixture(scope="module")
def big():
    m = synth.random_flexible_molecule(60, 10, 5)
    return m, P.rotors(m.n, m.bonds, m.torsions)


def test_builder_sets_every_dihedral_and_keeps_geometry(big):
    m, rot = big
    assert len(rot) >= 8
    g = np.random.default_rng(3)
    theta = g.uniform(-math.pi, math.pi, len(rot))
    com = np.array([3.0, -1.0, 7.5])
    q = g.standard_normal(4)
    x = P.build(m.xyz, m.mass, rot, com, q, theta)
    got = np.array([P.dihedral(*(x[i] for i in r["quad"])) for r in rot])
    assert np.abs(np.angle(np.exp(1j * (got - theta)))).max() < 1e-12
    bl = lambda y: np.linalg.norm(y[m.bonds[:, 0]] - y[m.bonds[:, 1]], axis=1)
    assert np.abs(bl(x) - bl(m.xyz)).max() < 1e-12
    u = lambda y: y[m.angles[:, 0]] - y[m.angles[:, 1]]
    w = lambda y: y[m.angles[:, 2]] - y[m.angles[:, 1]]
    cosang = lambda y: np.sum(u(y) * w(y), 1) / np.linalg.norm(u(y), axis=1) / np.linalg.norm(w(y), axis=1)
    assert np.abs(cosang(x) - cosang(m.xyz)).max() < 1e-12
    assert np.allclose(P.centre_of_mass(x, m.mass), com, atol=1e-12)


def test_builder_without_torsion_change_is_rigid_placement(big):
    m, rot = big
    theta = np.array([P.dihedral(*(m.xyz[i] for i in r["quad"])) for r in rot])
    com = np.array([[1.0, 2.0, 3.0]])
    q = np.array([[0.5, 0.5, -0.5, 0.5]])
    x = P.build(m.xyz, m.mass, rot, com[0], q[0], theta)
    body = m.xyz - P.centre_of_mass(m.xyz, m.mass)
    assert np.abs(x - odyn.rigid_positions(com, q, body)[0]).max() < 1e-12
    # zero quaternion: no rotation
    x0 = P.build(m.xyz, m.mass, rot, com[0], np.zeros(4), theta)
    assert np.abs(x0 - (body + com[0])).max() < 1e-12


def test_horn_matches_svd_kabsch():
    g = np.random.default_rng(8)
    z = g.standard_normal((25, 3))
    mass = g.uniform(1, 16, 25)
    z -= (z * mass[:, None]).sum(0) / mass.sum()
    q_true = g.standard_normal(4)
    q_true /= np.linalg.norm(q_true)
    y = z @ odyn.quat_matrix(q_true).T + 0.01 * g.standard_normal((25, 3))
    y -= (y * mass[:, None]).sum(0) / mass.sum()
    q = P.horn_quaternion(z, y, mass)
    # Kabsch by singular value decomposition of the weighted covariance
    H = (z * mass[:, None]).T @ y
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(Vt.T @ U.T))])
    R_svd = Vt.T @ D @ U.T
    assert np.abs(odyn.quat_matrix(q) - R_svd).max() < 1e-12
    # exact data: the rotation itself
    q_exact = P.horn_quaternion(z, z @ odyn.quat_matrix(q_true).T, mass)
    assert np.abs(q_exact - q_true * np.sign(q_true[0])).max() < 1e-12


def test_targets_invert_the_builder(big):
    m, rot = big
    g = np.random.default_rng(4)
    for _ in range(3):
        theta = g.uniform(-math.pi, math.pi, len(rot))
        q = g.standard_normal(4)
        q /= np.linalg.norm(q)
        com = g.uniform(-5, 5, 3)
        x = P.build(m.xyz, m.mass, rot, com, q, theta)
        c2, q2, t2 = P.targets(m.xyz, m.mass, rot, x)
        assert np.allclose(c2, com, atol=1e-12)
        assert np.abs(np.angle(np.exp(1j * (t2 - theta)))).max() < 1e-12
        assert abs(abs(np.dot(q2, q)) - 1.0) < 1e-12
        assert np.abs(P.build(m.xyz, m.mass, rot, c2, q2, t2) - x).max() < 1e-11
