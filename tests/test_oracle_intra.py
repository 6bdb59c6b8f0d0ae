"""Pins of the oracle's intramolecular force field (reduced UFF-like form)."""
import math

import numpy as np
import pytest

from oracle import intra
from paper_2508_15522_gb300 import synth


def _four_atoms(phi_deg):
    """i-j-k-l with unit bonds, right angles at j and k, dihedral phi."""
    p = math.radians(phi_deg)
    return np.array([[1.0, 0, 0], [0, 0, 0], [0, 0, 1.0], [math.cos(p), math.sin(p), 1.0]])


def test_dihedral_angle_known_geometries():
    import torch
    for deg in (0.0, 60.0, 90.0, 180.0, -120.0):
        x = torch.tensor(_four_atoms(deg)[None])
        phi = float(intra.dihedral(x, 0, 1, 2, 3)[0])
        assert math.cos(phi) == pytest.approx(math.cos(math.radians(deg)), abs=1e-12)
        assert abs(math.sin(phi)) == pytest.approx(abs(math.sin(math.radians(deg))), abs=1e-12)


def _torsion_only(V=0.2, n=3, cn0=-1.0):
    m = synth.Molecule(["C"] * 4, _four_atoms(180.0), np.zeros(4), np.full(4, 1.9),
                       np.full(4, 0.07), np.full(4, 12.0))
    m.torsions = np.array([[0, 1, 2, 3]], np.int32)
    m.torsion_V = np.array([V]); m.torsion_n = np.array([n], np.int32)
    m.torsion_cos_nphi0 = np.array([cn0])
    return m


def test_torsion_energy_special_angles():
    """V/2 [1 - cos(n phi0) cos(n phi)] with n = 3, phi0 = 180 deg: zero at
    180 and 60 deg, V at 0 deg, V/2 at 90 deg."""
    m = _torsion_only()
    for deg, want in ((180.0, 0.0), (60.0, 0.0), (0.0, 0.2), (90.0, 0.1)):
        E, _ = intra.energy_forces(_four_atoms(deg)[None], m, terms=("torsion",))
        assert E[0] == pytest.approx(want, abs=1e-12)


def test_bond_and_angle_energy_closed_forms():
    """k_b (r - r0)^2 per bond and k_theta (cos theta - cos theta0)^2 per
    angle, on a three-atom molecule with chosen lengths and angle."""
    th, th0 = math.radians(100.0), math.radians(120.0)
    x = np.array([[1.2, 0.0, 0.0], [0.0, 0.0, 0.0], [0.9 * math.cos(th), 0.9 * math.sin(th), 0.0]])
    m = synth.Molecule(["C", "C", "O"], x.copy(), np.zeros(3), np.full(3, 1.9), np.full(3, 0.07), np.full(3, 12.0))
    m.bonds = np.array([[0, 1], [1, 2]], np.int32)
    m.bond_k = np.array([3.0, 5.0]); m.bond_r0 = np.array([1.0, 1.0])
    m.angles = np.array([[0, 1, 2]], np.int32)
    m.angle_k = np.array([0.7]); m.angle_cos0 = np.array([math.cos(th0)])
    Eb, _ = intra.energy_forces(x[None], m, terms=("bond",))
    assert Eb[0] == pytest.approx(3.0 * 0.2 ** 2 + 5.0 * 0.1 ** 2, abs=1e-12)
    Ea, _ = intra.energy_forces(x[None], m, terms=("angle",))
    assert Ea[0] == pytest.approx(0.7 * (math.cos(th) - math.cos(th0)) ** 2, abs=1e-12)


def test_reference_geometry_is_bonded_minimum():
    mol = synth.chain_molecule()
    E, F = intra.energy_forces(mol.xyz[None], mol, terms=("bond", "angle"))
    assert abs(E[0]) < 1e-20 and np.abs(F).max() < 1e-8


def test_exclusions_of_a_chain():
    ex = intra.excluded_pairs(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    allowed = {(i, j) for i in range(5) for j in range(i + 1, 5) if not ex[i, j]}
    assert allowed == {(0, 3), (0, 4), (1, 4)}


def test_nonbonded_single_pair():
    """Two unbonded atoms: Morse minimum at R_i + R_j with depth
    -eps_i eps_j, plus k_e q_i q_j / r."""
    m = synth.Molecule(["C", "O"], np.zeros((2, 3)), np.array([0.2, -0.2]), np.array([1.9, 1.7]),
                       np.array([0.07, 0.05]), np.array([12.0, 16.0]))
    r0 = 3.6
    x = np.array([[[0, 0, 0], [r0, 0, 0]]], float)
    E, F = intra.energy_forces(x, m, terms=("nonbonded",))
    assert E[0] == pytest.approx(-0.07 * 0.05 + 14.399645 * (-0.04) / r0, rel=1e-12)
    # Morse part exerts no force at its minimum; only Coulomb remains
    assert F[0, 1, 0] == pytest.approx(14.399645 * (-0.04) / r0 ** 2, rel=1e-9)


def test_invariance_and_zero_net_force_and_torque():
    mol = synth.random_flexible_molecule(24, 6, 7)
    g = synth.rng(41)
    x = mol.xyz + 0.1 * g.standard_normal(mol.xyz.shape)
    E, F = intra.energy_forces(x[None], mol)
    assert np.abs(F[0].sum(0)).max() < 1e-9
    assert np.abs(np.cross(x, F[0]).sum(0)).max() < 1e-9
    Rm = synth.quat_to_matrix(synth.random_quaternions(1, g))[0]
    E2, _ = intra.energy_forces((x @ Rm.T + np.array([3.0, -1.0, 2.0]))[None], mol)
    assert E2[0] == pytest.approx(E[0], rel=1e-12, abs=1e-12)


def test_forces_match_finite_difference():
    mol = synth.chain_molecule()
    x = mol.xyz + 0.05 * synth.rng(42).standard_normal(mol.xyz.shape)
    E, F = intra.energy_forces(x[None], mol)
    h = 1e-6
    for a in range(mol.n):
        for c in range(3):
            xp = x.copy(); xp[a, c] += h
            xm = x.copy(); xm[a, c] -= h
            fd = -(intra.energy_forces(xp[None], mol)[0][0] - intra.energy_forces(xm[None], mol)[0][0]) / (2 * h)
            assert fd == pytest.approx(F[0, a, c], abs=1e-6)
