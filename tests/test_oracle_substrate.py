"""Pins of the oracle's substrate channels, Ewald sum, pairwise reference and
grid construction (Sec. 3, Sec. 4, Sec. 5)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import bspline, grid, substrate
from paper_2508_15522_gb300 import synth


class _Sub:
    pass


def _single_atom_substrate(R=1.8, eps=0.09, q=0.0, L=40.0):
    s = _Sub()
    s.xyz = np.array([[0.0, 0.0, 0.0]])
    s.R = np.array([R]); s.eps = np.array([eps]); s.q = np.array([q])
    s.cell = np.diag([L, L, 3 * L])
    return s


def test_morse_factorisation_identity():
    """Eq. E_Morse = P_i V^P + L_i V^L with the factors of Eq. V_Morse."""
    sub = synth.rocksalt_slab(ncell=2)
    g = synth.rng(31)
    pts = g.uniform(0, 1, (60, 3)) * np.array([11.28, 11.28, 6.0]) + np.array([0, 0, sub.z_top + 1.5])
    mol = synth.c24h8o6_core()
    Ri = np.resize(mol.R, 60); ei = np.resize(mol.eps, 60)
    E_direct, G_direct = substrate.morse_pair_energy(pts, Ri, ei, sub.xyz, sub.R, sub.eps, sub.cell)
    VP, VL, gP, gL = substrate.morse_channels(pts, sub.xyz, sub.R, sub.eps, sub.cell)
    P, L = substrate.factor_params(Ri, ei, 1.5)
    assert np.abs(P * VP + L * VL - E_direct).max() < 1e-13 * np.abs(P * VP).max() + 1e-15
    assert np.abs(P[:, None] * gP + L[:, None] * gL - G_direct).max() < 1e-12 * np.abs(P[:, None] * gP).max()


def test_single_pair_morse_minimum():
    """One substrate atom: the pair energy is minimal at R_i + R_j with
    depth -eps_i eps_j (Eq. E_Morse)."""
    sub = _single_atom_substrate()
    Ri, ei = 1.6, 0.05
    z = np.linspace(2.0, 6.0, 4001)
    pts = np.stack([np.full_like(z, 20.0), np.full_like(z, 20.0), z], 1)
    sub.xyz = np.array([[20.0, 20.0, 0.0]])
    E, _ = substrate.morse_pair_energy(pts, np.full(len(z), Ri), np.full(len(z), ei),
                                       sub.xyz, sub.R, sub.eps, sub.cell)
    k = np.argmin(E)
    assert z[k] == pytest.approx(Ri + 1.8, abs=1e-3)
    assert E[k] == pytest.approx(-ei * 0.09, rel=1e-6)


def test_morse_gradient_finite_difference():
    sub = synth.rocksalt_slab(ncell=2)
    pts = synth.rng(32).uniform(0, 1, (10, 3)) * np.array([8, 8, 3]) + np.array([0, 0, sub.z_top + 2])
    VP, VL, gP, gL = substrate.morse_channels(pts, sub.xyz, sub.R, sub.eps, sub.cell)
    h = 1e-5
    for a in range(3):
        d = np.zeros(3); d[a] = h
        p1 = substrate.morse_channels(pts + d, sub.xyz, sub.R, sub.eps, sub.cell)
        m1 = substrate.morse_channels(pts - d, sub.xyz, sub.R, sub.eps, sub.cell)
        assert np.abs((p1[0] - m1[0]) / (2 * h) - gP[:, a]).max() < 1e-7
        assert np.abs((p1[1] - m1[1]) / (2 * h) - gL[:, a]).max() < 1e-7


def test_ewald_madelung_constant():
    """Site potential in bulk rock salt: -M q / r0 (M = 1.747565)."""
    M = read_golden("madelung_nacl.txt")[0][0]
    a = 5.64
    base = np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]])
    X = np.concatenate([base, base + np.array([.5, 0, 0])]) * a
    q = np.array([1.0] * 4 + [-1.0] * 4)
    beta, rc, kmax = substrate.ewald_params(1e-12, 8.0)
    phi, _ = substrate.ewald_potential(X[:1], X, q, np.eye(3) * a, beta, rc, kmax,
                                       slab=False, exclude=0)
    assert -phi[0] * (a / 2) == pytest.approx(M, abs=2e-6)


def test_ewald_equals_direct_image_sums_of_a_neutral_dipole_free_cell():
    """Bulk Ewald vs the direct Coulomb sum over expanding cubes of images:
    for a neutral cell with no dipole and no second moment (rock salt on the
    quarter positions) the cube sums converge to the Ewald potential itself,
    faster than 1/N^3."""
    a = 5.64
    plus = np.array([[.25, .25, .25], [.75, .75, .25], [.75, .25, .75], [.25, .75, .75]])
    minus = np.array([[.75, .75, .75], [.25, .25, .75], [.25, .75, .25], [.75, .25, .25]])
    X = np.concatenate([plus, minus]) * a
    q = np.array([1.0] * 4 + [-1.0] * 4)
    pts = np.array([[0.03, 0.11, 0.07], [0.61, 0.12, 0.44], [0.37, 0.71, 0.93], [0.5, 0.5, 0.5]]) * a
    beta, rc, kmax = substrate.ewald_params(1e-12, 8.0)
    phi, _ = substrate.ewald_potential(pts, X, q, np.eye(3) * a, beta, rc, kmax, slab=False)
    errs = []
    for N in (6, 12):
        r = np.arange(-N, N + 1)
        n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3) * a
        direct = np.array([(q[None, :] / np.linalg.norm(p[None, None, :] - X[None] - n[:, None, :], axis=2)).sum()
                           for p in pts])
        errs.append(np.abs(direct - phi).max())
    assert errs[1] < 5e-7 and errs[1] < errs[0] / 8


def test_ewald_matches_exact_slab_fourier_sum():
    """Above a neutral slab the EW3DC potential equals the exact 2D-periodic
    open-boundary potential (Sec. 4: vacuum padding + dipole correction)."""
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, 0.2)
    pts = synth.uniform_points(25, box, 33, zband=(0.0, 8.0))
    ew = substrate.ewald_params(1e-12, 9.0)
    phi, _ = substrate.ewald_potential(pts, sub.xyz, sub.q, sub.cell, *ew)
    ref = substrate.slab_fourier_potential(pts, sub.xyz, sub.q, sub.cell[0], sub.cell[1], gmax=60.0)
    assert np.abs(phi - ref).max() < 1e-11


def test_ewald_independent_of_splitting_even_when_charged():
    """The neutralising-background term makes phi independent of beta."""
    g = synth.rng(34)
    X = g.uniform(0, 1, (7, 3)) * np.array([6.0, 7.0, 3.0])
    q = g.uniform(-1, 1, 7)                       # net charge != 0
    cell = np.array([[6.0, 0, 0], [1.0, 7.0, 0], [0, 0, 20.0]])
    pts = g.uniform(0, 1, (9, 3)) * np.array([6, 7, 8]) + np.array([0, 0, 3.5])
    a = substrate.ewald_potential(pts, X, q, cell, *substrate.ewald_params(1e-13, 7.0))
    b = substrate.ewald_potential(pts, X, q, cell, *substrate.ewald_params(1e-13, 10.0))
    assert np.abs(a[0] - b[0]).max() < 1e-10
    assert np.abs(a[1] - b[1]).max() < 1e-9


def test_ewald_gradient_finite_difference():
    sub = synth.rocksalt_slab(ncell=2)
    pts = synth.rng(35).uniform(0, 1, (5, 3)) * np.array([8, 8, 4]) + np.array([0, 0, sub.z_top + 1.5])
    ew = substrate.ewald_params(1e-12, 9.0)
    _, gr = substrate.ewald_potential(pts, sub.xyz, sub.q, sub.cell, *ew)
    h = 1e-4
    for a in range(3):
        d = np.zeros(3); d[a] = h
        fp = substrate.ewald_potential(pts + d, sub.xyz, sub.q, sub.cell, *ew)[0]
        fm = substrate.ewald_potential(pts - d, sub.xyz, sub.q, sub.cell, *ew)[0]
        assert np.abs((fp - fm) / (2 * h) - gr[:, a]).max() < 1e-9


def test_slab_fourier_leading_shell_closed_form():
    """One checkerboard layer (+q at (0,0), (a/2,a/2); -q at (a/2,0),
    (0,a/2) in an a x a cell): far above it only the |G| = 2 pi sqrt2/a shell
    survives, phi = 16 q/(a sqrt2) exp(-|G| z) cos(2 pi x/a) cos(2 pi y/a)."""
    a, q = 5.64, 0.7
    X = np.array([[0, 0, 0], [a / 2, a / 2, 0], [a / 2, 0, 0], [0, a / 2, 0]])
    Q = np.array([q, q, -q, -q])
    g = synth.rng(36)
    pts = np.stack([g.uniform(0, a, 20), g.uniform(0, a, 20), np.full(20, 8.0)], 1)
    phi = substrate.slab_fourier_potential(pts, X, Q, [a, 0, 0], [0, a, 0], gmax=30.0)
    G = 2 * math.pi * math.sqrt(2) / a
    ref = 16 * q / (a * math.sqrt(2)) * math.exp(-G * 8.0) * np.cos(2 * np.pi * pts[:, 0] / a) * np.cos(2 * np.pi * pts[:, 1] / a)
    G2 = 2 * math.pi * math.sqrt(10) / a
    assert np.abs(phi - ref).max() < 40 * q / a * math.exp(-G2 * 8.0)
    assert np.abs(ref).max() > 1e3 * np.abs(phi - ref).max()


def test_grid_dims_golden():
    for Lx, Ly, Lz, h, nx, ny, nz in read_golden("grid_dims.txt"):
        n, _ = grid.grid_dims((Lx, Ly, Lz), h)
        assert n == (int(nx), int(ny), int(nz))


def test_tile_periodicity_of_pairwise_reference():
    """The 2a x 2a tile is a period of the pristine slab (folding, Sec. 4)."""
    sub = synth.rocksalt_slab(ncell=2)
    g = synth.rng(37)
    pts = g.uniform(0, 1, (8, 3)) * np.array([11.28, 11.28, 4.0]) + np.array([0, 0, sub.z_top + 2])
    mol = synth.chain_molecule()
    Q, R, eps = mol.q[:8], mol.R[:8], mol.eps[:8]
    ew = substrate.ewald_params(1e-12, 9.0)
    E0, F0 = substrate.pairwise_reference(pts, Q, R, eps, sub, ewald=ew)
    for sh in ((11.28, 0, 0), (0, 11.28, 0), (5.64, -5.64, 0)):
        E1, F1 = substrate.pairwise_reference(pts + np.array(sh), Q, R, eps, sub, ewald=ew)
        assert np.abs(E1 - E0).max() < 1e-11 and np.abs(F1 - F0).max() < 1e-10


def test_pairwise_force_is_minus_gradient():
    sub = synth.rocksalt_slab(ncell=2)
    mol = synth.chain_molecule()
    pts = synth.rng(38).uniform(0, 1, (mol.n, 3)) * np.array([8, 8, 3]) + np.array([0, 0, sub.z_top + 2.2])
    ew = substrate.ewald_params(1e-12, 9.0)
    E, F = substrate.pairwise_reference(pts, mol.q, mol.R, mol.eps, sub, ewald=ew)
    h = 1e-5
    for a in range(3):
        d = np.zeros(3); d[a] = h
        Ep, _ = substrate.pairwise_reference(pts + d, mol.q, mol.R, mol.eps, sub, ewald=ew)
        Em, _ = substrate.pairwise_reference(pts - d, mol.q, mol.R, mol.eps, sub, ewald=ew)
        assert np.abs(-(Ep - Em) / (2 * h) - F[:, a]).max() < 1e-7


@pytest.mark.slow
def test_grid_interpolation_vs_pairwise_morse_at_0p1():
    """Morse channels on a 0.1 A grid over the a x a tile: interpolated atom
    energies match the direct pair sum within the classical cubic-spline
    bound (5/384) h^4 f'''' summed over the three axes, f'''' <= (2 alpha)^4 f
    for the Pauli channel (Sec. 5 accuracy claim; Hall & Meyer 1976)."""
    sub = synth.rocksalt_slab(ncell=2)
    a = 5.64
    origin, length = (0.0, 0.0, sub.z_top + 1.0), (a, a, 5.0)
    vals, coefs, n, h = grid.build_grid(sub, origin, length, 0.1, channels=("P", "L"))
    mol = synth.c24h8o6_core()
    g = synth.rng(39)
    pts = np.stack([g.uniform(0, a, 76), g.uniform(0, a, 76), g.uniform(2.0, 4.0, 76) + sub.z_top + 1.0], 1)
    Q = np.zeros(76); R = np.resize(mol.R, 76); eps = np.resize(mol.eps, 76)
    E, F, below = grid.grid_energy_forces(coefs, ("P", "L"), origin, h, pts, Q, R, eps)
    Eref, Fref = substrate.pairwise_reference(pts, Q, R, eps, sub)
    P, _ = substrate.factor_params(R, eps, 1.5)
    VP, _, _, _ = substrate.morse_channels(pts, sub.xyz, sub.R, sub.eps, sub.cell)
    bound = 3 * 5 / 384 * 0.1 ** 4 * 3.0 ** 4 * np.abs(P * VP) * math.exp(3.0 * 0.2) + 1e-9
    assert not below.any()
    assert (np.abs(E - Eref) <= bound).all()
    assert np.abs(E - Eref).max() < 5e-5          # eV per atom at 0.1 A
    assert np.abs(F - Fref).max() < 2e-3


@pytest.mark.slow
def test_ghost_nodes_floor_cells_vs_pairwise_morse():
    """Eight ghost planes below the floor: Morse energies of atoms in the
    first three cells above the floor (1.0-1.3 A above the top ions) match
    the direct pair sums within the interior cubic-spline bound of the test
    above (Hall & Meyer), where the clamped fit without ghost planes is off
    by far more; the node values of the planes above the floor are those of
    the grid without ghosts."""
    sub = synth.rocksalt_slab(ncell=2)
    a, G = 5.64, 8
    origin, length = (0.0, 0.0, sub.z_top + 1.0), (a, a, 2.0)
    mol = synth.c24h8o6_core()
    g = synth.rng(41)
    pts = np.stack([g.uniform(0, a, 76), g.uniform(0, a, 76), g.uniform(0.0, 0.3, 76) + sub.z_top + 1.0], 1)
    Q = np.zeros(76); R = np.resize(mol.R, 76); eps = np.resize(mol.eps, 76)
    Eref, _ = substrate.pairwise_reference(pts, Q, R, eps, sub)
    P, _ = substrate.factor_params(R, eps, 1.5)
    VP, _, _, _ = substrate.morse_channels(pts, sub.xyz, sub.R, sub.eps, sub.cell)
    bound = 3 * 5 / 384 * 0.1 ** 4 * 3.0 ** 4 * np.abs(P * VP) * math.exp(3.0 * 0.1) + 1e-9
    err = {}
    for ghost in (0, G):
        vals, coefs, n, h = grid.build_grid(sub, origin, length, 0.1, channels=("P", "L"), ghost=ghost)
        o = grid.node_origin(origin, length, 0.1, ghost)
        E, F, below = grid.grid_energy_forces(coefs, ("P", "L"), o, h, pts, Q, R, eps, ghost=ghost)
        assert not below.any()
        err[ghost] = np.abs(E - Eref)
        if ghost:
            v0, _, _, _ = grid.build_grid(sub, origin, length, 0.1, channels=("P", "L"))
            assert np.abs(vals[:, :, :, ghost:] - v0).max() <= 1e-12 * np.abs(v0).max()
    assert (err[G] <= bound).all()
    assert (err[0] > bound).mean() > 0.5 and err[0].max() > 10 * err[G].max()
