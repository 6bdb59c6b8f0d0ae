"""Grid geometry, grid construction and grid-interpolated energies/forces.

Oracle (test infrastructure).  Follows Sec. 3 (channels C, P, L and their
combination, Eqs. E, E_Coulomb, E_Morse, V_Morse), Sec. 4 (folding into the
substrate tile; Ewald electrostatics) and Sec. 5 (B-spline fit and
tricubic interpolation).

Grid geometry reading: for a box length L and target spacing h the node
count is n = ceil(L/h - 1e-9) and the actual spacing L/n; x and y are
periodic with period L (the box must be a lattice period of the substrate),
z is not.

Ghost nodes (reading of the z boundary, which the paper leaves open): the
fit clamps the coefficients at the lowest node plane, which makes the
interpolant first order in the cell above it.  With ``ghost`` = G > 0 the
node values are also computed on G planes below the box (z0 - G h ...
z0 - h) and fitted with the rest; the box's lower face z0 stays the floor
of the grid (points below it are flagged), and the clamped end acts G
planes further down, where its error has decayed (by about 2 - sqrt(3)
per plane) before it reaches the floor cell.
"""
from __future__ import annotations

import math

import numpy as np

from . import bspline, substrate

CHANNELS = ("C", "P", "L")


def grid_dims(length, spacing):
    n = [int(math.ceil(L / spacing - 1e-9)) for L in length]
    return tuple(n), tuple(L / k for L, k in zip(length, n))


def node_origin(origin, length, spacing, ghost=0):
    """Coordinates of the first node: the box origin, lowered by ``ghost``
    z spacings."""
    _, h = grid_dims(length, spacing)
    return (origin[0], origin[1], origin[2] - ghost * h[2])


def node_points(origin, length, spacing, ghost=0):
    """All node coordinates, shape (nx*ny*(nz+ghost), 3), z fastest; the
    node count in z includes the ghost planes below the box."""
    n, h = grid_dims(length, spacing)
    n = (n[0], n[1], n[2] + ghost)
    o = node_origin(origin, length, spacing, ghost)
    axes = [o[a] + np.arange(n[a]) * h[a] for a in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), n, h


def node_values(sub, origin, length, spacing, channels=("C", "P", "L"),
                alpha=1.5, rcut=17.0, ewald=None, ghost=0):
    """Channel values at every node (Sec. 3): V^C in volts (Ewald, Sec. 4),
    V^P and V^L by direct sums (Eq. V_Morse).  Shape (C, nx, ny, nz + ghost)."""
    pts, n, h = node_points(origin, length, spacing, ghost)
    out = []
    VP = VL = None
    for ch in channels:
        if ch == "C":
            vc, _ = substrate.coulomb_channel(pts, sub.xyz, sub.q, sub.cell, ewald)
            out.append(vc)
        else:
            if VP is None:
                VP, VL, _, _ = substrate.morse_channels(pts, sub.xyz, sub.R, sub.eps,
                                                        sub.cell, alpha, rcut)
            out.append(VP if ch == "P" else VL)
    return np.stack(out).reshape((len(channels),) + n), n, h


def build_grid(sub, origin, length, spacing, channels=("C", "P", "L"),
               alpha=1.5, rcut=17.0, ewald=None, ghost=0):
    """Node values and exact B-spline coefficients (C, nx, ny, nz + ghost);
    with ghost > 0 the first node lies at node_origin(...), ghost planes
    below the box."""
    vals, n, h = node_values(sub, origin, length, spacing, channels, alpha, rcut, ewald, ghost)
    return vals, bspline.fit_exact(vals), n, h


def grid_energy_forces(coefs, channels, origin, spacing, points, Q, R, eps,
                       alpha=1.5, dtype=np.float64, ghost=0):
    """Per-atom E_i = Q_i f_C + P_i f_P + L_i f_L and F_i = -grad E_i from the
    interpolated channels (Eqs. E, E_Coulomb, E_Morse; forces are the
    analytic gradient of the interpolant, Sec. 5).  The per-atom factors are
    formed in float64 and rounded to ``dtype``.  ``origin`` is the first
    node; ``ghost`` planes of it lie below the floor (flagged points).
    Returns (E (N,), F (N,3), below (N,))."""
    f, g, below = bspline.eval_grid(coefs, origin, spacing, points, dtype, below_u=ghost)
    P_, L_ = substrate.factor_params(R, eps, alpha)
    fac = {"C": np.asarray(Q, np.float64), "P": P_, "L": L_}
    E = np.zeros(len(points), dtype)
    G = np.zeros((len(points), 3), dtype)
    for c, ch in enumerate(channels):
        w = fac[ch].astype(dtype)
        E = E + w * f[:, c]
        G = G + w[:, None] * g[:, c, :]
    return E, -G, below
