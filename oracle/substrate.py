"""Substrate potentials and the FP64 pairwise reference (Sec. 3, Sec. 4).

Oracle (test infrastructure).  Units: A, eV, e.  Coulomb potentials are
returned in volts (eV per e): the paper writes Eq. E_Coulomb in Gaussian
units; the reading is V^C = k_e * sum_j Q_j / |r - r_j| with
k_e = 14.399645 eV*A/e^2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

KE = 14.399645  # eV*A/e^2


def factor_params(R, eps, alpha):
    """Per-atom Morse factors of Eq. V_Morse: P_i = eps_i exp(2 alpha R_i),
    L_i = -2 eps_i exp(alpha R_i)."""
    R = np.asarray(R, np.float64)
    eps = np.asarray(eps, np.float64)
    return eps * np.exp(2 * alpha * R), -2 * eps * np.exp(alpha * R)


def _inplane_images(cell, extent):
    """Integer pairs (n1, n2) of in-plane lattice translations with
    |n1 A1 + n2 A2| <= extent (a superset of those that can bring an atom of
    the cell within ``extent`` - span of a point folded into the cell)."""
    a1, a2 = cell[0, :2], cell[1, :2]
    area = abs(a1[0] * a2[1] - a1[1] * a2[0])
    h1 = area / np.linalg.norm(a2)
    h2 = area / np.linalg.norm(a1)
    n1 = int(math.ceil(extent / h1)) + 1
    n2 = int(math.ceil(extent / h2)) + 1
    return [(i, j) for i in range(-n1, n1 + 1) for j in range(-n2, n2 + 1)
            if np.linalg.norm(i * a1 + j * a2) <= extent]


def _fold_points(points, cell):
    """Translate points by in-plane lattice vectors into the supercell (the
    sums below are lattice-periodic, so this changes nothing but keeps the
    image ranges small)."""
    A = cell[:2, :2].T
    frac = np.linalg.solve(A, points[:, :2].T).T
    shift = np.floor(frac) @ cell[:2, :2]
    out = points.copy()
    out[:, :2] -= shift
    return out


def morse_channels(points, sub_xyz, sub_R, sub_eps, cell, alpha=1.5, rcut=17.0):
    """V^P, V^L of Eq. V_Morse at the points and their gradients.

    V^P(r) = sum_j eps_j exp(-2 alpha (|r - r_j| - R_j)),
    V^L(r) = sum_j eps_j exp(-alpha (|r - r_j| - R_j)),
    summed over the substrate atoms and all their in-plane periodic images
    with |r - r_j| < rcut (hard cutoff, reading of Sec. 6's 17 A cutoff).
    Returns (VP (N,), VL (N,), gradVP (N,3), gradVL (N,3)).
    """
    P = _fold_points(np.asarray(points, np.float64), cell)
    X = np.asarray(sub_xyz, np.float64)
    VP = np.zeros(len(P)); VL = np.zeros(len(P))
    gP = np.zeros((len(P), 3)); gL = np.zeros((len(P), 3))
    span = np.linalg.norm(cell[0, :2]) + np.linalg.norm(cell[1, :2])
    for (n1, n2) in _inplane_images(cell, rcut + span):
        shift = n1 * cell[0] + n2 * cell[1]
        d = P[:, None, :] - (X[None, :, :] + shift)
        r = np.sqrt(np.sum(d * d, -1))
        inside = r < rcut
        eP = np.where(inside, sub_eps * np.exp(-2 * alpha * (r - sub_R)), 0.0)
        eL = np.where(inside, sub_eps * np.exp(-alpha * (r - sub_R)), 0.0)
        VP += eP.sum(1)
        VL += eL.sum(1)
        rs = np.where(r > 0, r, 1.0)
        gP += np.sum((-2 * alpha * eP / rs)[..., None] * d, 1)
        gL += np.sum((-alpha * eL / rs)[..., None] * d, 1)
    return VP, VL, gP, gL


def morse_pair_energy(points, R_i, eps_i, sub_xyz, sub_R, sub_eps, cell,
                      alpha=1.5, rcut=17.0):
    """Direct (unfactorised) Morse energy of Eq. E_Morse for atoms at the
    points with parameters (R_i, eps_i), and its gradient:
    E_i = sum_j eps_i eps_j [exp(-2a(d - R_i - R_j)) - 2 exp(-a(d - R_i - R_j))].
    """
    P = _fold_points(np.asarray(points, np.float64), cell)
    X = np.asarray(sub_xyz, np.float64)
    R_i = np.asarray(R_i, np.float64)[:, None]
    eps_i = np.asarray(eps_i, np.float64)[:, None]
    E = np.zeros(len(P)); G = np.zeros((len(P), 3))
    span = np.linalg.norm(cell[0, :2]) + np.linalg.norm(cell[1, :2])
    for (n1, n2) in _inplane_images(cell, rcut + span):
        shift = n1 * cell[0] + n2 * cell[1]
        d = P[:, None, :] - (X[None, :, :] + shift)
        r = np.sqrt(np.sum(d * d, -1))
        inside = r < rcut
        x = r - R_i - sub_R[None, :]
        ep = eps_i * sub_eps[None, :]
        e2 = np.exp(-2 * alpha * x)
        e1 = np.exp(-alpha * x)
        E += np.where(inside, ep * (e2 - 2 * e1), 0.0).sum(1)
        dEdr = np.where(inside, ep * (-2 * alpha * e2 + 2 * alpha * e1), 0.0)
        rs = np.where(r > 0, r, 1.0)
        G += np.sum((dEdr / rs)[..., None] * d, 1)
    return E, G


# ---------------------------------------------------------------------------
# electrostatics
# ---------------------------------------------------------------------------
def ewald_params(tol=1e-10, rcut=12.0):
    """(beta, rcut, kmax) so that the real-space tail erfc(beta*rcut) and the
    reciprocal tail exp(-kmax^2/(4 beta^2)) are both ~tol."""
    s = math.sqrt(-math.log(tol))
    beta = s / rcut
    return beta, rcut, 2 * beta * s


def _kvectors(cell, kmax):
    B = 2 * np.pi * np.linalg.inv(cell).T        # rows b1, b2, b3
    M = [int(math.ceil(kmax * np.linalg.norm(cell[i]) / (2 * np.pi))) + 1 for i in range(3)]
    m = np.array(np.meshgrid(*[np.arange(-Mi, Mi + 1) for Mi in M], indexing="ij")).reshape(3, -1).T
    K = m @ B
    k2 = np.sum(K * K, 1)
    keep = (k2 > 0) & (k2 < kmax * kmax)
    return K[keep], k2[keep]


def ewald_potential(points, xyz, q, cell, beta, rcut, kmax, slab=True, exclude=None):
    """Electrostatic potential (e/A, Gaussian units) of point charges in the
    3D-periodic cell ``cell`` (rows A1, A2, A3), and its gradient, by Ewald
    summation (Sec. 4):

    phi(r) = sum_j sum_n q_j erfc(beta d)/d                   (d = |r - r_j - n| < rcut)
           + (4 pi / V) sum_{k != 0, |k| < kmax} exp(-k^2/4beta^2)/k^2 Re[S(k) exp(i k.r)]
           - pi Q / (beta^2 V)                                 (neutralising background)
           + (4 pi / V) M_z z                                  (slab dipole correction, Yeh-Berkowitz)

    with S(k) = sum_j q_j exp(-i k.r_j), Q = sum q_j, M_z = sum q_j z_j.
    ``slab=False`` drops the dipole term (bulk 3D periodicity).  ``exclude``
    = index of an atom sitting at every point: its n = 0 real-space term is
    skipped and its self term -2 beta q/sqrt(pi) added (site potential).
    """
    P = _fold_points(np.asarray(points, np.float64), cell)
    X = np.asarray(xyz, np.float64)
    q = np.asarray(q, np.float64)
    V = abs(np.linalg.det(cell))
    phi = np.zeros(len(P)); grad = np.zeros((len(P), 3))
    # real space: every lattice translation that can bring an atom within
    # rcut of a point (points folded into the in-plane cell)
    recip_len = [np.linalg.norm(r) for r in np.linalg.inv(cell).T]   # 1/h_i
    span_xy = np.linalg.norm(cell[0]) + np.linalg.norm(cell[1])
    span_z = np.max(np.abs(P[:, None, 2] - X[None, :, 2])) if len(P) else 0.0
    N = [int(math.ceil((rcut + span_xy) * recip_len[0])),
         int(math.ceil((rcut + span_xy) * recip_len[1])),
         int(math.ceil((rcut + span_z) * recip_len[2]))]
    for n1 in range(-N[0], N[0] + 1):
        for n2 in range(-N[1], N[1] + 1):
            for n3 in range(-N[2], N[2] + 1):
                shift = n1 * cell[0] + n2 * cell[1] + n3 * cell[2]
                d = P[:, None, :] - (X[None, :, :] + shift)
                r = np.sqrt(np.sum(d * d, -1))
                use = r < rcut
                if exclude is not None:
                    use &= r > 1e-9          # the site's own n = 0 term
                if not use.any():
                    continue
                rs = np.where(use, r, 1.0)
                term = np.where(use, q[None, :] * erfc(beta * rs) / rs, 0.0)
                phi += term.sum(1)
                dphidr = np.where(use, -q[None, :] * (erfc(beta * rs) / rs ** 2
                                  + 2 * beta / math.sqrt(math.pi) * np.exp(-(beta * rs) ** 2) / rs), 0.0)
                grad += np.sum((dphidr / rs)[..., None] * d, 1)
    # reciprocal space
    K, k2 = _kvectors(cell, kmax)
    S = (q[None, :] * np.exp(-1j * (K @ X.T))).sum(1)             # (K,)
    A = (4 * np.pi / V) * np.exp(-k2 / (4 * beta * beta)) / k2     # (K,)
    chunk = 2048
    for s in range(0, len(P), chunk):
        ph = np.exp(1j * (P[s:s + chunk] @ K.T)) * (A * S)[None, :]  # (n, K)
        phi[s:s + chunk] += ph.real.sum(1)
        grad[s:s + chunk] += -(ph.imag @ K)
    Q = q.sum()
    phi += -np.pi * Q / (beta * beta * V)
    if slab:
        Mz = np.sum(q * X[:, 2])
        phi += 4 * np.pi / V * Mz * P[:, 2]
        grad[:, 2] += 4 * np.pi / V * Mz
    if exclude is not None:
        phi += -2 * beta * q[exclude] / math.sqrt(math.pi)
    return phi, grad


def slab_fourier_potential(points, xyz, q, a1, a2, gmax):
    """Exact potential (Gaussian units) of point charges periodic in the plane
    spanned by a1, a2 and open in z, at points above all charges.

    phi(rho, z) = sum_{G != 0} (2 pi / (A |G|)) sum_j q_j exp(-|G|(z - z_j)) cos(G.(rho - rho_j))
                  - (2 pi / A) sum_j q_j (z - z_j)
    (a sheet of charge density sigma has potential -2 pi sigma |z| and its
    Fourier component G has 2 pi sigma_G exp(-|G||z|)/|G|).  Used only to
    pin the Ewald sum; truncated at |G| < gmax.
    """
    P = np.asarray(points, np.float64)
    X = np.asarray(xyz, np.float64)
    q = np.asarray(q, np.float64)
    a1 = np.asarray(a1, np.float64)[:2]; a2 = np.asarray(a2, np.float64)[:2]
    A = abs(a1[0] * a2[1] - a1[1] * a2[0])
    Bm = 2 * np.pi * np.linalg.inv(np.array([a1, a2])).T
    M1 = int(math.ceil(gmax * np.linalg.norm(a1) / (2 * np.pi))) + 1
    M2 = int(math.ceil(gmax * np.linalg.norm(a2) / (2 * np.pi))) + 1
    phi = np.zeros(len(P))
    dz = P[:, None, 2] - X[None, :, 2]
    if np.any(dz <= 0):
        raise ValueError("points must lie above all charges")
    for m1 in range(-M1, M1 + 1):
        for m2 in range(-M2, M2 + 1):
            if m1 == 0 and m2 == 0:
                continue
            G = m1 * Bm[0] + m2 * Bm[1]
            g = np.linalg.norm(G)
            if g >= gmax:
                continue
            arg = (P[:, None, :2] - X[None, :, :2]) @ G
            phi += (2 * np.pi / (A * g)) * np.sum(q[None, :] * np.exp(-g * dz) * np.cos(arg), 1)
    phi += -(2 * np.pi / A) * np.sum(q[None, :] * dz, 1)
    return phi


def coulomb_channel(points, xyz, q, cell, ewald=None):
    """V^C = k_e * phi_Ewald (volts) and its gradient at the points."""
    beta, rcut, kmax = ewald if ewald is not None else ewald_params()
    phi, g = ewald_potential(points, xyz, q, cell, beta, rcut, kmax, slab=True)
    return KE * phi, KE * g


def pairwise_reference(points, Q, R, eps, sub, alpha=1.5, rcut=17.0, ewald=None):
    """FP64 molecule-substrate reference for atoms at the points (Eq. E):
    per-atom energy E_i = direct Morse pair sum + Q_i V^C(r_i), and force
    F_i = -grad E_i.  ``sub`` needs xyz, q, R, eps, cell.
    Returns (E (N,), F (N, 3))."""
    Em, Gm = morse_pair_energy(points, R, eps, sub.xyz, sub.R, sub.eps, sub.cell, alpha, rcut)
    if np.any(sub.q != 0):
        VC, GC = coulomb_channel(points, sub.xyz, sub.q, sub.cell, ewald)
    else:
        VC = np.zeros(len(points)); GC = np.zeros((len(points), 3))
    Q = np.asarray(Q, np.float64)
    E = Em + Q * VC
    F = -(Gm + Q[:, None] * GC)
    return E, F
