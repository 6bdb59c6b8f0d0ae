"""Seeded synthetic inputs: substrates, molecules, replica poses, grid boxes.

This module only *generates data*.  It holds none of GridFF's arithmetic (no
Morse factorisation, no Ewald sum, no B-spline, no force field, no integrator):
both the CUDA library and the CPU oracle consume what it produces.  Every
function takes an explicit seed (numpy PCG64) so that a test, ``smoke()`` and
``bench.py`` see identical inputs.

The paper's own systems (PTCDA on NaCl(001), xylitol on NaCl with a Cl
vacancy; Sec. 6 and Sec. 7) are not available, so these generators build
stand-ins with the same shapes: rock-salt (001) slabs with a = 5.64 A and
+-0.7 e ions, fcc(111) metal slabs, a 10-atom C/H/O chain, a planar 38-atom
C24H8O6 core, and random flexible molecules of 10-120 atoms.

Units: Angstrom, eV, elementary charge e, fs, amu.  Morse parameters are
given per element as (R, eps) where the pair well depth is eps_i*eps_j and
the pair equilibrium distance is R_i + R_j (the mixing that the factorised
Morse form of Sec. 3 requires).  The values are synthetic, chosen in the
usual range of universal-force-field-like parameters; they are not a
published table.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# element -> (R [A], eps [sqrt(eV)], mass [amu]); synthetic values.
ELEMENTS = {
    "H": (1.45, 0.0436, 1.008),
    "C": (1.93, 0.0678, 12.011),
    "O": (1.75, 0.0510, 15.999),
    "Na": (1.49, 0.0361, 22.990),
    "Cl": (1.97, 0.0990, 35.453),
    "M": (1.65, 0.1300, 196.97),   # generic fcc metal
}

MORSE_ALPHA = 1.5      # 1/A, same for all pairs (Sec. 6)
MORSE_RCUT = 17.0      # A, hard cutoff of the substrate sums (Sec. 6)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# substrates
# ---------------------------------------------------------------------------
@dataclass
class Substrate:
    """Rigid substrate: atoms of one periodic supercell.

    ``cell`` rows are the lattice vectors A1, A2, A3 (A); A1 and A2 lie in the
    surface plane, A3 = (0, 0, Lz) is the vacuum-padded height used by the
    3D-periodic Ewald sum.  ``z_top`` is the height of the top atomic layer.
    ``tile`` is an orthogonal in-plane period (Lx, Ly) of the pristine lattice
    that a grid may cover instead of the whole supercell.
    """
    xyz: np.ndarray          # (n, 3) float64
    q: np.ndarray            # (n,) float64
    R: np.ndarray            # (n,) float64
    eps: np.ndarray          # (n,) float64
    elements: list
    cell: np.ndarray         # (3, 3) float64
    z_top: float
    tile: tuple

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def _params(elements):
    R = np.array([ELEMENTS[e][0] for e in elements], dtype=np.float64)
    eps = np.array([ELEMENTS[e][1] for e in elements], dtype=np.float64)
    return R, eps


def rocksalt_slab(a: float = 5.64, ncell: int = 4, layers: int = 2,
                  charge: float = 0.7, grid_height: float = 20.0,
                  z_gap: float = 1.0, vacuum_factor: float = 3.0,
                  cation_morse: tuple | None = None) -> Substrate:
    """NaCl(001)-like slab: ``ncell`` x ``ncell`` primitive surface cells.

    Primitive in-plane vectors a1 = (a/2)(1, 1, 0), a2 = (a/2)(1, -1, 0), one
    cation and one anion per cell and layer, layers a/2 apart, species
    alternating between layers.  The orthogonal tile 2a x 2a is a period of
    the pristine slab.  The Ewald height Lz is ``vacuum_factor`` times the
    z-extent from the bottom layer to the top of the grid box.
    ``cation_morse`` = (R, eps) replaces the cation's Morse parameters
    (default: the Na entry of ELEMENTS).
    """
    a1 = np.array([a / 2, a / 2, 0.0])
    a2 = np.array([a / 2, -a / 2, 0.0])
    xyz, q, el = [], [], []
    for l in range(layers):
        z = l * a / 2
        cat_off = np.array([a / 2, 0.0, 0.0]) if (l % 2) else np.zeros(3)
        an_off = np.zeros(3) if (l % 2) else np.array([a / 2, 0.0, 0.0])
        for m1 in range(ncell):
            for m2 in range(ncell):
                base = m1 * a1 + m2 * a2 + np.array([0.0, 0.0, z])
                xyz.append(base + cat_off); q.append(+charge); el.append("Na")
                xyz.append(base + an_off); q.append(-charge); el.append("Cl")
    xyz = np.array(xyz)
    z_top = (layers - 1) * a / 2
    Lz = vacuum_factor * (z_top + z_gap + grid_height)
    cell = np.array([ncell * a1, ncell * a2, [0.0, 0.0, Lz]])
    R, eps = _params(el)
    if cation_morse is not None:
        na = np.array(el) == "Na"
        R[na], eps[na] = cation_morse
    return Substrate(xyz, np.array(q), R, eps, el, cell, z_top, (2 * a, 2 * a))


# Cation Morse parameters (R [A], eps [sqrt(eV)]) of the minima-hopping
# stand-in substrate, synthetic: a hard cation whose repulsive wall keeps
# molecule atoms (charges up to +-0.3 e) at least 2 A above the top ion
# plane over cations, anions and the anion vacancy alike, where the default
# Na entry lets a negative atom sink into the vacancy below the grid floor.
# With it the minima over the vacancy (O -0.3 e: 2.4 A, -1.44 eV) stay the
# deepest, over cations 3.4-4.0 A and anions 3.2-3.5 A (pairwise Morse +
# Ewald energies of single atoms, 4 x 4 x 3 slab with one Cl vacancy).
HARD_CATION = (2.5, 0.3)


def hopping_substrate() -> Substrate:
    """Stand-in of the minima-hopping substrate (Sec. 7: NaCl(001) with a Cl
    vacancy): the 4 x 4 primitive-cell, 3-layer rock-salt slab with hard
    cations (HARD_CATION) and the top-layer anion nearest the supercell
    centre removed."""
    return with_top_vacancy(rocksalt_slab(a=5.64, ncell=4, layers=3, charge=0.7, cation_morse=HARD_CATION))


def with_top_vacancy(sub: Substrate, element: str = "Cl") -> Substrate:
    """The slab with one ``element`` atom of the top layer removed (the one
    nearest the centre of the supercell).  The defect repeats with the
    supercell, so the grid tile becomes the orthogonal period of the
    supercell lattice, A1 + A2 and A1 - A2 for the rock-salt supercell."""
    top = np.where((np.abs(sub.xyz[:, 2] - sub.z_top) < 1e-6) &
                   (np.array(sub.elements) == element))[0]
    centre = 0.5 * (sub.cell[0] + sub.cell[1])
    k = top[np.argmin(np.linalg.norm(sub.xyz[top, :2] - centre[:2], axis=1))]
    keep = np.ones(sub.n, bool)
    keep[k] = False
    ex = sub.cell[0] + sub.cell[1]
    ey = sub.cell[0] - sub.cell[1]
    return Substrate(sub.xyz[keep], sub.q[keep], sub.R[keep], sub.eps[keep],
                     [e for e, kk in zip(sub.elements, keep) if kk], sub.cell, sub.z_top,
                     (float(abs(ex[0])), float(abs(ey[1]))))


def fcc111_slab(a: float = 4.08, ncell: int = 12, layers: int = 4,
                grid_height: float = 20.0, z_gap: float = 1.0,
                vacuum_factor: float = 3.0) -> Substrate:
    """Neutral fcc(111) metal-like slab, ABC stacking, ``ncell`` x ``ncell``.

    Nearest-neighbour distance d = a/sqrt(2), in-plane vectors d(1, 0) and
    d(1/2, sqrt(3)/2), layer spacing a/sqrt(3).  The orthogonal tile
    4d x 2*sqrt(3)*d is a period of the pristine slab.
    """
    d = a / math.sqrt(2.0)
    a1 = np.array([d, 0.0, 0.0])
    a2 = np.array([d / 2, d * math.sqrt(3) / 2, 0.0])
    dz = a / math.sqrt(3.0)
    shifts = [np.zeros(3), (a1 + a2) / 3, 2 * (a1 + a2) / 3]
    xyz, el = [], []
    for l in range(layers):
        s = shifts[l % 3] + np.array([0.0, 0.0, l * dz])
        for m1 in range(ncell):
            for m2 in range(ncell):
                xyz.append(m1 * a1 + m2 * a2 + s); el.append("M")
    xyz = np.array(xyz)
    z_top = (layers - 1) * dz
    Lz = vacuum_factor * (z_top + z_gap + grid_height)
    cell = np.array([ncell * a1, ncell * a2, [0.0, 0.0, Lz]])
    R, eps = _params(el)
    return Substrate(xyz, np.zeros(len(el)), R, eps, el, cell, z_top,
                     (4 * d, 2 * math.sqrt(3) * d))


@dataclass
class GridBox:
    """Orthogonal box covered by a grid: origin and lengths (A)."""
    origin: tuple
    length: tuple
    spacing: float


def grid_box_for(sub: Substrate, spacing: float, height: float = 20.0,
                 z_gap: float = 1.0) -> GridBox:
    """Grid box over the substrate's orthogonal tile, starting ``z_gap`` A
    above the top layer and ``height`` A tall."""
    return GridBox((0.0, 0.0, sub.z_top + z_gap),
                   (sub.tile[0], sub.tile[1], height), spacing)


# ---------------------------------------------------------------------------
# molecules
# ---------------------------------------------------------------------------
@dataclass
class Molecule:
    """One molecule template: geometry, per-atom parameters and topology."""
    elements: list
    xyz: np.ndarray              # (n, 3) reference geometry
    q: np.ndarray                # (n,) charges, sum 0
    R: np.ndarray
    eps: np.ndarray
    mass: np.ndarray
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    bond_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    bond_r0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    angles: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.int32))
    angle_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    angle_cos0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    torsions: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.int32))
    torsion_V: np.ndarray = field(default_factory=lambda: np.zeros(0))
    torsion_n: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    torsion_cos_nphi0: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n(self) -> int:
        return len(self.elements)


def _finish(elements, xyz, q, bonds, geom_from_xyz=True,
            k_bond=15.0, k_angle=3.0, V_tors=0.05, n_tors=3) -> Molecule:
    R, eps = _params(elements)
    mass = np.array([ELEMENTS[e][2] for e in elements])
    bonds = np.array(sorted(tuple(sorted(b)) for b in bonds), dtype=np.int32).reshape(-1, 2)
    n = len(elements)
    nbr = [[] for _ in range(n)]
    for i, j in bonds:
        nbr[i].append(int(j)); nbr[j].append(int(i))
    angles = []
    for j in range(n):
        for ii in range(len(nbr[j])):
            for kk in range(ii + 1, len(nbr[j])):
                angles.append((nbr[j][ii], j, nbr[j][kk]))
    torsions = []
    for j, k in bonds:
        for i in nbr[j]:
            if i == k:
                continue
            for l in nbr[k]:
                if l == j or l == i:
                    continue
                torsions.append((i, j, k, l))
    angles = np.array(angles, dtype=np.int32).reshape(-1, 3)
    torsions = np.array(torsions, dtype=np.int32).reshape(-1, 4)
    # reference geometry values -> equilibrium parameters (generated data)
    r0 = np.linalg.norm(xyz[bonds[:, 0]] - xyz[bonds[:, 1]], axis=1) if len(bonds) else np.zeros(0)
    if len(angles):
        u = xyz[angles[:, 0]] - xyz[angles[:, 1]]
        w = xyz[angles[:, 2]] - xyz[angles[:, 1]]
        c0 = np.sum(u * w, 1) / np.linalg.norm(u, axis=1) / np.linalg.norm(w, axis=1)
    else:
        c0 = np.zeros(0)
    return Molecule(list(elements), np.asarray(xyz, np.float64), np.asarray(q, np.float64),
                    R, eps, mass, bonds, np.full(len(bonds), k_bond), r0,
                    angles, np.full(len(angles), k_angle), c0,
                    torsions, np.full(len(torsions), V_tors),
                    np.full(len(torsions), n_tors, np.int32),
                    np.full(len(torsions), -1.0))   # cos(n*phi0) with n*phi0 = 3*180 deg


def _zero_sum(q):
    q = np.asarray(q, np.float64)
    return q - q.mean()


def chain_molecule(seed: int = 1001) -> Molecule:
    """10-atom C/H/O chain: heavy backbone C-C-O-C-O (two rotatable inner
    bonds) with five hydrogens; random charges U(-0.3, 0.3) shifted to sum 0."""
    g = rng(seed)
    heavy = ["C", "C", "O", "C", "O"]
    bl = {"CC": 1.52, "CO": 1.43, "OC": 1.43, "CH": 1.09, "OH": 0.97}
    # zig-zag backbone in the xz plane with tetrahedral-ish angles
    theta = math.radians(111.0)
    pos = [np.zeros(3)]
    direction = np.array([1.0, 0.0, 0.0])
    for k in range(1, len(heavy)):
        L = bl[heavy[k - 1] + heavy[k]]
        if k > 1:
            sgn = 1.0 if k % 2 else -1.0
            ang = sgn * (math.pi - theta)
            c, s = math.cos(ang), math.sin(ang)
            direction = np.array([c * direction[0] - s * direction[2], 0.0,
                                  s * direction[0] + c * direction[2]])
        pos.append(pos[-1] + L * direction)
    elements = list(heavy)
    bonds = [(k, k + 1) for k in range(len(heavy) - 1)]
    # hydrogens: 2 on C0, 1 on C1, 1 on C3, 1 on terminal O4
    h_on = [0, 0, 1, 3, 4]
    for cnt, host in enumerate(h_on):
        hostpos = pos[host]
        # direction away from bonded heavy neighbours, plus a y-offset
        away = np.zeros(3)
        for (i, j) in bonds:
            if i == host:
                away += hostpos - pos[j]
            if j == host:
                away += hostpos - pos[i]
        away /= max(np.linalg.norm(away), 1e-9)
        side = np.array([0.0, 1.0 if cnt % 2 == 0 else -1.0, 0.0])
        d = away + 0.9 * side
        d /= np.linalg.norm(d)
        L = bl["OH"] if heavy[host] == "O" else bl["CH"]
        pos.append(hostpos + L * d)
        elements.append("H")
        bonds.append((host, len(elements) - 1))
    xyz = np.array(pos)
    xyz -= xyz.mean(0)
    q = _zero_sum(g.uniform(-0.3, 0.3, len(elements)))
    return _finish(elements, xyz, q, bonds)


def _principal_frame(xyz, mass):
    com = (mass[:, None] * xyz).sum(0) / mass.sum()
    b = xyz - com
    I = np.zeros((3, 3))
    for m, r in zip(mass, b):
        I += m * (np.dot(r, r) * np.eye(3) - np.outer(r, r))
    w, V = np.linalg.eigh(I)
    if np.linalg.det(V) < 0:
        V[:, 2] *= -1
    return b @ V, w


def c24h8o6_core() -> Molecule:
    """Planar 38-atom C24H8O6 core, generated on a honeycomb lattice.

    Six fused hexagons (C-C 1.40 A): a four-ring rhombus with one extra ring
    fused at each end, which gives 24 carbons with 14 edge sites.  The six
    edge carbons farthest from the centre along the long axis carry C=O
    oxygens (1.21 A), the other eight carry hydrogens (1.08 A).  Charges:
    O -0.3 e, H +0.15 e, each carbon bonded to an O +0.1 e (total 0).
    Returned in its principal-axes frame centred at the centre of mass (the
    rigid-body convention of the library).
    """
    bond = 1.40
    T1 = np.array([bond * math.sqrt(3), 0.0])
    T2 = np.array([bond * math.sqrt(3) / 2, 1.5 * bond])
    rings = [(0, 0), (1, 0), (0, 1), (1, 1), (-1, 0), (2, 1)]
    verts = []
    for (i, j) in rings:
        c = i * T1 + j * T2
        for k in range(6):
            ang = math.radians(30 + 60 * k)
            v = c + bond * np.array([math.cos(ang), math.sin(ang)])
            if not any(np.linalg.norm(v - w) < 1e-6 for w in verts):
                verts.append(v)
    C = np.array(verts)
    C -= C.mean(0)
    if len(C) != 24:
        raise RuntimeError("honeycomb patch does not have 24 sites")
    d = np.linalg.norm(C[:, None] - C[None], axis=2)
    cc = [(i, j) for i in range(24) for j in range(i + 1, 24) if abs(d[i, j] - bond) < 1e-3]
    deg = np.zeros(24, int)
    for i, j in cc:
        deg[i] += 1; deg[j] += 1
    edge = [i for i in range(24) if deg[i] == 2]
    if len(edge) != 14:
        raise RuntimeError("honeycomb patch does not have 14 edge sites")
    # long axis of the carbon patch
    w, V = np.linalg.eigh(C.T @ C)
    axis = V[:, -1]
    edge_sorted = sorted(edge, key=lambda i: (-abs(float(C[i] @ axis)), i))
    o_hosts, h_hosts = edge_sorted[:6], edge_sorted[6:]
    xyz = [np.array([c[0], c[1], 0.0]) for c in C]
    elements = ["C"] * 24
    bonds = list(cc)
    q = [0.0] * 24
    for hosts, el, L, qq in ((o_hosts, "O", 1.21, -0.3), (h_hosts, "H", 1.08, 0.15)):
        for h in hosts:
            nb = [j for (i, j) in cc if i == h] + [i for (i, j) in cc if j == h]
            away = 2 * C[h] - C[nb[0]] - C[nb[1]]
            away /= np.linalg.norm(away)
            xyz.append(np.array([C[h, 0] + L * away[0], C[h, 1] + L * away[1], 0.0]))
            elements.append(el)
            bonds.append((h, len(elements) - 1))
            q.append(qq)
            if el == "O":
                q[h] = 0.1
    xyz = np.array(xyz)
    mass = np.array([ELEMENTS[e][2] for e in elements])
    b, _ = _principal_frame(xyz, mass)
    return _finish(elements, b, np.array(q), bonds)


def random_flexible_molecule(n_atoms: int, n_torsions: int, seed: int) -> Molecule:
    """Random tree-shaped C/H/O molecule with ``n_atoms`` atoms.

    Heavy atoms form a chain with branches; about a third of the atoms are
    hydrogens.  ``n_torsions`` caps the rotatable inner bonds that carry a
    torsion term.  Charges U(-0.3, 0.3), shifted to sum 0.
    """
    g = rng(seed)
    n_atoms = int(max(n_atoms, 4))
    n_heavy = max(2, int(round(n_atoms * 0.62)))
    n_h = n_atoms - n_heavy
    elements = list(g.choice(["C", "C", "C", "O"], size=n_heavy))
    parent = [-1] + [int(g.integers(max(0, k - 2), k)) for k in range(1, n_heavy)]
    pos = np.zeros((n_atoms, 3))
    nbr = [[] for _ in range(n_atoms)]
    cos_max = math.cos(math.radians(150.0))    # bond angles at most 150 degrees

    def place(a, others, length, clearance):
        # up to 200 random directions from atom a: the first that keeps
        # `clearance` from every other atom and opens no angle wider than
        # 150 degrees with a's bonds (near-linear angles leave the torsions
        # about the bond ill-defined), else the best by (angle kept, distance
        # to the nearest atom)
        bonded = [(pos[j] - pos[a]) / np.linalg.norm(pos[j] - pos[a]) for j in nbr[a]]
        best, best_key = None, None
        for _ in range(200):
            d = g.normal(size=3)
            d /= np.linalg.norm(d)
            cand = pos[a] + length * d
            near = np.linalg.norm(others - cand, axis=1).min() if len(others) else np.inf
            angle_ok = all(float(d @ u) > cos_max for u in bonded)
            if near > clearance and angle_ok:
                return cand
            key = (angle_ok, near)
            if best_key is None or key > best_key:
                best, best_key = cand, key
        return best

    for k in range(1, n_heavy):
        pos[k] = place(parent[k], np.delete(pos[:k], parent[k], axis=0), 1.50, 2.2)
        nbr[parent[k]].append(k); nbr[k].append(parent[k])
    bonds = [(parent[k], k) for k in range(1, n_heavy)]
    for h in range(n_h):
        host = int(g.integers(0, n_heavy))
        pos[n_heavy + h] = place(host, np.delete(pos[:n_heavy + h], host, axis=0), 1.09, 1.6)
        nbr[host].append(n_heavy + h); nbr[n_heavy + h].append(host)
        elements.append("H")
        bonds.append((host, n_heavy + h))
    xyz = pos.copy()
    xyz -= xyz.mean(0)
    q = _zero_sum(g.uniform(-0.3, 0.3, n_atoms))
    mol = _finish(elements, xyz, q, bonds)
    if len(mol.torsions) > 0:
        # keep torsion terms only around the first ``n_torsions`` inner bonds
        inner = []
        for t in mol.torsions:
            key = (int(min(t[1], t[2])), int(max(t[1], t[2])))
            if key not in inner:
                inner.append(key)
        keep_bonds = set(inner[:n_torsions])
        keep = [k for k, t in enumerate(mol.torsions)
                if (int(min(t[1], t[2])), int(max(t[1], t[2]))) in keep_bonds]
        mol.torsions = mol.torsions[keep]
        mol.torsion_V = mol.torsion_V[keep]
        mol.torsion_n = mol.torsion_n[keep]
        mol.torsion_cos_nphi0 = mol.torsion_cos_nphi0[keep]
    return mol


def rigid_molecule(n_atoms: int, seed: int) -> Molecule:
    """A generated molecule of ``n_atoms`` atoms (random tree geometry) used
    as a rigid body: coordinates in its principal-axes frame centred at the
    centre of mass, no intramolecular terms."""
    m = random_flexible_molecule(n_atoms, 0, seed)
    body, _ = _principal_frame(m.xyz, m.mass)
    return Molecule(m.elements, body, m.q, m.R, m.eps, m.mass)


def uneven_sizes(n_rep: int, seed: int, lo: int = 10, hi: int = 120) -> np.ndarray:
    """Log-uniform molecule sizes in [lo, hi]."""
    g = rng(seed)
    return np.clip(np.round(np.exp(g.uniform(math.log(lo), math.log(hi), n_rep))), lo, hi).astype(int)


def uneven_batch(n_rep: int, n_templates: int, seed: int, lo: int = 10, hi: int = 120):
    """A batch of flexible replicas of uneven size: ``n_templates`` random
    molecules with log-uniform sizes in [lo, hi] and 0-12 torsion bonds
    (uniform), and the template of every replica (uniform).  Returns
    (templates, template_of)."""
    g = rng(seed)
    sizes = uneven_sizes(n_templates, seed + 1, lo, hi)
    tors = g.integers(0, 13, n_templates)
    mols = [random_flexible_molecule(int(n), int(t), seed + 100 + k) for k, (n, t) in enumerate(zip(sizes, tors))]
    return mols, g.integers(0, n_templates, n_rep).astype(np.int32)


# ---------------------------------------------------------------------------
# replica poses
# ---------------------------------------------------------------------------
def random_quaternions(n: int, g: np.random.Generator) -> np.ndarray:
    """Uniform random unit quaternions (w, x, y, z), Shoemake's method."""
    u1, u2, u3 = g.random(n), g.random(n), g.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    return np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                     b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], 1)[:, [1, 0, 2, 3]]


def quat_to_matrix(q: np.ndarray) -> np.ndarray:
    """Rotation matrices of unit quaternions (w, x, y, z); generic geometry
    used only to place generated molecules."""
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def rigid_poses(mol: Molecule, sub: Substrate, n_rep: int, seed: int,
                h_lo: float = 3.0, h_hi: float = 5.0, min_clear: float = 2.0):
    """Random rigid poses: COM xy uniform over the tile, COM height
    U(h_lo, h_hi) above the top layer, uniform random orientation; a pose is
    lifted until its lowest atom is ``min_clear`` A above the top layer.
    Returns (com (n,3), quat (n,4)) in float64."""
    g = rng(seed)
    quat = random_quaternions(n_rep, g)
    Rm = quat_to_matrix(quat)
    body = mol.xyz
    lowest = np.einsum("nij,aj->nai", Rm, body)[:, :, 2].min(1)
    com = np.stack([g.uniform(0, sub.tile[0], n_rep), g.uniform(0, sub.tile[1], n_rep),
                    sub.z_top + g.uniform(h_lo, h_hi, n_rep)], 1)
    need = sub.z_top + min_clear - (com[:, 2] + lowest)
    com[:, 2] += np.maximum(need, 0.0)
    return com, quat


def flexible_positions(mol: Molecule, sub: Substrate, n_rep: int, seed: int,
                       h_lo: float = 3.0, h_hi: float = 5.0, min_clear: float = 2.0):
    """Cartesian start positions (n_rep, n, 3) of a flexible molecule placed
    like ``rigid_poses`` (geometry centred on its mean position)."""
    com, quat = rigid_poses(_centred(mol), sub, n_rep, seed, h_lo, h_hi, min_clear)
    Rm = quat_to_matrix(quat)
    return np.einsum("nij,aj->nai", Rm, _centred(mol).xyz) + com[:, None, :]


def _centred(mol: Molecule) -> Molecule:
    import copy
    m = copy.copy(mol)
    m.xyz = mol.xyz - mol.xyz.mean(0)
    return m


def uniform_points(n: int, box: GridBox, seed: int, zband=(2.0, 8.0)) -> np.ndarray:
    """Points uniform over the tile in x, y and over [z0+zband[0], z0+zband[1]]
    in z (no locality; the interpolation roofline workload)."""
    g = rng(seed)
    x0, y0, z0 = box.origin
    return np.stack([x0 + g.uniform(0, box.length[0], n), y0 + g.uniform(0, box.length[1], n),
                     z0 + g.uniform(zband[0], zband[1], n)], 1)


def random_coefficients(shape, n_channels: int, seed: int, scale=(1.0, 0.3, 0.1)) -> np.ndarray:
    """Random coefficient grid (n_channels, nx, ny, nz), float64, of the given
    per-channel magnitudes; used where an interpolation test wants a field
    that does not come from a substrate."""
    g = rng(seed)
    out = np.empty((n_channels,) + tuple(shape))
    for c in range(n_channels):
        out[c] = scale[c % len(scale)] * g.standard_normal(shape)
    return out


def atom_params(mol: Molecule):
    """(q, R, eps, mass) float64 arrays of a molecule template."""
    return mol.q.copy(), mol.R.copy(), mol.eps.copy(), mol.mass.copy()


# ---------------------------------------------------------------------------
# learned pose proposal: initial weights and training inputs
# ---------------------------------------------------------------------------
def mlp_weights(sizes, seed: int):
    """He-uniform initial weights W_l [out][in] and zero biases of an MLP with
    layer widths ``sizes`` (float64)."""
    g = rng(seed)
    Ws, bs = [], []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = math.sqrt(6.0 / n_in)
        Ws.append(g.uniform(-lim, lim, (n_out, n_in)))
        bs.append(np.zeros(n_out))
    return Ws, bs


def noise(n: int, dim: int, seed: int) -> np.ndarray:
    """Standard-normal noise inputs (n, dim), float32."""
    return rng(seed).standard_normal((n, dim)).astype(np.float32)
