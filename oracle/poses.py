"""Flexible-molecule poses: rotatable bonds, the pose builder and its inverse.

Oracle (test infrastructure).  The learned pose proposal (the network of
the sampling loop, Sec. 7 starting configurations) outputs a centre of
mass, an orientation quaternion and up to 12 torsion angles.  For a flexible
molecule those torsions act on its rotatable bonds: this module states
which bonds these are, how a pose (com, q, theta) becomes atom positions
(torsion rotations down the bond tree, then rotate, then translate) and how
a relaxed structure gives the pose that rebuilds it (dihedrals, then the
best rotation by Horn's quaternion method).  Plain Python loops over bonds
and atoms, FP64.

Definitions (the paper gives none; these are the readings the library
follows):

* root: the lowest-index atom bonded to exactly one other atom (atom 0 if
  there is none); breadth-first search from it over the bond graph,
  neighbours in increasing index order, gives each atom its parent and
  depth.
* candidate bonds: the central bonds (b, c) of the torsion terms, distinct,
  in the order of their first torsion term.  A candidate is rotatable when
  it is a tree edge of the search (one end is the other's parent), removing
  it disconnects the graph (no ring), the end nearer the root (b) has a
  parent and the far end (c) has a neighbour other than b.  The first 12
  rotatable candidates are kept.
* reference quadruple of bond (b, c): (parent(b), b, c, d), d the
  lowest-index neighbour of c other than b.  theta is its dihedral.
* moving side: the atoms reached from c without crossing (b, c).
* build order: by depth of b, then by kept order.  Every rotation moves
  only atoms below its c, so a later rotation never changes an earlier
  dihedral and the builder sets every dihedral exactly.
"""
from __future__ import annotations

import math

import numpy as np

from .dynamics import quat_matrix

MAX_ROT = 12


def dihedral(xa, xb, xc, xd) -> float:
    """Signed dihedral angle of a-b-c-d (radians, (-pi, pi]): the angle
    from the plane (a, b, c) to the plane (b, c, d), positive for a right-
    handed turn about b -> c."""
    b1 = np.asarray(xb, float) - np.asarray(xa, float)
    b2 = np.asarray(xc, float) - np.asarray(xb, float)
    b3 = np.asarray(xd, float) - np.asarray(xc, float)
    n1 = np.cross(b1, b2)
    n2 = np.cross(b2, b3)
    return math.atan2(float(np.linalg.norm(b2) * np.dot(b1, n2)), float(np.dot(n1, n2)))


def rotate_about(x, origin, axis, angle):
    """Rodrigues rotation of points x (m, 3) about the line through origin
    along the unit vector axis, by angle (right-hand rule)."""
    k = np.asarray(axis, float)
    p = np.asarray(x, float) - origin
    c, s = math.cos(angle), math.sin(angle)
    return origin + p * c + np.cross(k, p) * s + np.outer(p @ k, k) * (1.0 - c)


def rotors(n_atoms, bonds, torsions):
    """Rotatable bonds of a template: list of dicts with the reference
    quadruple 'quad' (a, b, c, d), the moving atoms 'move' (sorted list) and
    'depth' (of b), in build order."""
    nbr = [[] for _ in range(n_atoms)]
    for i, j in bonds:
        nbr[int(i)].append(int(j))
        nbr[int(j)].append(int(i))
    for lst in nbr:
        lst.sort()
    root = 0
    for i in range(n_atoms):
        if len(nbr[i]) == 1:
            root = i
            break
    parent = [-1] * n_atoms
    depth = [-1] * n_atoms
    depth[root] = 0
    queue = [root]
    for u in queue:
        for v in nbr[u]:
            if depth[v] < 0:
                depth[v] = depth[u] + 1
                parent[v] = u
                queue.append(v)
    seen = set()
    kept = []
    for t in torsions:
        j, k = int(t[1]), int(t[2])
        key = (min(j, k), max(j, k))
        if key in seen:
            continue
        seen.add(key)
        if parent[k] == j:
            b, c = j, k
        elif parent[j] == k:
            b, c = k, j
        else:
            continue                      # not a tree edge: in a ring
        if parent[b] < 0:
            continue
        others = [v for v in nbr[c] if v != b]
        if not others:
            continue
        # atoms reached from c without the bond (b, c)
        move = {c}
        stack = [c]
        ring = False
        while stack:
            u = stack.pop()
            for v in nbr[u]:
                if u == c and v == b:
                    continue
                if v == b:
                    ring = True
                    continue
                if v not in move:
                    move.add(v)
                    stack.append(v)
        if ring:
            continue
        kept.append({"quad": (parent[b], b, c, others[0]), "move": sorted(move), "depth": depth[b]})
        if len(kept) == MAX_ROT:
            break
    order = sorted(range(len(kept)), key=lambda i: (kept[i]["depth"], i))
    return [kept[i] for i in order]


def centre_of_mass(x, mass):
    m = np.asarray(mass, float)
    return (np.asarray(x, float) * m[:, None]).sum(0) / m.sum()


def build(xyz, mass, rot, com, quat, theta):
    """Atom positions (n, 3) of the pose (com, quat, theta): starting from
    the reference geometry xyz, set the dihedral of rotor k to theta[k] by
    rotating its moving side about its bond (build order), then rotate the
    molecule about its centre of mass by the unit quaternion quat (w, x, y,
    z; a zero quaternion means no rotation) and put that centre at com."""
    x = np.array(xyz, dtype=float)
    for k, r in enumerate(rot):
        a, b, c, d = r["quad"]
        delta = theta[k] - dihedral(x[a], x[b], x[c], x[d])
        axis = (x[c] - x[b]) / np.linalg.norm(x[c] - x[b])
        idx = np.array(r["move"])
        x[idx] = rotate_about(x[idx], x[b].copy(), axis, delta)
    q = np.asarray(quat, float)
    nq = np.linalg.norm(q)
    q = q / nq if nq > 0 else np.array([1.0, 0.0, 0.0, 0.0])
    x = x - centre_of_mass(x, mass)
    return x @ quat_matrix(q).T + np.asarray(com, float)


def horn_quaternion(z, y, mass):
    """Unit quaternion q (w >= 0) of the rotation R minimising
    sum_i m_i |R z_i - y_i|^2 for centred point sets z, y (Horn 1987: the
    eigenvector of the largest eigenvalue of the 4x4 matrix N)."""
    S = np.einsum("i,ia,ib->ab", np.asarray(mass, float), z, y)
    sxx, sxy, sxz = S[0]
    syx, syy, syz = S[1]
    szx, szy, szz = S[2]
    N = np.array([[sxx + syy + szz, syz - szy, szx - sxz, sxy - syx],
                  [syz - szy, sxx - syy - szz, sxy + syx, szx + sxz],
                  [szx - sxz, sxy + syx, -sxx + syy - szz, syz + szy],
                  [sxy - syx, szx + sxz, syz + szy, -sxx - syy + szz]])
    w, v = np.linalg.eigh(N)
    q = v[:, -1]
    return q if q[0] >= 0 else -q


def targets(xyz, mass, rot, y):
    """Pose (com, quat, theta) of the positions y (n, 3): theta = the
    rotors' dihedrals in y, com = the centre of mass of y, quat = the
    rotation that best maps the built geometry with those torsions (centred)
    onto y (centred), mass-weighted."""
    y = np.asarray(y, float)
    theta = np.array([dihedral(*(y[i] for i in r["quad"])) for r in rot])
    z = build(xyz, mass, rot, np.zeros(3), np.array([1.0, 0.0, 0.0, 0.0]), theta)
    com = centre_of_mass(y, mass)
    return com, horn_quaternion(z, y - com, mass), theta
