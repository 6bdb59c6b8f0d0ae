"""Intramolecular force field: reduced UFF-like form (FP64, PyTorch CPU).

Oracle (test infrastructure).  The paper models intramolecular interactions
with UFF (Sec. 6, Sec. 8) without stating the terms; the reading used here
(and by the library) is

  bond      k_b (r - r0)^2
  angle     k_t (cos(theta) - cos(theta0))^2
  torsion   V/2 [1 - cos(n phi0) cos(n phi)]
  nonbonded Morse with the molecule-substrate mixing of Eq. E_Morse,
            eps_i eps_j [e^{-2a(r - R_i - R_j)} - 2 e^{-a(r - R_i - R_j)}],
            plus k_e q_i q_j / r, on every pair more than two bonds apart;
            no cutoff, no 1-4 scaling.

Forces are the definition F = -dE/dx, obtained with torch.autograd.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import torch

KE = 14.399645


def excluded_pairs(n: int, bonds) -> np.ndarray:
    """Boolean (n, n): True where atoms are at most two bonds apart (or i=j),
    by breadth-first search on the bond graph."""
    adj = [[] for _ in range(n)]
    for i, j in np.asarray(bonds).reshape(-1, 2):
        adj[int(i)].append(int(j)); adj[int(j)].append(int(i))
    ex = np.zeros((n, n), bool)
    for s in range(n):
        dist = {s: 0}
        dq = deque([s])
        while dq:
            u = dq.popleft()
            if dist[u] == 2:
                continue
            for w in adj[u]:
                if w not in dist:
                    dist[w] = dist[u] + 1
                    dq.append(w)
        for w in dist:
            ex[s, w] = True
    return ex


def dihedral(x, i, j, k, l):
    """Dihedral angle of atoms (i, j, k, l); x: (..., n, 3) tensor."""
    b1 = x[..., j, :] - x[..., i, :]
    b2 = x[..., k, :] - x[..., j, :]
    b3 = x[..., l, :] - x[..., k, :]
    n1 = torch.cross(b1, b2, dim=-1)
    n2 = torch.cross(b2, b3, dim=-1)
    m1 = torch.cross(n1, b2 / torch.linalg.norm(b2, dim=-1, keepdim=True), dim=-1)
    return torch.atan2((m1 * n2).sum(-1), (n1 * n2).sum(-1))


def energy(x, mol, alpha=1.5, terms=("bond", "angle", "torsion", "nonbonded")):
    """Intramolecular energy per replica; x: (R, n, 3) float64 tensor."""
    E = torch.zeros(x.shape[0], dtype=x.dtype)
    if "bond" in terms:
        for (i, j), k, r0 in zip(mol.bonds, mol.bond_k, mol.bond_r0):
            r = torch.linalg.norm(x[:, i] - x[:, j], dim=-1)
            E = E + float(k) * (r - float(r0)) ** 2
    if "angle" in terms:
        for (i, j, l), k, c0 in zip(mol.angles, mol.angle_k, mol.angle_cos0):
            u = x[:, i] - x[:, j]
            w = x[:, l] - x[:, j]
            c = (u * w).sum(-1) / torch.linalg.norm(u, dim=-1) / torch.linalg.norm(w, dim=-1)
            E = E + float(k) * (c - float(c0)) ** 2
    if "torsion" in terms:
        for (i, j, k, l), V, n, cn0 in zip(mol.torsions, mol.torsion_V, mol.torsion_n,
                                           mol.torsion_cos_nphi0):
            phi = dihedral(x, i, j, k, l)
            E = E + 0.5 * float(V) * (1 - float(cn0) * torch.cos(int(n) * phi))
    if "nonbonded" in terms:
        ex = excluded_pairs(mol.n, mol.bonds)
        for i in range(mol.n):
            for j in range(i + 1, mol.n):
                if ex[i, j]:
                    continue
                r = torch.linalg.norm(x[:, i] - x[:, j], dim=-1)
                s = r - float(mol.R[i] + mol.R[j])
                ee = float(mol.eps[i] * mol.eps[j])
                E = E + ee * (torch.exp(-2 * alpha * s) - 2 * torch.exp(-alpha * s))
                E = E + KE * float(mol.q[i] * mol.q[j]) / r
    return E


def energy_forces(x, mol, alpha=1.5, terms=("bond", "angle", "torsion", "nonbonded")):
    """(E (R,), F (R, n, 3)) as float64 numpy arrays; F = -dE/dx."""
    xt = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    E = energy(xt, mol, alpha, terms)
    (g,) = torch.autograd.grad(E.sum(), xt)
    return E.detach().numpy(), -g.numpy()
