"""Random starting poses and the RMSD uniqueness filter of relaxed minima.

Oracle (test infrastructure).  Sec. 7 of the paper starts molecules from
random placements over the surface and counts two relaxed structures as the
same minimum when their RMSD is below a threshold (0.1 A), which covers the
conformation, the adsorption site and the orientation.  This module restates
both plainly: per-atom positions, per-pair RMSD, a quadratic scan.

The random draws are those of the library's counter-based generator
(SplitMix64 of the seed and the counter 64 r + j, see ``mlp.splitmix64``);
the orientation is uniform on SO(3) by Shoemake's subgroup algorithm.
"""
from __future__ import annotations

import numpy as np

from .dynamics import quat_matrix
from .mlp import splitmix64


def uniform(seed: int, r: int, j: int) -> float:
    """Uniform [0, 1) draw j of row r (24 bits)."""
    return (splitmix64(seed ^ splitmix64(64 * r + j)) >> 40) / 2.0 ** 24


def random_poses(body, n_rep, seed, origin_xy, tile_xy, z_lo, z_hi, z_floor):
    """Poses (n_rep, 7): centre of mass uniform over the tile and [z_lo, z_hi),
    orientation (w, x, y, z) uniform, raised until the lowest atom of the body
    coordinates ``body`` (n, 3) is at z_floor."""
    out = np.zeros((n_rep, 7))
    for r in range(n_rep):
        u = [uniform(seed, r, j) for j in range(6)]
        a, b = np.sqrt(1 - u[0]), np.sqrt(u[0])
        q = np.array([b * np.cos(2 * np.pi * u[2]), a * np.sin(2 * np.pi * u[1]),
                      a * np.cos(2 * np.pi * u[1]), b * np.sin(2 * np.pi * u[2])])
        c = np.array([origin_xy[0] + u[3] * tile_xy[0], origin_xy[1] + u[4] * tile_xy[1],
                      z_lo + u[5] * (z_hi - z_lo)])
        lowest = (body @ quat_matrix(q).T)[:, 2].min()
        c[2] = max(c[2], z_floor - lowest)
        out[r, :3], out[r, 3:] = c, q
    return out


def positions(body, pose):
    """Atom positions r_i = R(q) b_i + c of one rigid pose."""
    q = np.asarray(pose[3:7], np.float64)
    return body @ quat_matrix(q / np.linalg.norm(q)).T + np.asarray(pose[:3], np.float64)


def rmsd(body, pa, pb, tile_xy):
    """RMSD of two rigid poses; the centres of mass by the minimum image in x, y."""
    dc = np.asarray(pa[:3], np.float64) - np.asarray(pb[:3], np.float64)
    for a in range(2):
        dc[a] -= tile_xy[a] * np.round(dc[a] / tile_xy[a])
    pb = np.array(pb, np.float64)
    pb[:3] = np.asarray(pa[:3], np.float64) - dc
    d = positions(body, pa) - positions(body, pb)
    return float(np.sqrt(np.mean(np.sum(d * d, 1))))


def dup_of(body, poses, tile_xy, threshold):
    """For each pose, the first earlier pose within ``threshold`` RMSD, else -1."""
    out = []
    for i in range(len(poses)):
        found = -1
        for j in range(i):
            if rmsd(body, poses[i], poses[j], tile_xy) < threshold:
                found = j
                break
        out.append(found)
    return np.array(out, np.int32)


def rmsd_xyz(a, b, tile_xy):
    """RMSD of two structures (n, 3) of one molecule after shifting b by
    whole tile periods in x, y toward a's mean position; no alignment."""
    a = np.asarray(a, np.float64); b = np.array(b, np.float64)
    d = a[:, :2].mean(0) - b[:, :2].mean(0)
    for k in range(2):
        b[:, k] += tile_xy[k] * np.round(d[k] / tile_xy[k])
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, 1))))


def dup_of_xyz(structs, tile_xy, threshold):
    out = []
    for i in range(len(structs)):
        found = -1
        for j in range(i):
            if rmsd_xyz(structs[i], structs[j], tile_xy) < threshold:
                found = j
                break
        out.append(found)
    return np.array(out, np.int32)
