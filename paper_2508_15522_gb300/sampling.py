"""Sampling of adsorption minima of a rigid molecule over a substrate grid.

Two ways to choose where FIRE relaxations start, both on the device:

* random starts (Sec. 7: random placements over the surface), drawn by
  ``gridff_random_poses``;
* learned proposals: a pose-proposal MLP (descriptor + noise in, pose out;
  bfloat16 tensor-core GEMMs) trained with a winner-takes-all pose loss on
  the low-energy minima that earlier relaxations found
  (``gridff_mlp_train_step``), sampled by ``gridff_mlp_propose``.

Every batch then relaxes all replicas in one ``gridff_relax`` launch and
reads back the final poses, energies and status words.  A relaxation is a
*hit* when it converged and its energy is within ``tol`` (0.01 eV) of the
best-known minimum energy; hits are deduplicated with the RMSD filter of
Sec. 7 (``gridff_rmsd_unique``, 0.1 A).  This module only orders the calls
and moves their inputs and outputs; the arithmetic runs in the library.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import gridff as G

N_DESC = 64
N_NOISE = 16
HIDDEN = (256, 256, 256)


@dataclass
class Batch:
    poses: np.ndarray        # (n, 7) final poses
    energy: np.ndarray       # (n,) eV
    converged: np.ndarray    # (n,) bool
    wall_s: float            # proposal + relaxation + read-back, host clock
    kernel_ms: float         # the relaxation launch alone (CUDA events)


@dataclass
class Surface:
    """Where the molecule may sit: the periodic tile and the height band of
    the random starts (all A)."""
    origin_xy: tuple
    tile_xy: tuple
    z_lo: float
    z_hi: float
    z_floor: float


@dataclass
class Sampler:
    ctx: G.Context
    grid: G.Grid
    mol: object                      # molecule template (principal body frame)
    surface: Surface
    n_rep: int = 4096
    nsteps: int = 2000
    fire: G.FireParams = field(default_factory=lambda: G.fire_params(f_conv=1e-3))

    def __post_init__(self):
        self.reps = G.Replicas(self.ctx, [self.mol], [0] * self.n_rep, rigid=True)
        self.desc = G.molecule_descriptor(self.mol)

    def _relax(self, t0) -> Batch:
        G.relax(self.ctx, self.grid, self.reps, self.nsteps, self.fire, check=False)
        fs = self.reps.fire_state()
        x, _ = self.reps.get_state()
        wall = time.perf_counter() - t0
        conv = (fs["status"] & G.REP_CONVERGED) != 0
        return Batch(x.reshape(-1, 7), fs["energy"], conv, wall, self.ctx.last_kernel_ms())

    def random_batch(self, seed: int) -> Batch:
        s = self.surface
        t0 = time.perf_counter()
        self.reps.random_poses(seed, s.origin_xy, s.tile_xy, s.z_lo, s.z_hi, s.z_floor)
        return self._relax(t0)

    def proposal_batch(self, net: G.MLP, seed: int) -> Batch:
        s = self.surface
        t0 = time.perf_counter()
        net.propose(self.reps, self.desc, seed, s.origin_xy, s.tile_xy)
        return self._relax(t0)

    def unique(self, poses: np.ndarray, energy: np.ndarray, threshold: float = 0.1) -> np.ndarray:
        """Indices of the structurally unique poses, lowest energy first."""
        order = np.argsort(energy, kind="stable")
        dup = self.reps.rmsd_unique(poses[order], self.surface.tile_xy, threshold)
        return order[dup < 0]

    def close(self):
        self.reps.close()


def hits(b: Batch, e_best: float, tol: float = 0.01) -> np.ndarray:
    """Converged relaxations within tol of the best-known energy."""
    return b.converged & (b.energy <= e_best + tol)


def pose_targets(poses: np.ndarray, surface: Surface) -> np.ndarray:
    """(n, 19) training targets: centre folded into the tile, unit
    quaternion, no torsions (rigid)."""
    T = np.zeros((len(poses), G.MLP_OUT), np.float32)
    c = poses[:, :3].astype(np.float64)
    for a in range(2):
        c[:, a] = surface.origin_xy[a] + np.mod(c[:, a] - surface.origin_xy[a], surface.tile_xy[a])
    q = poses[:, 3:7].astype(np.float64)
    T[:, :3] = c
    T[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    return T


def init_params(sizes, seed: int, out_bias=None):
    """He-uniform weights, zero biases; optional initial output bias."""
    g = np.random.default_rng(seed)
    Ws, bs = [], []
    for i, o in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / i)
        Ws.append(g.uniform(-lim, lim, (o, i)).astype(np.float32))
        bs.append(np.zeros(o, np.float32))
    if out_bias is not None:
        bs[-1][:] = out_bias
    return Ws, bs


def train(net: G.MLP, desc: np.ndarray, targets: np.ndarray, surface: Surface, steps: int,
          batch: int = 256, K: int = 8, lr: float = 1e-3, seed: int = 0):
    """Winner-takes-all training on a set of target poses; returns the loss
    of every step.  Each step draws `batch` targets and K noise rows per
    target."""
    g = np.random.default_rng(seed)
    tp = G.train_params(lr=lr, tile=surface.tile_xy)
    d = np.broadcast_to(desc.astype(np.float32), (batch * K, N_DESC))
    losses = []
    for _ in range(steps):
        idx = g.integers(0, len(targets), batch)
        x = np.concatenate([d, g.standard_normal((batch * K, N_NOISE), np.float32)], 1)
        losses.append(net.train_step(x, targets[idx], K, tp))
    return np.array(losses)


def new_network(ctx: G.Context, targets: np.ndarray, seed: int = 0) -> G.MLP:
    net = G.MLP(ctx, (N_DESC + N_NOISE,) + HIDDEN + (G.MLP_OUT,))
    out_bias = np.zeros(G.MLP_OUT, np.float32)
    out_bias[:3] = targets[:, :3].mean(0)
    out_bias[3] = 1.0
    Ws, bs = init_params(net.sizes, seed, out_bias)
    net.set_params(Ws, bs)
    return net
