"""Sampling of adsorption minima over a substrate grid.

Minima hopping of flexible molecules (Sec. 7): Langevin thermalisation,
FIRE relaxation and the RMSD uniqueness filter, repeated (`MinimaHopping`).

Two ways to choose where FIRE relaxations start (rigid molecules:
`Sampler`; flexible molecules, whose poses carry torsions: `FlexSampler`):

* random starts (Sec. 7: random placements over the surface), drawn by
  ``gridff_random_poses`` (rigid) or drawn as poses with uniform torsions
  and placed by ``gridff_build_poses`` (flexible);
* learned proposals: a pose-proposal MLP (descriptor + noise in, pose out;
  bfloat16 tensor-core GEMMs) trained with a winner-takes-all pose loss on
  the low-energy minima that earlier relaxations found
  (``gridff_mlp_train_step``), sampled by ``gridff_mlp_propose``.

Every start is raised, if needed, until its lowest atom is at the surface's
z_floor (``gridff_random_poses`` does it for rigid random starts,
``gridff_lift`` for the others), so that no arm starts atoms inside the
substrate's repulsive wall.  Every batch then relaxes all replicas in one
``gridff_relax`` launch and
reads back the final poses, energies and status words.  A relaxation counts
as a minimum only when it converged with finite values and no atom of the
final structure below the grid floor (`accepted`; for rigid batches, whose
positions are not read back, no atom below the floor at any step): the grid
defines no energy below its floor, where the kernels clamp to the bottom
plane.  It is a
*hit* when it is a minimum and its energy is within ``tol`` (0.01 eV) of the
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
    poses: np.ndarray        # (n, 7) final poses (rigid) or (n, atoms, 3) positions (flexible)
    energy: np.ndarray       # (n,) eV
    converged: np.ndarray    # (n,) bool: accepted minima (see `accepted`)
    wall_s: float            # proposal + relaxation + read-back, host clock
    kernel_ms: float         # the relaxation launch alone (CUDA events)


def accepted(status: np.ndarray, x: np.ndarray | None = None, z_floor: float | None = None) -> np.ndarray:
    """Relaxations that count as minima: converged with finite values and,
    given the final structures x (n, atoms, 3) and the grid floor z_floor,
    no atom of the final structure below the floor; without them, no atom
    below the grid at any step of the relaxation (the status bit, which also
    rejects an excursion that the relaxation came back from)."""
    status = np.asarray(status)
    ok = ((status & G.REP_CONVERGED) != 0) & ((status & G.REP_NONFINITE) == 0)
    if x is None:
        return ok & ((status & G.REP_BELOW) == 0)
    return ok & (np.asarray(x)[..., 2] >= z_floor).all(axis=-1)


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
        conv = accepted(fs["status"])
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
        self.reps.lift(s.z_floor)           # no atom below the floor of the random starts
        return self._relax(t0)

    def targets(self) -> np.ndarray:
        """Training targets (n_rep, 19) of the current (relaxed) poses: centre
        folded into the tile, unit quaternion with w >= 0, no torsions
        (`gridff_pose_targets`)."""
        return self.reps.pose_targets(self.surface.origin_xy, self.surface.tile_xy)[0]

    def unique(self, poses: np.ndarray, energy: np.ndarray, threshold: float = 0.1) -> np.ndarray:
        """Indices of the structurally unique poses, lowest energy first."""
        order = np.argsort(energy, kind="stable")
        dup = self.reps.rmsd_unique(poses[order], self.surface.tile_xy, threshold)
        return order[dup < 0]

    def close(self):
        self.reps.close()


@dataclass
class FlexSampler:
    """Random starts and learned proposals for a flexible molecule.  A pose
    is (centre, orientation, up to 12 torsions) and becomes atom positions
    through the library's pose builder (`gridff_build_poses`); random starts
    draw the centre over the tile and the height band, the orientation
    uniformly and every torsion uniformly in (-pi, pi].  After each batch the
    relaxed structures are also turned into poses (`gridff_pose_targets`),
    the training targets of the proposal network."""
    ctx: G.Context
    grid: G.Grid
    mol: object
    surface: Surface
    n_rep: int = 4096
    nsteps: int = 2000
    fire: G.FireParams = field(default_factory=lambda: G.fire_params(f_conv=1e-3))

    def __post_init__(self):
        self.reps = G.Replicas(self.ctx, [self.mol], [0] * self.n_rep)
        self.desc = G.molecule_descriptor(self.mol)
        self.n_rot = len(self.reps.template_rotors(0))

    def _relax(self, t0) -> Batch:
        G.relax(self.ctx, self.grid, self.reps, self.nsteps, self.fire, check=False)
        fs = self.reps.fire_state()
        x = self.reps.positions().reshape(self.n_rep, self.mol.n, 3)
        wall = time.perf_counter() - t0
        conv = accepted(fs["status"], x, self.grid.floor)
        return Batch(x, fs["energy"], conv, wall, self.ctx.last_kernel_ms())

    def random_batch(self, seed: int) -> Batch:
        s = self.surface
        t0 = time.perf_counter()
        g = np.random.default_rng(seed)
        P = np.zeros((self.n_rep, G.MLP_OUT), np.float32)
        P[:, 0] = s.origin_xy[0] + g.uniform(0, s.tile_xy[0], self.n_rep)
        P[:, 1] = s.origin_xy[1] + g.uniform(0, s.tile_xy[1], self.n_rep)
        P[:, 2] = g.uniform(s.z_lo, s.z_hi, self.n_rep)
        P[:, 3:7] = g.standard_normal((self.n_rep, 4))
        P[:, 7:7 + self.n_rot] = g.uniform(-np.pi, np.pi, (self.n_rep, self.n_rot))
        self.reps.build_poses(P)
        self.reps.lift(s.z_floor)
        return self._relax(t0)

    def proposal_batch(self, net: G.MLP, seed: int) -> Batch:
        s = self.surface
        t0 = time.perf_counter()
        net.propose(self.reps, self.desc, seed, s.origin_xy, s.tile_xy)
        self.reps.lift(s.z_floor)
        return self._relax(t0)

    def targets(self):
        """Poses (n_rep, 19) and torsion masks of the current (relaxed) state."""
        return self.reps.pose_targets(self.surface.origin_xy, self.surface.tile_xy)

    def unique(self, x: np.ndarray, energy: np.ndarray, threshold: float = 0.1) -> np.ndarray:
        """Indices of the structurally unique structures (n, atoms, 3),
        lowest energy first (`gridff_rmsd_unique_xyz`)."""
        order = np.argsort(energy, kind="stable")
        dup = G.rmsd_unique_xyz(self.ctx, x[order], self.surface.tile_xy, threshold)
        return order[dup < 0]

    def close(self):
        self.reps.close()


def hits(b: Batch, e_best: float, tol: float = 0.01) -> np.ndarray:
    """Accepted minima within tol of the best-known energy."""
    return b.converged & (b.energy <= e_best + tol)


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


def train_on_device(net: G.MLP, desc: np.ndarray, targets: np.ndarray, surface: Surface, steps: int,
                    batch: int = 256, K: int = 8, lr: float = 1e-3, seed: int = 0):
    """The same training, with the batches drawn on the device and no host
    round trip between steps (gridff_mlp_train); returns the losses."""
    net.set_targets(targets)
    return net.train(steps, batch, K, desc, seed, G.train_params(lr=lr, tile=surface.tile_xy))


def new_network(ctx: G.Context, targets: np.ndarray, seed: int = 0) -> G.MLP:
    net = G.MLP(ctx, (N_DESC + N_NOISE,) + HIDDEN + (G.MLP_OUT,))
    out_bias = np.zeros(G.MLP_OUT, np.float32)
    out_bias[:3] = targets[:, :3].mean(0)
    out_bias[3] = 1.0
    Ws, bs = init_params(net.sizes, seed, out_bias)
    net.set_params(Ws, bs)
    return net


class MinimaHopping:
    """Minima hopping of flexible replicas adsorbed on the substrate (Sec. 7):
    every hop thermalises all replicas by Langevin dynamics at T for
    `md_steps` steps (BAOAB, `gridff_langevin`), relaxes them by FIRE until
    |F| < f_conv (0.1 meV/A in the paper), and compares every accepted
    structure with all minima found so far by the RMSD criterion
    (`gridff_rmsd_unique_xyz`, 0.1 A), lowest energy first.  The next hop
    starts from the relaxed structures; a replica whose relaxed structure
    has an atom below the grid floor, or that went non-finite, starts it
    from its initial structure instead (`restart`).  `curve` records
    (seconds of sampling, unique minima, accepted relaxations) after each
    hop, `below` the replicas restarted."""

    def __init__(self, ctx: G.Context, grid: G.Grid, mol, x0: np.ndarray, tile_xy, temperature=300.0,
                 md_steps=1000, dt=1.0, gamma=0.01, f_conv=1e-4, relax_steps=5000, rmsd=0.1, seed=1,
                 restart=True):
        self.ctx, self.grid, self.mol, self.tile = ctx, grid, mol, tuple(tile_xy)
        n_rep = len(x0)
        self.x0 = np.array(x0, np.float32).reshape(n_rep, mol.n, 3)
        self.restart = restart
        self.reps = G.Replicas(ctx, [mol], [0] * n_rep)
        self.reps.set_state(self.x0.ravel())
        self.T, self.md_steps, self.dt, self.gamma = temperature, md_steps, dt, gamma
        self.fire = G.fire_params(f_conv=f_conv)
        self.relax_steps, self.rmsd, self.seed = relax_steps, rmsd, seed
        self.step = 0
        self.db_x = np.zeros((0, mol.n, 3), np.float32)
        self.db_E = np.zeros(0)
        self.elapsed = 0.0
        self.curve = []
        self.below = []                  # replicas restarted, per hop

    def hop(self):
        t0 = time.perf_counter()
        G.langevin(self.ctx, self.grid, self.reps, self.md_steps, self.dt, self.T, self.gamma, self.seed,
                   step0=self.step)
        self.step += self.md_steps
        G.relax(self.ctx, self.grid, self.reps, self.relax_steps, self.fire, check=False)
        fs = self.reps.fire_state()
        x = self.reps.positions().reshape(self.x0.shape)
        conv = accepted(fs["status"], x, self.grid.floor)
        lost = ((fs["status"] & G.REP_NONFINITE) != 0) | (x[..., 2] < self.grid.floor).any(axis=-1)
        self.below.append(int(np.count_nonzero(lost)))
        cand_x, cand_E = x[conv], fs["energy"][conv]
        order = np.argsort(cand_E, kind="stable")
        cand_x, cand_E = cand_x[order], cand_E[order]
        S = np.concatenate([self.db_x, cand_x])
        dup = G.rmsd_unique_xyz(self.ctx, S, self.tile, self.rmsd) if len(S) else np.zeros(0, np.int32)
        new = dup[len(self.db_x):] < 0
        self.db_x = np.concatenate([self.db_x, cand_x[new]])
        self.db_E = np.concatenate([self.db_E, cand_E[new]])
        if self.restart and lost.any():
            xs, vs = self.reps.get_state()
            xs = xs.reshape(self.x0.shape)
            vs = vs.reshape(self.x0.shape)
            xs[lost] = self.x0[lost]
            vs[lost] = 0.0
            self.reps.set_state(xs.ravel(), vs.ravel())
        self.elapsed += time.perf_counter() - t0
        self.curve.append((self.elapsed, len(self.db_x), int(conv.sum())))
        return self.curve[-1]

    def close(self):
        self.reps.close()
