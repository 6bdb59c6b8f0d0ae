"""Rigid-body kinematics, FIRE relaxation and NVE integration (FP64).

Oracle (test infrastructure), vectorised over independent replicas (the
paper's multi-replica scheme, Sec. 7).  Units: A, fs, amu, eV; an
acceleration F/m in eV/(A amu) is ACC * F/m in A/fs^2.

FIRE (Sec. 6 uses FIRE with a 1e-3 eV/A force threshold; the published
algorithm is Bitzek et al. 2006).  Reading of the steps, for one replica
that has not converged, per iteration:

  1. F <- F(x)
  2. if |F| < f_conv (2-norm over all 3N components, Sec. 7): converged,
     no update
  3. P = F.v
  4. if P > 0: v <- (1 - a) v + a |v| F/|F|;  if N+ > N_min:
     dt <- min(dt f_inc, dt_max), a <- a f_a;  N+ <- N+ + 1
     else:      v <- 0, dt <- dt f_dec, a <- a_start, N+ <- 0
  5. v <- v + ACC F/m dt                    (semi-implicit Euler)
  6. dr = v dt, capped per atom at d_max;  x <- x + dr

Rigid molecules (body frame = principal axes, centred at the centre of
mass) apply the same rule to the translation (v, F_tot) and to the rotation
(body angular velocity w, body torque tau) separately, with P = F_tot.v +
tau.w, |F_tot|^2 + |tau|^2 as the convergence norm, w <- w + ACC tau/I dt,
and the orientation advanced by the exact rotation of angle |w| dt about w
(capped so that no atom moves more than d_max).

NVE: velocity Verlet for flexible molecules; the NO_SQUISH symplectic
splitting (Miller et al., J. Chem. Phys. 116, 8649 (2002)) for rigid ones.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ACC = 9.648533e-3            # A/fs^2 per eV/(A amu)

CONVERGED = 1
BELOW_GRID = 2
NOT_FINITE = 4


@dataclass
class FireParams:
    dt_start: float = 0.5
    dt_max: float = 2.0
    n_min: int = 5
    f_inc: float = 1.1
    f_dec: float = 0.5
    alpha_start: float = 0.1
    f_alpha: float = 0.99
    d_max: float = 0.1
    f_conv: float = 1e-3


# ---------------------------------------------------------------------------
# quaternions (w, x, y, z)
# ---------------------------------------------------------------------------
def quat_matrix(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z], -1),
    ], -2)


def quat_mul(a, b):
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], -1)


def rigid_constants(body, mass):
    """Total mass, principal moments (body frame must be principal and
    centred at the centre of mass) and the largest atom radius."""
    b = np.asarray(body, np.float64)
    m = np.asarray(mass, np.float64)
    M = m.sum()
    I = np.array([np.sum(m * (np.sum(b * b, 1) - b[:, k] ** 2)) for k in range(3)])
    return M, I, float(np.max(np.linalg.norm(b, axis=1)))


def rigid_positions(com, quat, body):
    """r_i = R(q) b_i + com; shapes (R,3), (R,4), (n,3) -> (R, n, 3)."""
    return np.einsum("rij,nj->rni", quat_matrix(quat), body) + com[:, None, :]


def rigid_reduce(F, quat, body):
    """Total force (lab frame) and torque about the centre of mass in the
    body frame: tau_b = sum_i b_i x (R^T F_i)."""
    Ft = F.sum(1)
    Fb = np.einsum("rji,rnj->rni", quat_matrix(quat), F)     # R^T F
    tau = np.cross(np.broadcast_to(body, Fb.shape), Fb).sum(1)
    return Ft, tau


def _rotate_body(quat, w, angle):
    """q <- q (x) (cos(angle/2), sin(angle/2) w/|w|), renormalised."""
    wn = np.linalg.norm(w, axis=-1)
    axis = np.where(wn[:, None] > 0, w / np.where(wn > 0, wn, 1.0)[:, None], 0.0)
    dq = np.concatenate([np.cos(angle / 2)[:, None], np.sin(angle / 2)[:, None] * axis], 1)
    q = quat_mul(quat, dq)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# force functions
# ---------------------------------------------------------------------------
def make_force_fn(coefs, channels, origin, spacing, mol, alpha=1.5, intra=True,
                  dtype=np.float64, ghost=0):
    """Force function x (R, n, 3) -> (E (R,), F (R, n, 3), flags (R,)): grid
    interaction (Sec. 3, Sec. 5) plus, for flexible molecules, the
    intramolecular terms."""
    from . import grid as ogrid
    from . import intra as ointra

    def fn(x):
        Rn, n, _ = x.shape
        pts = x.reshape(-1, 3)
        Q = np.tile(mol.q, Rn); Rr = np.tile(mol.R, Rn); ep = np.tile(mol.eps, Rn)
        E, F, below = ogrid.grid_energy_forces(coefs, channels, origin, spacing, pts,
                                               Q, Rr, ep, alpha, dtype, ghost)
        E = E.astype(np.float64).reshape(Rn, n).sum(1)
        F = F.astype(np.float64).reshape(Rn, n, 3)
        flags = np.where(below.reshape(Rn, n).any(1), BELOW_GRID, 0)
        if intra and len(mol.bonds):
            Ei, Fi = ointra.energy_forces(x, mol, alpha)
            E = E + Ei
            F = F + Fi
        return E, F, flags
    return fn


# ---------------------------------------------------------------------------
# FIRE
# ---------------------------------------------------------------------------
def fire_flexible(x, v, mass, force_fn, nsteps, p: FireParams = FireParams(), state=None):
    """FIRE on flexible replicas. x, v: (R, n, 3). Returns a dict with the
    final x, v, E, status flags, per-replica evaluation counts and the FIRE
    scalars (dt, alpha, nplus)."""
    x = np.array(x, np.float64); v = np.array(v, np.float64)
    Rn = x.shape[0]
    m = np.asarray(mass, np.float64)[None, :, None]
    st = dict(dt=np.full(Rn, p.dt_start), alpha=np.full(Rn, p.alpha_start),
              nplus=np.zeros(Rn, np.int64), status=np.zeros(Rn, np.int64),
              steps=np.zeros(Rn, np.int64))
    if state is not None:
        st.update({k: np.array(val) for k, val in state.items()})
    E = np.zeros(Rn)
    for _ in range(nsteps):
        active = (st["status"] & (CONVERGED | NOT_FINITE)) == 0
        if not active.any():
            break
        Ea, F, flags = force_fn(x)
        E = np.where(active, Ea, E)
        st["status"] |= np.where(active, flags, 0)
        st["steps"] += active
        bad = active & ~(np.isfinite(F).all((1, 2)) & np.isfinite(x).all((1, 2)))
        st["status"] |= np.where(bad, NOT_FINITE, 0)
        f2 = np.sum(F * F, (1, 2))
        conv = active & ~bad & (np.sqrt(f2) < p.f_conv)
        st["status"] |= np.where(conv, CONVERGED, 0)
        upd = active & ~bad & ~conv
        P = np.sum(F * v, (1, 2))
        v2 = np.sum(v * v, (1, 2))
        pos = upd & (P > 0)
        neg = upd & ~(P > 0)
        a = st["alpha"][:, None, None]
        scale = np.sqrt(v2 / np.where(f2 > 0, f2, 1.0))[:, None, None]
        v = np.where(pos[:, None, None], (1 - a) * v + a * scale * F, v)
        grow = pos & (st["nplus"] > p.n_min)
        st["dt"] = np.where(grow, np.minimum(st["dt"] * p.f_inc, p.dt_max), st["dt"])
        st["alpha"] = np.where(grow, st["alpha"] * p.f_alpha, st["alpha"])
        st["nplus"] = np.where(pos, st["nplus"] + 1, st["nplus"])
        v = np.where(neg[:, None, None], 0.0, v)
        st["dt"] = np.where(neg, st["dt"] * p.f_dec, st["dt"])
        st["alpha"] = np.where(neg, p.alpha_start, st["alpha"])
        st["nplus"] = np.where(neg, 0, st["nplus"])
        dt = st["dt"][:, None, None]
        v = np.where(upd[:, None, None], v + ACC * F / m * dt, v)
        dr = v * dt
        dn = np.linalg.norm(dr, axis=2, keepdims=True)
        dr = np.where(dn > p.d_max, dr * (p.d_max / np.where(dn > 0, dn, 1.0)), dr)
        x = np.where(upd[:, None, None], x + dr, x)
    st.update(x=x, v=v, E=E)
    return st


def fire_rigid(com, quat, vel, omega, body, mass, force_fn, nsteps,
               p: FireParams = FireParams(), state=None):
    """FIRE on rigid replicas (pose = centre of mass + quaternion; velocities
    = COM velocity (lab) and angular velocity (body frame))."""
    com = np.array(com, np.float64); quat = np.array(quat, np.float64)
    vel = np.array(vel, np.float64); omega = np.array(omega, np.float64)
    body = np.asarray(body, np.float64)
    M, I, rmax = rigid_constants(body, mass)
    Rn = com.shape[0]
    st = dict(dt=np.full(Rn, p.dt_start), alpha=np.full(Rn, p.alpha_start),
              nplus=np.zeros(Rn, np.int64), status=np.zeros(Rn, np.int64),
              steps=np.zeros(Rn, np.int64))
    if state is not None:
        st.update({k: np.array(val) for k, val in state.items()})
    E = np.zeros(Rn)
    for _ in range(nsteps):
        active = (st["status"] & (CONVERGED | NOT_FINITE)) == 0
        if not active.any():
            break
        x = rigid_positions(com, quat, body)
        Ea, F, flags = force_fn(x)
        E = np.where(active, Ea, E)
        st["status"] |= np.where(active, flags, 0)
        st["steps"] += active
        Ft, tau = rigid_reduce(F, quat, body)
        bad = active & ~(np.isfinite(Ft).all(1) & np.isfinite(tau).all(1))
        st["status"] |= np.where(bad, NOT_FINITE, 0)
        f2 = np.sum(Ft * Ft, 1) + np.sum(tau * tau, 1)
        conv = active & ~bad & (np.sqrt(f2) < p.f_conv)
        st["status"] |= np.where(conv, CONVERGED, 0)
        upd = active & ~bad & ~conv
        P = np.sum(Ft * vel, 1) + np.sum(tau * omega, 1)
        pos = upd & (P > 0)
        neg = upd & ~(P > 0)
        a = st["alpha"][:, None]
        fn_ = np.linalg.norm(Ft, axis=1, keepdims=True)
        tn_ = np.linalg.norm(tau, axis=1, keepdims=True)
        vn_ = np.linalg.norm(vel, axis=1, keepdims=True)
        wn_ = np.linalg.norm(omega, axis=1, keepdims=True)
        Fhat = np.where(fn_ > 0, Ft / np.where(fn_ > 0, fn_, 1.0), 0.0)
        That = np.where(tn_ > 0, tau / np.where(tn_ > 0, tn_, 1.0), 0.0)
        vel = np.where(pos[:, None], (1 - a) * vel + a * vn_ * Fhat, vel)
        omega = np.where(pos[:, None], (1 - a) * omega + a * wn_ * That, omega)
        grow = pos & (st["nplus"] > p.n_min)
        st["dt"] = np.where(grow, np.minimum(st["dt"] * p.f_inc, p.dt_max), st["dt"])
        st["alpha"] = np.where(grow, st["alpha"] * p.f_alpha, st["alpha"])
        st["nplus"] = np.where(pos, st["nplus"] + 1, st["nplus"])
        vel = np.where(neg[:, None], 0.0, vel)
        omega = np.where(neg[:, None], 0.0, omega)
        st["dt"] = np.where(neg, st["dt"] * p.f_dec, st["dt"])
        st["alpha"] = np.where(neg, p.alpha_start, st["alpha"])
        st["nplus"] = np.where(neg, 0, st["nplus"])
        dt = st["dt"]
        vel = np.where(upd[:, None], vel + ACC * Ft / M * dt[:, None], vel)
        omega = np.where(upd[:, None], omega + ACC * tau / I[None, :] * dt[:, None], omega)
        dr = vel * dt[:, None]
        dn = np.linalg.norm(dr, axis=1, keepdims=True)
        dr = np.where(dn > p.d_max, dr * (p.d_max / np.where(dn > 0, dn, 1.0)), dr)
        com = np.where(upd[:, None], com + dr, com)
        ang = np.linalg.norm(omega, axis=1) * dt
        ang = np.minimum(ang, p.d_max / rmax)
        quat = np.where(upd[:, None], _rotate_body(quat, omega, ang), quat)
    st.update(com=com, quat=quat, vel=vel, omega=omega, E=E)
    return st


# ---------------------------------------------------------------------------
# NVE
# ---------------------------------------------------------------------------
def kinetic_flexible(v, mass):
    return 0.5 * np.sum(np.asarray(mass)[None, :, None] * v * v, (1, 2)) / ACC


def nve_flexible(x, v, mass, force_fn, nsteps, dt, record_every=1):
    """Velocity Verlet.  Returns (x, v, trace) with trace[k] = total energy
    (eV) after every ``record_every`` steps (trace[0] = start)."""
    x = np.array(x, np.float64); v = np.array(v, np.float64)
    m = np.asarray(mass, np.float64)[None, :, None]
    E, F, _ = force_fn(x)
    trace = [E + kinetic_flexible(v, mass)]
    for s in range(nsteps):
        v = v + 0.5 * dt * ACC * F / m
        x = x + dt * v
        E, F, _ = force_fn(x)
        v = v + 0.5 * dt * ACC * F / m
        if (s + 1) % record_every == 0:
            trace.append(E + kinetic_flexible(v, mass))
    return x, v, np.array(trace)


def _S(q):
    """4x4 matrix with S(q) u = q (x) u; its columns are q, P1 q, P2 q, P3 q."""
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([np.stack([w, -x, -y, -z], -1),
                     np.stack([x, w, -z, y], -1),
                     np.stack([y, z, w, -x], -1),
                     np.stack([z, -y, x, w], -1)], -2)


def _perm(k, u):
    """P_k u for k = 1, 2, 3 (the k-th column map of S)."""
    w, x, y, z = u[..., 0], u[..., 1], u[..., 2], u[..., 3]
    if k == 1:
        return np.stack([-x, w, z, -y], -1)
    if k == 2:
        return np.stack([-y, -z, w, x], -1)
    return np.stack([-z, y, -x, w], -1)


def rigid_kinetic(vel, omega, M, I):
    return 0.5 * (M * np.sum(vel * vel, 1) + np.sum(I[None, :] * omega * omega, 1)) / ACC


def nve_rigid(com, quat, vel, omega, body, mass, force_fn, nsteps, dt, record_every=1):
    """NO_SQUISH rigid-body NVE: half kick (F_tot, body torque), drift of
    the centre of mass, free-rotor sub-rotations about body axes 3, 2, 1, 2, 3
    (dt/2, dt/2, dt, dt/2, dt/2), forces, half kick.  The conjugate
    quaternion momentum is p = 2 S(q) (0, I w).  Returns (com, quat, vel,
    omega, trace)."""
    com = np.array(com, np.float64); q = np.array(quat, np.float64)
    vel = np.array(vel, np.float64); omega = np.array(omega, np.float64)
    body = np.asarray(body, np.float64)
    M, I, _ = rigid_constants(body, mass)
    Lb = omega * I[None, :]
    pq = 2 * np.einsum("rij,rj->ri", _S(q), np.concatenate([np.zeros((len(q), 1)), Lb], 1))

    def forces(com, q):
        E, F, _ = force_fn(rigid_positions(com, q, body))
        Ft, tau = rigid_reduce(F, q, body)
        return E, Ft, tau

    def omega_of(q, pq):
        L = 0.5 * np.einsum("rji,rj->ri", _S(q), pq)[:, 1:]
        return L / I[None, :]

    def kick(pq, vel, q, Ft, tau, h):
        vel = vel + h * ACC * Ft / M
        T = np.concatenate([np.zeros((len(q), 1)), tau], 1)
        pq = pq + h * ACC * 2 * np.einsum("rij,rj->ri", _S(q), T)
        return pq, vel

    def rotate(k, h, q, pq):
        zeta = h * np.sum(pq * _perm(k, q), 1) / (4 * I[k - 1])
        c, s = np.cos(zeta)[:, None], np.sin(zeta)[:, None]
        return c * q + s * _perm(k, q), c * pq + s * _perm(k, pq)

    E, Ft, tau = forces(com, q)
    trace = [E + rigid_kinetic(vel, omega_of(q, pq), M, I)]
    for s in range(nsteps):
        pq, vel = kick(pq, vel, q, Ft, tau, 0.5 * dt)
        com = com + dt * vel
        for k, h in ((3, 0.5 * dt), (2, 0.5 * dt), (1, dt), (2, 0.5 * dt), (3, 0.5 * dt)):
            q, pq = rotate(k, h, q, pq)
        E, Ft, tau = forces(com, q)
        pq, vel = kick(pq, vel, q, Ft, tau, 0.5 * dt)
        if (s + 1) % record_every == 0:
            trace.append(E + rigid_kinetic(vel, omega_of(q, pq), M, I))
    return com, q, vel, omega_of(q, pq), np.array(trace)


KB = 8.617333262e-5   # eV/K


def langevin_noise(seed, replicas, step, n_comp):
    """xi[r, m] of the library's Langevin noise stream for global step
    `step`: the SplitMix64 output of splitmix64(seed ^ splitmix64(r)) ^
    (512 step + m), turned into a normal by Box-Muller (float64 here)."""
    from .mlp import splitmix64
    out = np.empty((len(replicas), n_comp))
    for k, r in enumerate(replicas):
        key = splitmix64(seed ^ splitmix64(int(r)))
        for m in range(n_comp):
            s = splitmix64(key ^ (512 * step + m))
            u1 = ((s >> 40) + 1) / 2.0 ** 24
            u2 = ((s >> 16) & 0xFFFFFF) / 2.0 ** 24
            out[k, m] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def langevin_baoab(x, v, mass, force_fn, nsteps, dt, T, gamma, noise):
    """Langevin dynamics by the BAOAB splitting (Leimkuhler and Matthews):
    half kick, half drift, exact Ornstein-Uhlenbeck step
    v <- c1 v + c2 sqrt(kB T / m) xi (c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2)),
    half drift, half kick.  noise(step) -> xi (R, n*3).  Returns (x, v, E)
    with E the energy of the final state."""
    x = np.array(x, np.float64); v = np.array(v, np.float64)
    R, n, _ = x.shape
    m = np.asarray(mass, np.float64)[None, :, None]
    c1 = np.exp(-gamma * dt)
    c2 = np.sqrt(1.0 - c1 * c1)
    sig = np.sqrt(KB * T * ACC / m)
    E, F, _ = force_fn(x)
    for s in range(nsteps):
        v = v + 0.5 * dt * ACC * F / m
        x = x + 0.5 * dt * v
        v = c1 * v + c2 * sig * noise(s).reshape(R, n, 3)
        x = x + 0.5 * dt * v
        E, F, _ = force_fn(x)
        v = v + 0.5 * dt * ACC * F / m
    return x, v, E
