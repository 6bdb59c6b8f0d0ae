// Fused hot path: per-atom tricubic B-spline interpolation of the substrate
// grid (Sec. 3, Sec. 5), intramolecular forces, per-replica warp reductions
// and FIRE / NVE updates (Sec. 6, Sec. 7), one warp per replica.
//
// Work split inside a warp: the 32 lanes form 8 quads; each quad evaluates
// one atom at a time.  Lane q of a quad gathers record q of each of the 16
// z-runs of the atom's 4x4x4 stencil, so one warp-wide load instruction
// fetches 8 whole runs (8 contiguous 64-byte segments) instead of 32
// scattered 16-byte pieces; the quad then sums its partial contractions with
// two shuffles.  Flexible replicas keep positions, velocities and forces in
// shared memory; the integrator updates run with lanes over atoms.
#include <math.h>

#include <vector>

#include "internal.h"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;
#ifndef GRIDFF_MIN_BLOCKS_PER_SM
#define GRIDFF_MIN_BLOCKS_PER_SM 4
#endif
constexpr int kMinBlocksPerSM = GRIDFF_MIN_BLOCKS_PER_SM;
#ifndef GRIDFF_STAGED_NB
#define GRIDFF_STAGED_NB 0
#endif
constexpr int kQuads = 8;                 // atoms evaluated per warp at a time
constexpr int kMaxA = GRIDFF_MAX_ATOMS;
constexpr unsigned kFull = 0xffffffffu;

struct FireP {
  float dt_start, dt_max, f_inc, f_dec, alpha_start, f_alpha, d_max, f_conv2;
  int n_min;
};

struct Control {
  const volatile int* abort_flag;   // host-mapped
  unsigned long long budget_ns;     // 0 = none
  DevResult* res;
};

// per-warp shared state of a flexible replica
struct WarpState {
  float x[3 * kMaxA];
  float v[3 * kMaxA];
  float f[3 * kMaxA];
  float eg[kMaxA];     // grid energy per atom
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float qsum(float v) {
  v += __shfl_xor_sync(kFull, v, 1);
  v += __shfl_xor_sync(kFull, v, 2);
  return v;
}

// Cubic B-spline weights w_j = B(t - j), j = -1..2, and dB/dt for t in [0,1),
// the polynomial pieces of Eq. Bspline on the four intervals.
__device__ __forceinline__ void bspline_weights(float t, float w[4], float dw[4]) {
  const float s = 1.f - t, t2 = t * t, t3 = t2 * t;
  const float sixth = 1.f / 6.f;
  w[0] = s * s * s * sixth;
  w[1] = fmaf(3.f, t3, fmaf(-6.f, t2, 4.f)) * sixth;
  w[2] = fmaf(-3.f, t3, fmaf(3.f, t2, fmaf(3.f, t, 1.f))) * sixth;
  w[3] = t3 * sixth;
  dw[0] = -0.5f * s * s;
  dw[1] = fmaf(1.5f, t2, -2.f * t);
  dw[2] = fmaf(-1.5f, t2, t + 0.5f);
  dw[3] = 0.5f * t2;
}

// Energy and force of one atom in the substrate field (Eqs. E, E_Coulomb,
// E_Morse), evaluated by the 4 lanes of a quad (q = lane & 3); every lane of
// the quad returns the full result.  The channels are combined per node with
// the atom's factors (Q, P, L); lane q accumulates the x/y-weighted sums of
// node z+q-1 over the 16 runs, applies its own z weight, and the quad sums.
// The force is minus the analytic gradient of the interpolant (Sec. 5).
// `act` false: the quad has no atom (it still takes part in the shuffles).
__device__ __forceinline__ void grid_quad(const GridView& g, int q, bool act, float x, float y, float z,
                                          float4 par, float& e, float& fx, float& fy, float& fz,
                                          int& flags) {
  // fold into the periodic tile (Sec. 4)
  float xr = x - g.x0, yr = y - g.y0;
  xr = fmaf(-g.Lx, floorf(xr * g.inv_Lx), xr);
  yr = fmaf(-g.Ly, floorf(yr * g.inv_Ly), yr);
  float ux = xr * g.inv_dx, uy = yr * g.inv_dy, uz = (z - g.z0) * g.inv_dz;
  float flx = floorf(ux), fly = floorf(uy);
  float tx = fminf(fmaxf(ux - flx, 0.f), 1.f), ty = fminf(fmaxf(uy - fly, 0.f), 1.f);
  int ix = (int)flx, iy = (int)fly;
  if (ix >= g.nx) ix -= g.nx;
  if (iy >= g.ny) iy -= g.ny;
  ix = min(max(ix, 0), g.nx - 1);     // any input, even non-finite, stays in bounds
  iy = min(max(iy, 0), g.ny - 1);
  if (act && uz < 0.f) flags |= GRIDFF_REP_BELOW;
  uz = fmaxf(uz, 0.f);
  bool inside = act && (uz < (float)(g.nz - 1));   // above the grid (or NaN): field ~ 0
  float flz = floorf(inside ? uz : 0.f);
  float tz = (inside ? uz : 0.f) - flz;
  int iz = min(max((int)flz, 0), g.nz - 2);
  float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
  bspline_weights(tx, wx, dwx);
  bspline_weights(ty, wy, dwy);
  bspline_weights(tz, wz, dwz);
  float S0 = 0.f, Sx = 0.f, Sy = 0.f;
  if (inside) {
    const float4* p0 = g.rec + ((long long)ix * g.nyp + iy) * g.nzp + iz + q;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float4 r[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) r[b] = __ldg(p0 + a * g.sx + b * g.nzp);
      float s = 0.f, sy = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float c = fmaf(par.x, r[b].x, fmaf(par.y, r[b].y, par.z * r[b].z));
        s = fmaf(wy[b], c, s);
        sy = fmaf(dwy[b], c, sy);
      }
      S0 = fmaf(wx[a], s, S0);
      Sx = fmaf(dwx[a], s, Sx);
      Sy = fmaf(wx[a], sy, Sy);
    }
  }
  const float wq = q == 0 ? wz[0] : q == 1 ? wz[1] : q == 2 ? wz[2] : wz[3];
  const float dwq = q == 0 ? dwz[0] : q == 1 ? dwz[1] : q == 2 ? dwz[2] : dwz[3];
  e = qsum(wq * S0);
  fx = -qsum(wq * Sx) * g.inv_dx;
  fy = -qsum(wq * Sy) * g.inv_dy;
  fz = -qsum(dwq * S0) * g.inv_dz;
}

__device__ __forceinline__ float3 ld3(const float* s, int i) {
  return make_float3(s[3 * i], s[3 * i + 1], s[3 * i + 2]);
}
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// This lane's share (terms q, q+4, ... of each list; partners q, q+4, ...)
// of the intramolecular force on template atom i, and of the energy counted
// at i: bonded terms once (at their first atom), nonbonded pairs half at
// each atom.  s_x holds the molecule's positions.
__device__ void intra_quad(const TemplateView& tv, int ab, int n, int i, int q, const float* s_x, float& Fx,
                           float& Fy, float& Fz, float& E) {
  const float3 xi = ld3(s_x, i);
  const int gi = ab + i;
  float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
  for (int t = tv.bond_off[gi] + q; t < tv.bond_off[gi + 1]; t += 4) {
    BondRec b = tv.bonds[t];
    float3 d = sub3(xi, ld3(s_x, b.j));
    float r = sqrtf(dot3(d, d));
    float dr = r - b.r0;
    float c = r > 0.f ? -2.f * b.k * dr / r : 0.f;
    fx += c * d.x;
    fy += c * d.y;
    fz += c * d.z;
    if (b.own) e += b.k * dr * dr;
  }
  for (int t = tv.angle_off[gi] + q; t < tv.angle_off[gi + 1]; t += 4) {
    AngleRec A = tv.angles[t];
    float3 xa = ld3(s_x, A.a), xb = ld3(s_x, A.b), xc = ld3(s_x, A.c);
    float3 u = sub3(xa, xb), w = sub3(xc, xb);
    float lu2 = dot3(u, u), lw2 = dot3(w, w);
    float inv = rsqrtf(lu2 * lw2);
    float c = dot3(u, w) * inv;
    float dEdc = 2.f * A.k * (c - A.cos0);
    float3 ga = make_float3(w.x * inv - c * u.x / lu2, w.y * inv - c * u.y / lu2, w.z * inv - c * u.z / lu2);
    float3 gc = make_float3(u.x * inv - c * w.x / lw2, u.y * inv - c * w.y / lw2, u.z * inv - c * w.z / lw2);
    float3 gr = A.role == 0 ? ga : A.role == 2 ? gc : make_float3(-ga.x - gc.x, -ga.y - gc.y, -ga.z - gc.z);
    fx -= dEdc * gr.x;
    fy -= dEdc * gr.y;
    fz -= dEdc * gr.z;
    if (A.role == 0) e += A.k * (c - A.cos0) * (c - A.cos0);
  }
  for (int t = tv.tors_off[gi] + q; t < tv.tors_off[gi + 1]; t += 4) {
    TorsionRec T = tv.tors[t];
    float3 xa = ld3(s_x, T.a), xb = ld3(s_x, T.b), xc = ld3(s_x, T.c), xd = ld3(s_x, T.d);
    float3 F = sub3(xa, xb), G = sub3(xb, xc), H = sub3(xd, xc);
    float3 A = cross3(F, G), B = cross3(H, G);
    float A2 = dot3(A, A), B2 = dot3(B, B), G2 = dot3(G, G);
    if (A2 < 1e-12f || B2 < 1e-12f || G2 < 1e-12f) continue;   // collinear: no torque
    float Gn = sqrtf(G2);
    float iAB = rsqrtf(A2 * B2);
    float cphi = dot3(A, B) * iAB;
    float sphi = dot3(cross3(B, A), G) * iAB / Gn;
    float phi = atan2f(sphi, cphi);
    float sn, cn;
    sincosf(T.n * phi, &sn, &cn);
    float dEdphi = 0.5f * T.V * T.cn0 * T.n * sn;
    float FG = dot3(F, G) / (A2 * Gn), HG = dot3(H, G) / (B2 * Gn);
    float ca = -Gn / A2, cd = Gn / B2;
    float3 gr;
    if (T.role == 0) {
      gr = make_float3(ca * A.x, ca * A.y, ca * A.z);
    } else if (T.role == 3) {
      gr = make_float3(cd * B.x, cd * B.y, cd * B.z);
    } else if (T.role == 1) {
      float a1 = -ca + FG;
      gr = make_float3(a1 * A.x - HG * B.x, a1 * A.y - HG * B.y, a1 * A.z - HG * B.z);
    } else {
      float b1 = -cd + HG;
      gr = make_float3(b1 * B.x - FG * A.x, b1 * B.y - FG * A.y, b1 * B.z - FG * A.z);
    }
    fx -= dEdphi * gr.x;
    fy -= dEdphi * gr.y;
    fz -= dEdphi * gr.z;
    if (T.role == 0) e += 0.5f * T.V * (1.f - T.cn0 * cn);
  }
  // nonbonded: Morse (eps_i eps_j, R_i + R_j) + Coulomb on pairs > 2 bonds apart
  const float4 nbi = tv.nb[gi];
  const uint32_t* ex = tv.excl + 4 * (size_t)gi;
  const uint32_t exw[4] = {ex[0], ex[1], ex[2], ex[3]};
  const float alpha = tv.alpha;
  float enb = 0.f;
  for (int j = q; j < n; j += 4) {
    if ((exw[j >> 5] >> (j & 31)) & 1u) continue;
    float4 nbj = tv.nb[ab + j];
    float3 d = sub3(xi, ld3(s_x, j));
    float r2 = dot3(d, d);
    float ir = rsqrtf(r2);
    float r = r2 * ir;
    float e1 = expf(-alpha * (r - nbi.y - nbj.y));
    float ee = nbi.z * nbj.z;
    float qq = GRIDFF_KE * nbi.x * nbj.x;
    float em = ee * e1 * (e1 - 2.f);
    float dEdr = 2.f * alpha * ee * e1 * (1.f - e1) - qq * ir * ir;
    float c = -dEdr * ir;
    fx += c * d.x;
    fy += c * d.y;
    fz += c * d.z;
    enb += em + qq * ir;
  }
  Fx += fx;
  Fy += fy;
  Fz += fz;
  E += e + 0.5f * enb;
}

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
  R[0] = w * w + x * x - y * y - z * z;
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = w * w - x * x + y * y - z * z;
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = w * w - x * x - y * y + z * z;
}

// q <- q (x) (cos(a/2), sin(a/2) u), normalised.
__device__ __forceinline__ void quat_advance(float q[4], float ux, float uy, float uz, float ang) {
  float s, c;
  sincosf(0.5f * ang, &s, &c);
  float bx = s * ux, by = s * uy, bz = s * uz;
  float w = q[0] * c - q[1] * bx - q[2] * by - q[3] * bz;
  float x = q[0] * bx + q[1] * c + q[2] * bz - q[3] * by;
  float y = q[0] * by - q[1] * bz + q[2] * c + q[3] * bx;
  float z = q[0] * bz + q[1] * by - q[2] * bx + q[3] * c;
  float inv = rsqrtf(w * w + x * x + y * y + z * z);
  q[0] = w * inv;
  q[1] = x * inv;
  q[2] = y * inv;
  q[3] = z * inv;
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// Per-replica stop check (abort flag, clock budget), every 32 steps.
__device__ __forceinline__ int stop_bits(const Control& ctl, unsigned long long t0, int lane) {
  int bits = 0;
  if (lane == 0) {
    if (*ctl.abort_flag) bits |= GRIDFF_REP_ABORTED;
    if (ctl.budget_ns && gtimer() - t0 > ctl.budget_ns) bits |= GRIDFF_REP_STEPLIMIT;
  }
  return __shfl_sync(kFull, bits, 0);
}

__device__ __forceinline__ void report(const Control& ctl, int n, int evals, int st, int steps) {
  atomicAdd(&ctl.res->atom_evals, (unsigned long long)n * (unsigned long long)evals);
  if (st & GRIDFF_REP_CONVERGED) atomicAdd(&ctl.res->n_converged, 1);
  atomicMax(&ctl.res->max_steps, steps);
  int sb = st & (GRIDFF_REP_ABORTED | GRIDFF_REP_STEPLIMIT);
  if (sb) atomicOr(&ctl.res->stop_bits, sb);
}

// Forces of one flexible replica whose positions are in s.x: grid term
// (quads over atoms) + intramolecular terms; writes s.f and s.eg and
// returns this lane's share of the energy (the caller sums the warp).
__device__ __forceinline__ double flex_forces(const GridView& g, bool use_grid, bool use_intra,
                                              const TemplateView& tv, int ab, int n, int lane, WarpState& s,
                                              int& flags) {
  __syncwarp();
  const int quad = lane >> 2, q = lane & 3;
  double e = 0.0;
  for (int base = 0; base < n; base += kQuads) {
    const int i = base + quad;
    const bool act = i < n;
    float x = 0.f, y = 0.f, z = 0.f;
    float4 par = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act) {
      x = s.x[3 * i];
      y = s.x[3 * i + 1];
      z = s.x[3 * i + 2];
      par = __ldg(&tv.par[ab + i]);
      if (!finite3(x, y, z)) flags |= GRIDFF_REP_NONFINITE;
    }
    float eg = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    if (use_grid) grid_quad(g, q, act, x, y, z, par, eg, fx, fy, fz, flags);
    float ix = 0.f, iy = 0.f, iz = 0.f, ie = 0.f;
    if (use_intra && act) intra_quad(tv, ab, n, i, q, s.x, ix, iy, iz, ie);
    ix = qsum(ix);
    iy = qsum(iy);
    iz = qsum(iz);
    e += (double)ie;
    if (act && q == 0) {
      s.f[3 * i] = fx + ix;
      s.f[3 * i + 1] = fy + iy;
      s.f[3 * i + 2] = fz + iz;
      s.eg[i] = eg;
      e += (double)eg;
    }
  }
  __syncwarp();
  return e;
}

// Grid forces of a rigid replica: total force (lab), body-frame torque and
// this lane's share of the energy.
__device__ __forceinline__ void rigid_forces(const GridView& g, const TemplateView& tv, int ab, int n, int lane,
                                             const float c[3], const float Rm[9], float Ft[3], float tq[3],
                                             double& e, int& flags) {
  const int quad = lane >> 2, q = lane & 3;
  for (int a = 0; a < 3; ++a) Ft[a] = tq[a] = 0.f;
  e = 0.0;
  for (int base = 0; base < n; base += kQuads) {
    const int i = base + quad;
    const bool act = i < n;
    float4 b = make_float4(0.f, 0.f, 0.f, 0.f), par = b;
    if (act) {
      b = __ldg(&tv.body[ab + i]);
      par = __ldg(&tv.par[ab + i]);
    }
    float px = Rm[0] * b.x + Rm[1] * b.y + Rm[2] * b.z + c[0];
    float py = Rm[3] * b.x + Rm[4] * b.y + Rm[5] * b.z + c[1];
    float pz = Rm[6] * b.x + Rm[7] * b.y + Rm[8] * b.z + c[2];
    float ei, fx, fy, fz;
    grid_quad(g, q, act, px, py, pz, par, ei, fx, fy, fz, flags);
    if (act && q == 0) {
      e += (double)ei;
      Ft[0] += fx;
      Ft[1] += fy;
      Ft[2] += fz;
      // body-frame force R^T f and torque b x (R^T f)
      float gx = Rm[0] * fx + Rm[3] * fy + Rm[6] * fz;
      float gy = Rm[1] * fx + Rm[4] * fy + Rm[7] * fz;
      float gz = Rm[2] * fx + Rm[5] * fy + Rm[8] * fz;
      tq[0] += b.y * gz - b.z * gy;
      tq[1] += b.z * gx - b.x * gz;
      tq[2] += b.x * gy - b.y * gx;
    }
  }
  for (int a = 0; a < 3; ++a) {
    Ft[a] = wsum(Ft[a]);
    tq[a] = wsum(tq[a]);
  }
  e = wsum(e);
}

// ---------------------------------------------------------------------------
// Shared-memory staged gather (cp.async): the stencil records of up to NB
// rounds of 8 atoms are in flight per warp without holding registers.
// Slot layout per stage: record j of lane l at float4 index j * 32 + l, so
// both the asynchronous writes and the reads are bank-conflict free.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

struct StencilPos {   // fold and cell of one atom (shared by issue and compute)
  int ix, iy, iz;
  float tx, ty, tz;
  bool inside;
};

__device__ __forceinline__ StencilPos locate(const GridView& g, bool act, float x, float y, float z, int& flags) {
  StencilPos sp;
  float xr = x - g.x0, yr = y - g.y0;
  xr = fmaf(-g.Lx, floorf(xr * g.inv_Lx), xr);
  yr = fmaf(-g.Ly, floorf(yr * g.inv_Ly), yr);
  float ux = xr * g.inv_dx, uy = yr * g.inv_dy, uz = (z - g.z0) * g.inv_dz;
  float flx = floorf(ux), fly = floorf(uy);
  sp.tx = fminf(fmaxf(ux - flx, 0.f), 1.f);
  sp.ty = fminf(fmaxf(uy - fly, 0.f), 1.f);
  int ix = (int)flx, iy = (int)fly;
  if (ix >= g.nx) ix -= g.nx;
  if (iy >= g.ny) iy -= g.ny;
  sp.ix = min(max(ix, 0), g.nx - 1);
  sp.iy = min(max(iy, 0), g.ny - 1);
  if (act && uz < 0.f) flags |= GRIDFF_REP_BELOW;
  uz = fmaxf(uz, 0.f);
  sp.inside = act && (uz < (float)(g.nz - 1));
  float flz = floorf(sp.inside ? uz : 0.f);
  sp.tz = (sp.inside ? uz : 0.f) - flz;
  sp.iz = min(max((int)flz, 0), g.nz - 2);
  return sp;
}

template <int NB>
__device__ __forceinline__ void rigid_forces_staged(const GridView& g, const TemplateView& tv, int ab, int n,
                                                    int lane, const float c[3], const float Rm[9], float Ft[3],
                                                    float tq[3], double& e, int& flags, float4* sbuf) {
  const int quad = lane >> 2, q = lane & 3;
  const int R = (n + kQuads - 1) / kQuads;
  for (int a = 0; a < 3; ++a) Ft[a] = tq[a] = 0.f;
  e = 0.0;
  auto atom = [&](int k, float4& b, float4& par, float p[3]) {
    const int i = k * kQuads + quad;
    const bool act = i < n;
    b = make_float4(0.f, 0.f, 0.f, 0.f);
    par = b;
    if (act) {
      b = __ldg(&tv.body[ab + i]);
      par = __ldg(&tv.par[ab + i]);
    }
    p[0] = Rm[0] * b.x + Rm[1] * b.y + Rm[2] * b.z + c[0];
    p[1] = Rm[3] * b.x + Rm[4] * b.y + Rm[5] * b.z + c[1];
    p[2] = Rm[6] * b.x + Rm[7] * b.y + Rm[8] * b.z + c[2];
    return act;
  };
  auto issue = [&](int k) {
    if (k < R) {
      float4 b, par;
      float p[3];
      int dummy = 0;
      bool act = atom(k, b, par, p);
      StencilPos sp = locate(g, act, p[0], p[1], p[2], dummy);
      if (sp.inside) {
        const float4* p0 = g.rec + ((long long)sp.ix * g.nyp + sp.iy) * g.nzp + sp.iz + q;
        float4* dst = sbuf + (k % NB) * 512 + lane;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) cp_async16(dst + (a * 4 + bb) * 32, p0 + a * g.sx + bb * g.nzp);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < NB; ++k) issue(k);
  for (int k = 0; k < R; ++k) {
    cp_async_wait<NB - 1>();
    float4 b, par;
    float p[3];
    bool act = atom(k, b, par, p);
    StencilPos sp = locate(g, act, p[0], p[1], p[2], flags);
    float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
    bspline_weights(sp.tx, wx, dwx);
    bspline_weights(sp.ty, wy, dwy);
    bspline_weights(sp.tz, wz, dwz);
    float S0 = 0.f, Sx = 0.f, Sy = 0.f;
    if (sp.inside) {
      const float4* src = sbuf + (k % NB) * 512 + lane;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        float s = 0.f, sy = 0.f;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          float4 r = src[(a * 4 + bb) * 32];
          float cc = fmaf(par.x, r.x, fmaf(par.y, r.y, par.z * r.z));
          s = fmaf(wy[bb], cc, s);
          sy = fmaf(dwy[bb], cc, sy);
        }
        S0 = fmaf(wx[a], s, S0);
        Sx = fmaf(dwx[a], s, Sx);
        Sy = fmaf(wx[a], sy, Sy);
      }
    }
    issue(k + NB);
    const float wq = q == 0 ? wz[0] : q == 1 ? wz[1] : q == 2 ? wz[2] : wz[3];
    const float dwq = q == 0 ? dwz[0] : q == 1 ? dwz[1] : q == 2 ? dwz[2] : dwz[3];
    float ei = qsum(wq * S0);
    float fx = -qsum(wq * Sx) * g.inv_dx;
    float fy = -qsum(wq * Sy) * g.inv_dy;
    float fz = -qsum(dwq * S0) * g.inv_dz;
    if (act && q == 0) {
      e += (double)ei;
      Ft[0] += fx;
      Ft[1] += fy;
      Ft[2] += fz;
      float gx = Rm[0] * fx + Rm[3] * fy + Rm[6] * fz;
      float gy = Rm[1] * fx + Rm[4] * fy + Rm[7] * fz;
      float gz = Rm[2] * fx + Rm[5] * fy + Rm[8] * fz;
      tq[0] += b.y * gz - b.z * gy;
      tq[1] += b.z * gx - b.x * gz;
      tq[2] += b.x * gy - b.y * gx;
    }
  }
  cp_async_wait<0>();
  for (int a = 0; a < 3; ++a) {
    Ft[a] = wsum(Ft[a]);
    tq[a] = wsum(tq[a]);
  }
  e = wsum(e);
}

// ---------------------------------------------------------------------------
// evaluation (no update)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
eval_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl,
            const int* __restrict__ rep_off, int n_rep, int rigid, const float* __restrict__ xs,
            int use_grid, int use_intra, double* __restrict__ E_out, float* __restrict__ F_out,
            float* __restrict__ Ea_out, int* __restrict__ st_out) {
  __shared__ WarpState s_all[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpState& s = s_all[wib];
  const int warp = blockIdx.x * kWarpsPerBlock + wib;
  const int n_warps = gridDim.x * kWarpsPerBlock;
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    __syncwarp();
    if (rigid) {
      const float* p = xs + 7 * (size_t)r;
      float Rm[9];
      quat_rot(p[3], p[4], p[5], p[6], Rm);
      for (int i = lane; i < n; i += 32) {
        float4 b = tv.body[ab + i];
        s.x[3 * i] = Rm[0] * b.x + Rm[1] * b.y + Rm[2] * b.z + p[0];
        s.x[3 * i + 1] = Rm[3] * b.x + Rm[4] * b.y + Rm[5] * b.z + p[1];
        s.x[3 * i + 2] = Rm[6] * b.x + Rm[7] * b.y + Rm[8] * b.z + p[2];
      }
    } else {
      for (int k = lane; k < 3 * n; k += 32) s.x[k] = xs[3 * (size_t)off + k];
    }
    int flags = 0;
    double E = flex_forces(g, use_grid, use_intra && !rigid, tv, ab, n, lane, s, flags);
    for (int i = lane; i < n; i += 32) {
      float* f = F_out + 3 * ((size_t)off + i);
      f[0] = s.f[3 * i];
      f[1] = s.f[3 * i + 1];
      f[2] = s.f[3 * i + 2];
      if (Ea_out) Ea_out[off + i] = s.eg[i];
      if (!finite3(f[0], f[1], f[2])) flags |= GRIDFF_REP_NONFINITE;
    }
    E = wsum(E);
    flags = __reduce_or_sync(kFull, flags);
    if (!isfinite(E)) flags |= GRIDFF_REP_NONFINITE;
    if (lane == 0) {
      E_out[r] = E;
      if (st_out) st_out[r] = flags;
    }
  }
}

// ---------------------------------------------------------------------------
// FIRE, rigid replicas
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
relax_rigid_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl, int n_rep,
                   float* pose, float* vel, float* fdt, float* falpha, int* fnp, int* status,
                   int* steps, double* energy, int nsteps, FireP fp, Control ctl, int use_grid) {
#if GRIDFF_STAGED_NB > 0
  extern __shared__ float4 s_stage[];
#endif
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t];
    const float4 rig = tv.rigid[t];
    const float rmax = tv.rmax[t];
    float c[3], q[4], v[3], w[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = pose[7 * (size_t)r + a];
      v[a] = vel[6 * (size_t)r + a];
      w[a] = vel[6 * (size_t)r + 3 + a];
    }
    for (int a = 0; a < 4; ++a) q[a] = pose[7 * (size_t)r + 3 + a];
    float dt = fdt[r], al = falpha[r];
    int np = fnp[r], st = status[r], evals = 0;
    double Elast = energy[r];
    for (int s = 0; s < nsteps; ++s) {
      if (st & (GRIDFF_REP_CONVERGED | GRIDFF_REP_NONFINITE)) break;
      if ((s & 31) == 0) {
        int sb = stop_bits(ctl, t0, lane);
        if (sb) {
          st |= sb;
          break;
        }
      }
      float Rm[9];
      quat_rot(q[0], q[1], q[2], q[3], Rm);
      float Ft[3], tq[3];
      double e = 0.0;
      int flags = 0;
      if (use_grid) {
#if GRIDFF_STAGED_NB > 0
        rigid_forces_staged<GRIDFF_STAGED_NB>(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags,
                                              s_stage + (threadIdx.x >> 5) * GRIDFF_STAGED_NB * 512);
#else
        rigid_forces(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags);
#endif
      } else {
        for (int a = 0; a < 3; ++a) Ft[a] = tq[a] = 0.f;
      }
      st |= __reduce_or_sync(kFull, flags);
      ++evals;
      Elast = e;
      if (!(finite3(Ft[0], Ft[1], Ft[2]) && finite3(tq[0], tq[1], tq[2]) && isfinite(e) &&
            finite3(c[0], c[1], c[2]))) {
        st |= GRIDFF_REP_NONFINITE;
        break;
      }
      float f2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2] + tq[0] * tq[0] + tq[1] * tq[1] +
                 tq[2] * tq[2];
      if (f2 < fp.f_conv2) {
        st |= GRIDFF_REP_CONVERGED;
        break;
      }
      // FIRE decision (identical in every lane: the sums are bitwise equal)
      float P = Ft[0] * v[0] + Ft[1] * v[1] + Ft[2] * v[2] + tq[0] * w[0] + tq[1] * w[1] + tq[2] * w[2];
      if (P > 0.f) {
        float fn = sqrtf(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
        float tn = sqrtf(tq[0] * tq[0] + tq[1] * tq[1] + tq[2] * tq[2]);
        float vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        float wn = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        float sf = fn > 0.f ? al * vn / fn : 0.f, sw = tn > 0.f ? al * wn / tn : 0.f;
        for (int a = 0; a < 3; ++a) {
          v[a] = (1.f - al) * v[a] + sf * Ft[a];
          w[a] = (1.f - al) * w[a] + sw * tq[a];
        }
        if (np > fp.n_min) {
          dt = fminf(dt * fp.f_inc, fp.dt_max);
          al *= fp.f_alpha;
        }
        ++np;
      } else {
        for (int a = 0; a < 3; ++a) v[a] = w[a] = 0.f;
        dt *= fp.f_dec;
        al = fp.alpha_start;
        np = 0;
      }
      const float aM = GRIDFF_ACC * dt / rig.x;
      v[0] += aM * Ft[0];
      v[1] += aM * Ft[1];
      v[2] += aM * Ft[2];
      w[0] += GRIDFF_ACC * dt * tq[0] / rig.y;
      w[1] += GRIDFF_ACC * dt * tq[1] / rig.z;
      w[2] += GRIDFF_ACC * dt * tq[2] / rig.w;
      float dr[3] = {v[0] * dt, v[1] * dt, v[2] * dt};
      float dn = sqrtf(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
      float sc = dn > fp.d_max ? fp.d_max / dn : 1.f;
      for (int a = 0; a < 3; ++a) c[a] += dr[a] * sc;
      float wn = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
      if (wn > 0.f) {
        float ang = fminf(wn * dt, fp.d_max / rmax);
        quat_advance(q, w[0] / wn, w[1] / wn, w[2] / wn, ang);
      }
    }
    if (lane == 0) {
      for (int a = 0; a < 3; ++a) {
        pose[7 * (size_t)r + a] = c[a];
        vel[6 * (size_t)r + a] = v[a];
        vel[6 * (size_t)r + 3 + a] = w[a];
      }
      for (int a = 0; a < 4; ++a) pose[7 * (size_t)r + 3 + a] = q[a];
      fdt[r] = dt;
      falpha[r] = al;
      fnp[r] = np;
      status[r] = st;
      int total = steps[r] + evals;
      steps[r] = total;
      energy[r] = Elast;
      report(ctl, n, evals, st, total);
    }
  }
}

// ---------------------------------------------------------------------------
// FIRE, flexible replicas
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
relax_flex_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl,
                  const int* __restrict__ rep_off, int n_rep, float* xs, float* vs, float* fdt,
                  float* falpha, int* fnp, int* status, int* steps, double* energy, int nsteps,
                  FireP fp, Control ctl, int use_grid, int use_intra) {
  __shared__ WarpState s_all[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpState& s = s_all[wib];
  const int warp = blockIdx.x * kWarpsPerBlock + wib;
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    __syncwarp();
    for (int k = lane; k < 3 * n; k += 32) {
      s.x[k] = xs[3 * (size_t)off + k];
      s.v[k] = vs[3 * (size_t)off + k];
    }
    float dt = fdt[r], al = falpha[r];
    int np = fnp[r], st = status[r], evals = 0;
    double Elast = energy[r];
    for (int it = 0; it < nsteps; ++it) {
      if (st & (GRIDFF_REP_CONVERGED | GRIDFF_REP_NONFINITE)) break;
      if ((it & 31) == 0) {
        int sb = stop_bits(ctl, t0, lane);
        if (sb) {
          st |= sb;
          break;
        }
      }
      int flags = 0;
      double e = flex_forces(g, use_grid, use_intra, tv, ab, n, lane, s, flags);
      float f2 = 0.f, P = 0.f, v2 = 0.f;
      for (int k = lane; k < 3 * n; k += 32) {
        float f = s.f[k], v = s.v[k];
        f2 = fmaf(f, f, f2);
        P = fmaf(f, v, P);
        v2 = fmaf(v, v, v2);
      }
      f2 = wsum(f2);
      P = wsum(P);
      v2 = wsum(v2);
      e = wsum(e);
      st |= __reduce_or_sync(kFull, flags);
      ++evals;
      Elast = e;
      if ((st & GRIDFF_REP_NONFINITE) || !isfinite(f2) || !isfinite(e)) {
        st |= GRIDFF_REP_NONFINITE;
        break;
      }
      if (f2 < fp.f_conv2) {
        st |= GRIDFF_REP_CONVERGED;
        break;
      }
      // FIRE decision (identical in every lane: the sums are bitwise equal)
      float keep, mixf;
      if (P > 0.f) {
        keep = 1.f - al;
        mixf = f2 > 0.f ? al * sqrtf(v2 / f2) : 0.f;
        if (np > fp.n_min) {
          dt = fminf(dt * fp.f_inc, fp.dt_max);
          al *= fp.f_alpha;
        }
        ++np;
      } else {
        keep = 0.f;
        mixf = 0.f;
        dt *= fp.f_dec;
        al = fp.alpha_start;
        np = 0;
      }
      for (int i = lane; i < n; i += 32) {
        const float im = 1.f / __ldg(&tv.body[ab + i]).w;
        float d[3];
        for (int a = 0; a < 3; ++a) {
          float f = s.f[3 * i + a];
          float vv = keep * s.v[3 * i + a] + mixf * f;
          vv += GRIDFF_ACC * f * im * dt;
          s.v[3 * i + a] = vv;
          d[a] = vv * dt;
        }
        float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        float sc = dn > fp.d_max ? fp.d_max / dn : 1.f;
        for (int a = 0; a < 3; ++a) s.x[3 * i + a] += d[a] * sc;
      }
    }
    __syncwarp();
    for (int k = lane; k < 3 * n; k += 32) {
      xs[3 * (size_t)off + k] = s.x[k];
      vs[3 * (size_t)off + k] = s.v[k];
    }
    if (lane == 0) {
      fdt[r] = dt;
      falpha[r] = al;
      fnp[r] = np;
      status[r] = st;
      int total = steps[r] + evals;
      steps[r] = total;
      energy[r] = Elast;
      report(ctl, n, evals, st, total);
    }
  }
}

// ---------------------------------------------------------------------------
// NVE, flexible replicas: velocity Verlet
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
run_flex_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl,
                const int* __restrict__ rep_off, int n_rep, float* xs, float* vs, int* status,
                double* energy, int nsteps, float dt, int rec_every, double* trace, Control ctl,
                int use_grid, int use_intra) {
  __shared__ WarpState s_all[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpState& s = s_all[wib];
  const int warp = blockIdx.x * kWarpsPerBlock + wib;
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    __syncwarp();
    for (int k = lane; k < 3 * n; k += 32) {
      s.x[k] = xs[3 * (size_t)off + k];
      s.v[k] = vs[3 * (size_t)off + k];
    }
    int st = status[r] & ~(GRIDFF_REP_ABORTED | GRIDFF_REP_STEPLIMIT);
    int flags = 0, evals = 0;
    double e = flex_forces(g, use_grid, use_intra, tv, ab, n, lane, s, flags);
    auto total = [&](double epot_lane) {
      double ke = 0.0;
      for (int i = lane; i < n; i += 32) {
        double m = __ldg(&tv.body[ab + i]).w;
        double vx = s.v[3 * i], vy = s.v[3 * i + 1], vz = s.v[3 * i + 2];
        ke += 0.5 * m * (vx * vx + vy * vy + vz * vz);
      }
      return wsum(epot_lane) + wsum(ke) / (double)GRIDFF_ACC;
    };
    double Etot = total(e);
    if (trace && lane == 0) trace[r] = Etot;
    int rec = 1;
    for (int it = 0; it < nsteps; ++it) {
      if ((it & 31) == 0) {
        int sb = stop_bits(ctl, t0, lane);
        if (sb) {
          st |= sb;
          break;
        }
      }
      for (int i = lane; i < n; i += 32) {
        const float h = 0.5f * dt * GRIDFF_ACC / __ldg(&tv.body[ab + i]).w;
        for (int a = 0; a < 3; ++a) {
          float vv = s.v[3 * i + a] + h * s.f[3 * i + a];
          s.v[3 * i + a] = vv;
          s.x[3 * i + a] += dt * vv;
        }
      }
      e = flex_forces(g, use_grid, use_intra, tv, ab, n, lane, s, flags);
      ++evals;
      for (int i = lane; i < n; i += 32) {
        const float h = 0.5f * dt * GRIDFF_ACC / __ldg(&tv.body[ab + i]).w;
        for (int a = 0; a < 3; ++a) s.v[3 * i + a] += h * s.f[3 * i + a];
      }
      __syncwarp();
      if (rec_every > 0 && (it + 1) % rec_every == 0) {
        Etot = total(e);
        if (trace && lane == 0) trace[(size_t)rec * n_rep + r] = Etot;
        ++rec;
      }
    }
    __syncwarp();
    for (int k = lane; k < 3 * n; k += 32) {
      xs[3 * (size_t)off + k] = s.x[k];
      vs[3 * (size_t)off + k] = s.v[k];
    }
    st |= __reduce_or_sync(kFull, flags);
    e = wsum(e);
    if (lane == 0) {
      status[r] = st;
      energy[r] = e;
      report(ctl, n, evals, st & ~GRIDFF_REP_CONVERGED, evals);
    }
  }
}

// ---------------------------------------------------------------------------
// NVE, rigid replicas: NO_SQUISH splitting (free-rotor sub-rotations about
// body axes 3, 2, 1, 2, 3 between half kicks).  Conjugate quaternion
// momentum p = 2 S(q) (0, I w); body angular momentum L_k = (P_k q . p)/2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void perm(int k, const float u[4], float o[4]) {
  if (k == 1) {
    o[0] = -u[1]; o[1] = u[0]; o[2] = u[3]; o[3] = -u[2];
  } else if (k == 2) {
    o[0] = -u[2]; o[1] = -u[3]; o[2] = u[0]; o[3] = u[1];
  } else {
    o[0] = -u[3]; o[1] = u[2]; o[2] = -u[1]; o[3] = u[0];
  }
}

// p += h * 2 S(q) (0, tau_b)  (S(q) u = q (x) u)
__device__ __forceinline__ void kick_rot(float p[4], const float q[4], const float tb[3], float h) {
  float s = 2.f * h;
  p[0] += s * (-q[1] * tb[0] - q[2] * tb[1] - q[3] * tb[2]);
  p[1] += s * (q[0] * tb[0] - q[3] * tb[1] + q[2] * tb[2]);
  p[2] += s * (q[3] * tb[0] + q[0] * tb[1] - q[1] * tb[2]);
  p[3] += s * (-q[2] * tb[0] + q[1] * tb[1] + q[0] * tb[2]);
}

__device__ __forceinline__ void free_rot(int k, float h, float Ik, float q[4], float p[4]) {
  float Pq[4], Pp[4];
  perm(k, q, Pq);
  perm(k, p, Pp);
  float zeta = h * (p[0] * Pq[0] + p[1] * Pq[1] + p[2] * Pq[2] + p[3] * Pq[3]) / (4.f * Ik);
  float sz, cz;
  sincosf(zeta, &sz, &cz);
  for (int a = 0; a < 4; ++a) {
    q[a] = cz * q[a] + sz * Pq[a];
    p[a] = cz * p[a] + sz * Pp[a];
  }
}

__device__ __forceinline__ void body_L(const float q[4], const float p[4], float L[3]) {
  for (int k = 1; k <= 3; ++k) {
    float Pq[4];
    perm(k, q, Pq);
    L[k - 1] = 0.5f * (p[0] * Pq[0] + p[1] * Pq[1] + p[2] * Pq[2] + p[3] * Pq[3]);
  }
}

__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
run_rigid_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl, int n_rep,
                 float* pose, float* vel, int* status, double* energy, int nsteps, float dt,
                 int rec_every, double* trace, Control ctl) {
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t];
    const float4 rig = tv.rigid[t];
    const float I[3] = {rig.y, rig.z, rig.w};
    float c[3], q[4], v[3], p[4];
    for (int a = 0; a < 3; ++a) {
      c[a] = pose[7 * (size_t)r + a];
      v[a] = vel[6 * (size_t)r + a];
    }
    for (int a = 0; a < 4; ++a) q[a] = pose[7 * (size_t)r + 3 + a];
    {
      float L[3] = {I[0] * vel[6 * (size_t)r + 3], I[1] * vel[6 * (size_t)r + 4], I[2] * vel[6 * (size_t)r + 5]};
      p[0] = 2.f * (-q[1] * L[0] - q[2] * L[1] - q[3] * L[2]);
      p[1] = 2.f * (q[0] * L[0] - q[3] * L[1] + q[2] * L[2]);
      p[2] = 2.f * (q[3] * L[0] + q[0] * L[1] - q[1] * L[2]);
      p[3] = 2.f * (-q[2] * L[0] + q[1] * L[1] + q[0] * L[2]);
    }
    int st = status[r] & ~(GRIDFF_REP_ABORTED | GRIDFF_REP_STEPLIMIT);
    int flags = 0, evals = 0;
    float Ft[3], tq[3];
    double e;
    float Rm[9];
    quat_rot(q[0], q[1], q[2], q[3], Rm);
    rigid_forces(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags);
    auto total = [&](double epot) {
      float L[3];
      body_L(q, p, L);
      double ke = 0.5 * rig.x * (double)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      for (int a = 0; a < 3; ++a) ke += 0.5 * (double)L[a] * (double)L[a] / (double)I[a];
      return epot + ke / (double)GRIDFF_ACC;
    };
    if (trace && lane == 0) trace[r] = total(e);
    int rec = 1;
    for (int it = 0; it < nsteps; ++it) {
      if ((it & 31) == 0) {
        int sb = stop_bits(ctl, t0, lane);
        if (sb) {
          st |= sb;
          break;
        }
      }
      const float h = 0.5f * dt;
      for (int a = 0; a < 3; ++a) v[a] += h * GRIDFF_ACC * Ft[a] / rig.x;
      float tb[3] = {GRIDFF_ACC * tq[0], GRIDFF_ACC * tq[1], GRIDFF_ACC * tq[2]};
      kick_rot(p, q, tb, h);
      for (int a = 0; a < 3; ++a) c[a] += dt * v[a];
      free_rot(3, h, I[2], q, p);
      free_rot(2, h, I[1], q, p);
      free_rot(1, dt, I[0], q, p);
      free_rot(2, h, I[1], q, p);
      free_rot(3, h, I[2], q, p);
      quat_rot(q[0], q[1], q[2], q[3], Rm);
      rigid_forces(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags);
      ++evals;
      for (int a = 0; a < 3; ++a) v[a] += h * GRIDFF_ACC * Ft[a] / rig.x;
      float tb2[3] = {GRIDFF_ACC * tq[0], GRIDFF_ACC * tq[1], GRIDFF_ACC * tq[2]};
      kick_rot(p, q, tb2, h);
      if (rec_every > 0 && (it + 1) % rec_every == 0) {
        if (trace && lane == 0) trace[(size_t)rec * n_rep + r] = total(e);
        ++rec;
      }
    }
    st |= __reduce_or_sync(kFull, flags);
    if (lane == 0) {
      float L[3];
      body_L(q, p, L);
      for (int a = 0; a < 3; ++a) {
        pose[7 * (size_t)r + a] = c[a];
        vel[6 * (size_t)r + a] = v[a];
        vel[6 * (size_t)r + 3 + a] = L[a] / I[a];
      }
      for (int a = 0; a < 4; ++a) pose[7 * (size_t)r + 3 + a] = q[a];
      status[r] = st;
      energy[r] = e;
      report(ctl, n, evals, st & ~GRIDFF_REP_CONVERGED, evals);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Staging {
  gridff_ctx* ctx;
  void* ptr = nullptr;
  explicit Staging(gridff_ctx* c) : ctx(c) {}
  ~Staging() {
    if (ptr) cudaFreeAsync(ptr, ctx->stream);
  }
};

int persistent_blocks(gridff_ctx* ctx, const void* kernel, int n_rep, size_t dyn_smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, dyn_smem);
  if (per_sm < 1) per_sm = 1;
  int need = (n_rep + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int cap = per_sm * ctx->n_sm;
  return need < cap ? need : cap;
}

GridView empty_view() {
  GridView v{};
  v.nx = v.ny = v.nz = 4;
  return v;
}

gridff_status check_common(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int flags) {
  if (!ctx || !R) return set_err(ctx, GRIDFF_EINVAL, "null argument");
  if (R->ctx != ctx) return set_err(ctx, GRIDFF_EINVAL, "replicas belong to another context");
  if (!(flags & GRIDFF_NO_GRID) && !grid) return set_err(ctx, GRIDFF_EINVAL, "grid is NULL");
  if (grid && grid->ctx != ctx) return set_err(ctx, GRIDFF_EINVAL, "grid belongs to another context");
  return GRIDFF_OK;
}

gridff_status finish_launch(gridff_ctx* ctx, DevResult* hres) {
  GRIDFF_CUDA(ctx, cudaGetLastError());
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(hres, ctx->result_dev, sizeof(DevResult), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  float ms = 0.f;
  GRIDFF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  ctx->last_ms = ms;
  if (hres->stop_bits & GRIDFF_REP_ABORTED) return set_err(ctx, GRIDFF_EABORTED, "aborted by the host flag");
  if (hres->stop_bits & GRIDFF_REP_STEPLIMIT)
    return set_err(ctx, GRIDFF_ESTEPLIMIT, "clock budget exhausted");
  return GRIDFF_OK;
}

}  // namespace

extern "C" {

gridff_status gridff_eval(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int flags,
                          double* E_out, float* F_out, float* Ea_out, int32_t* st_out) {
  gridff_status st = check_common(ctx, grid, R, flags);
  if (st != GRIDFF_OK) return st;
  if (!E_out || !F_out) return set_err(ctx, GRIDFF_EINVAL, "E_out and F_out are required");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  bool dev = flags & GRIDFF_DEVICE_PTRS;
  size_t nE = R->n_rep * sizeof(double), nF = 3 * (size_t)R->n_atoms * sizeof(float),
         nA = (size_t)R->n_atoms * sizeof(float), nS = R->n_rep * sizeof(int);
  Staging stg(ctx);
  double* dE = E_out;
  float* dF = F_out;
  float* dA = Ea_out;
  int* dS = st_out;
  if (!dev) {
    GRIDFF_CUDA(ctx, cudaMallocAsync(&stg.ptr, nE + nF + nA + nS + 64, s));
    char* p = (char*)stg.ptr;
    dE = (double*)p;
    dF = (float*)(p + nE);
    dA = Ea_out ? (float*)(p + nE + nF) : nullptr;
    dS = st_out ? (int*)(p + nE + nF + nA) : nullptr;
  }
  GridView gv = grid ? grid->view() : empty_view();
  int blocks = persistent_blocks(ctx, (const void*)eval_kernel, R->n_rep);
  eval_kernel<<<blocks, kThreads, 0, s>>>(gv, R->tv, R->rep_tmpl, R->rep_off, R->n_rep, R->rigid, R->x,
                                          !(flags & GRIDFF_NO_GRID), !(flags & GRIDFF_NO_INTRA), dE, dF,
                                          dA, dS);
  GRIDFF_CUDA(ctx, cudaGetLastError());
  if (!dev) {
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(E_out, dE, nE, cudaMemcpyDeviceToHost, s));
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(F_out, dF, nF, cudaMemcpyDeviceToHost, s));
    if (Ea_out) GRIDFF_CUDA(ctx, cudaMemcpyAsync(Ea_out, dA, nA, cudaMemcpyDeviceToHost, s));
    if (st_out) GRIDFF_CUDA(ctx, cudaMemcpyAsync(st_out, dS, nS, cudaMemcpyDeviceToHost, s));
  }
  if (!(dev && (flags & GRIDFF_ASYNC))) GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

gridff_status gridff_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int32_t nsteps,
                           const gridff_fire_params* prm, int flags, gridff_relax_result* result) {
  gridff_status st = check_common(ctx, grid, R, flags);
  if (st != GRIDFF_OK) return st;
  if (nsteps < 0) return set_err(ctx, GRIDFF_EINVAL, "nsteps < 0");
  gridff_fire_params def;
  gridff_fire_params_default(&def);
  const gridff_fire_params& P = prm ? *prm : def;
  if (!(P.dt_start > 0) || !(P.dt_max > 0) || !(P.d_max > 0) || P.f_conv < 0)
    return set_err(ctx, GRIDFF_EINVAL, "bad FIRE parameters");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  if (!(flags & GRIDFF_CONTINUE)) {
    // reset FIRE scalars, status and counters (fill on the device)
    std::vector<float> dt(R->n_rep, P.dt_start), al(R->n_rep, P.alpha_start);
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(R->fire_dt, dt.data(), R->n_rep * sizeof(float), cudaMemcpyHostToDevice, s));
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(R->fire_alpha, al.data(), R->n_rep * sizeof(float), cudaMemcpyHostToDevice, s));
    GRIDFF_CUDA(ctx, cudaMemsetAsync(R->fire_nplus, 0, R->n_rep * sizeof(int), s));
    GRIDFF_CUDA(ctx, cudaMemsetAsync(R->status, 0, R->n_rep * sizeof(int), s));
    GRIDFF_CUDA(ctx, cudaMemsetAsync(R->steps, 0, R->n_rep * sizeof(int), s));
    GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  } else {
    // a continued relaxation clears only the stop bits of the previous call
    // (kept in the status words; converged/non-finite replicas stay frozen)
  }
  GRIDFF_CUDA(ctx, cudaMemsetAsync(ctx->result_dev, 0, sizeof(DevResult), s));
  FireP fp{P.dt_start, P.dt_max, P.f_inc, P.f_dec, P.alpha_start, P.f_alpha, P.d_max,
           P.f_conv * P.f_conv, P.n_min};
  Control ctl{ctx->ctrl_dev, (unsigned long long)(P.clock_budget_s > 0 ? P.clock_budget_s * 1e9 : 0),
              (DevResult*)ctx->result_dev};
  GridView gv = grid ? grid->view() : empty_view();
  int use_grid = !(flags & GRIDFF_NO_GRID), use_intra = !(flags & GRIDFF_NO_INTRA);
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
  if (R->rigid) {
    size_t dyn = (size_t)GRIDFF_STAGED_NB * 512 * sizeof(float4) * kWarpsPerBlock;
    if (dyn > 48 * 1024)
      GRIDFF_CUDA(ctx, cudaFuncSetAttribute(relax_rigid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int blocks = persistent_blocks(ctx, (const void*)relax_rigid_kernel, R->n_rep, dyn);
    relax_rigid_kernel<<<blocks, kThreads, dyn, s>>>(gv, R->tv, R->rep_tmpl, R->n_rep, R->x, R->v, R->fire_dt,
                                                   R->fire_alpha, R->fire_nplus, R->status, R->steps,
                                                   R->energy, nsteps, fp, ctl, use_grid);
  } else {
    int blocks = persistent_blocks(ctx, (const void*)relax_flex_kernel, R->n_rep);
    relax_flex_kernel<<<blocks, kThreads, 0, s>>>(gv, R->tv, R->rep_tmpl, R->rep_off, R->n_rep, R->x, R->v,
                                                  R->fire_dt, R->fire_alpha, R->fire_nplus, R->status,
                                                  R->steps, R->energy, nsteps, fp, ctl, use_grid, use_intra);
  }
  DevResult h{};
  gridff_status rs = finish_launch(ctx, &h);
  if (result) {
    result->atom_evals = (int64_t)h.atom_evals;
    result->n_converged = h.n_converged;
    result->max_steps = h.max_steps;
  }
  if (flags & GRIDFF_CONTINUE) {
    // nothing else: stop bits stay visible in the status words
  }
  return rs;
}

gridff_status gridff_run(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int32_t nsteps,
                         const gridff_md_params* prm, int flags, double* energy_trace) {
  gridff_status st = check_common(ctx, grid, R, flags);
  if (st != GRIDFF_OK) return st;
  if (!prm || !(prm->dt > 0) || nsteps < 0 || prm->record_every < 0)
    return set_err(ctx, GRIDFF_EINVAL, "bad MD parameters");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  int rec_every = prm->record_every;
  size_t n_rec = rec_every > 0 ? (size_t)(nsteps / rec_every) + 1 : 1;
  size_t tbytes = n_rec * R->n_rep * sizeof(double);
  Staging stg(ctx);
  double* dtrace = nullptr;
  bool dev = flags & GRIDFF_DEVICE_PTRS;
  if (energy_trace) {
    if (dev) {
      dtrace = energy_trace;
    } else {
      GRIDFF_CUDA(ctx, cudaMallocAsync(&stg.ptr, tbytes, s));
      dtrace = (double*)stg.ptr;
    }
  }
  GRIDFF_CUDA(ctx, cudaMemsetAsync(ctx->result_dev, 0, sizeof(DevResult), s));
  Control ctl{ctx->ctrl_dev, (unsigned long long)(prm->clock_budget_s > 0 ? prm->clock_budget_s * 1e9 : 0),
              (DevResult*)ctx->result_dev};
  GridView gv = grid ? grid->view() : empty_view();
  int use_grid = !(flags & GRIDFF_NO_GRID), use_intra = !(flags & GRIDFF_NO_INTRA);
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
  if (R->rigid) {
    if (!use_grid) return set_err(ctx, GRIDFF_EINVAL, "rigid replicas need the grid term");
    int blocks = persistent_blocks(ctx, (const void*)run_rigid_kernel, R->n_rep);
    run_rigid_kernel<<<blocks, kThreads, 0, s>>>(gv, R->tv, R->rep_tmpl, R->n_rep, R->x, R->v, R->status,
                                                 R->energy, nsteps, prm->dt, rec_every, dtrace, ctl);
  } else {
    int blocks = persistent_blocks(ctx, (const void*)run_flex_kernel, R->n_rep);
    run_flex_kernel<<<blocks, kThreads, 0, s>>>(gv, R->tv, R->rep_tmpl, R->rep_off, R->n_rep, R->x, R->v,
                                                R->status, R->energy, nsteps, prm->dt, rec_every, dtrace, ctl,
                                                use_grid, use_intra);
  }
  DevResult h{};
  gridff_status rs = finish_launch(ctx, &h);
  if (energy_trace && !dev) {
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(energy_trace, dtrace, tbytes, cudaMemcpyDeviceToHost, s));
    GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  }
  return rs;
}

}  // extern "C"
