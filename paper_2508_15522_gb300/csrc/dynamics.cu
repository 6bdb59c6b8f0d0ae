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

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "interp.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;
#ifndef GRIDFF_MIN_BLOCKS_PER_SM
#define GRIDFF_MIN_BLOCKS_PER_SM 4
#endif
constexpr int kMinBlocksPerSM = GRIDFF_MIN_BLOCKS_PER_SM;
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

// per-warp shared state of the unique-term relaxation: positions and forces
// only (velocities stay in global memory, read and written once per step,
// which leaves more of the SM's shared storage to the L1 cache)
struct WarpStateXF {
  float x[3 * kMaxA];
  float f[3 * kMaxA];
};
__device__ __forceinline__ void store_eg(WarpState& s, int i, float e) { s.eg[i] = e; }
__device__ __forceinline__ void store_eg(WarpStateXF&, int, float) {}

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

// Per-warp stencil cache in shared memory.  Slot i (i < S) holds, for the
// atom evaluated by a quad, the 64 node values c = Q b^C + P b^P + L b^L
// of its 4x4x4 stencil (combined with that atom's fixed factors) and the
// cell they belong to.  Between consecutive steps an atom usually stays in
// its cell, so the gather is served from shared memory; it goes to global
// memory only when the cell changes.  Layout: lane q of the quad holds the
// 16 values of node z+q-1 for the 16 (x, y) runs, as 4 float4; float4 j of
// lane q of slot i sits at index (j * S + i) * 4 + q, so a warp access to 8
// consecutive slots is contiguous (no bank conflicts).
struct StencilCache {
  float4* val;   // [4 * S * 4]
  int* key;      // [S] packed cell index, -1 = empty
  int S;
};

// Channel-combined values c = Q C + P P + L L of the 16 (x, y) runs at one
// z-node: records base + a sx + b nzp, run m = 4a + b, for the grid's record
// kind (channel scales folded into the atom's factors; the branch is
// uniform over the warp).
// KIND >= 0: the record kind is known at compile time (no other code is
// generated); KIND < 0: dispatch on g.kind.
template <int KIND = -1>
__device__ __forceinline__ void gather_runs(const GridView& g, long long base, float4 par, float cv[16]) {
  const float fc = par.x * g.sC, fp = par.y * g.sP, fl = par.z * g.sL;
  switch (KIND >= 0 ? KIND : g.kind) {
    case REC_F32x4: {
      const float4* p = (const float4*)g.rec + base;
      float4 r[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) r[m] = __ldg(p + (m >> 2) * g.sx + (m & 3) * g.nzp);
#pragma unroll
      for (int m = 0; m < 16; ++m) cv[m] = fmaf(fc, r[m].x, fmaf(fp, r[m].y, fl * r[m].z));
      break;
    }
    case REC_F32x2: {
      const float2* p = (const float2*)g.rec + base;
      float2 r[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) r[m] = __ldg(p + (m >> 2) * g.sx + (m & 3) * g.nzp);
#pragma unroll
      for (int m = 0; m < 16; ++m) cv[m] = fmaf(fp, r[m].x, fl * r[m].y);
      break;
    }
    case REC_F16x4:
    case REC_BF16x4: {
      const uint2* p = (const uint2*)g.rec + base;
      uint2 r[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) r[m] = __ldg(p + (m >> 2) * g.sx + (m & 3) * g.nzp);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        float2 a, b;
        if (g.kind == REC_F16x4) {
          a = __half22float2(*reinterpret_cast<const __half2*>(&r[m].x));
          b = __half22float2(*reinterpret_cast<const __half2*>(&r[m].y));
        } else {
          a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r[m].x));
          b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r[m].y));
        }
        cv[m] = fmaf(fc, a.x, fmaf(fp, a.y, fl * b.x));
      }
      break;
    }
    default: {   // REC_F16x2, REC_BF16x2
      const unsigned* p = (const unsigned*)g.rec + base;
      unsigned r[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) r[m] = __ldg(p + (m >> 2) * g.sx + (m & 3) * g.nzp);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float2 a = g.kind == REC_F16x2 ? __half22float2(*reinterpret_cast<const __half2*>(&r[m]))
                                             : __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r[m]));
        cv[m] = fmaf(fp, a.x, fl * a.y);
      }
      break;
    }
  }
}

// Energy and force of one atom in the substrate field (Eqs. E, E_Coulomb,
// E_Morse), evaluated by the 4 lanes of a quad (q = lane & 3); every lane of
// the quad returns the full result.  Lane q gathers record q of each of
// the 16 z-runs (one warp load fetches 8 whole 64-byte runs), combines the
// channels with the atom's factors (Q, P, L), accumulates the x/y-weighted
// sums for node z+q-1, applies its own z weight, and the quad sums.  The
// force is minus the analytic gradient of the interpolant (Sec. 5).
// `act` false: the quad has no atom (it still takes part in the shuffles).
// `slot` >= 0: the atom may use stencil-cache slot `slot`.
// kPartial: return this lane's share (the 4 shares of a quad sum to the
// atom's value) instead of the quad sum.
template <bool kPartial = false, int KIND = -1>
__device__ __forceinline__ void grid_quad(const GridView& g, int q, bool act, float x, float y, float z,
                                          float4 par, float& e, float& fx, float& fy, float& fz, int& flags,
                                          const StencilCache& sc, int slot) {
  const Cell cl = locate(g, act, x, y, z, flags);
  float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
  bspline_weights(cl.tx, wx, dwx);
  bspline_weights(cl.ty, wy, dwy);
  bspline_weights(cl.tz, wz, dwz);
  float cv[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) cv[j] = 0.f;
  if (cl.inside) {
    const int key = (cl.ix * g.ny + cl.iy) * g.nz + cl.iz;
    const bool cached = slot >= 0 && slot < sc.S;
    if (cached && sc.key[slot] == key) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float4 v = sc.val[(j * sc.S + slot) * 4 + q];
        cv[4 * j] = v.x;
        cv[4 * j + 1] = v.y;
        cv[4 * j + 2] = v.z;
        cv[4 * j + 3] = v.w;
      }
    } else {
      gather_runs<KIND>(g, ((long long)cl.ix * g.nyp + cl.iy) * g.nzp + cl.iz + q, par, cv);
      if (cached) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          sc.val[(j * sc.S + slot) * 4 + q] = make_float4(cv[4 * j], cv[4 * j + 1], cv[4 * j + 2], cv[4 * j + 3]);
        if (q == 0) sc.key[slot] = key;
      }
    }
  }
  float S0 = 0.f, Sx = 0.f, Sy = 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float s = 0.f, sy = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      s = fmaf(wy[b], cv[4 * a + b], s);
      sy = fmaf(dwy[b], cv[4 * a + b], sy);
    }
    S0 = fmaf(wx[a], s, S0);
    Sx = fmaf(dwx[a], s, Sx);
    Sy = fmaf(wx[a], sy, Sy);
  }
  const float wq = q == 0 ? wz[0] : q == 1 ? wz[1] : q == 2 ? wz[2] : wz[3];
  const float dwq = q == 0 ? dwz[0] : q == 1 ? dwz[1] : q == 2 ? dwz[2] : dwz[3];
  e = wq * S0;
  fx = -wq * Sx * g.inv_dx;
  fy = -wq * Sy * g.inv_dy;
  fz = -dwq * S0 * g.inv_dz;
  if (!kPartial) {
    e = qsum(e);
    fx = qsum(fx);
    fy = qsum(fy);
    fz = qsum(fz);
  }
}

// Bytes of one warp's cache with S slots (a multiple of 16).
__host__ __device__ constexpr size_t cache_bytes(int S) { return (size_t)S * 256 + (((size_t)S * 4 + 15) & ~size_t(15)); }

// Bytes of one replica's share in the sub-warp kernels: its stencil cache
// and the cells its lanes publish for the refill queue (int2 per slot).
__host__ __device__ constexpr size_t sw_cache_bytes(int S) { return cache_bytes(S) + (((size_t)S * 8 + 15) & ~size_t(15)); }

// Bytes of one warp's dynamic shared memory in the unique-term flexible
// kernel: its stencil cache and the staged nonbonded parameters.
__host__ __device__ constexpr size_t flex_terms_warp_bytes(int S) { return cache_bytes(S) + (size_t)kMaxA * 16; }

__device__ __forceinline__ StencilCache warp_cache(unsigned char* dyn, int S, int wib) {
  StencilCache sc;
  unsigned char* base = dyn + (size_t)wib * cache_bytes(S);
  sc.val = (float4*)base;
  sc.key = (int*)(base + (size_t)S * 256);
  sc.S = S;
  return sc;
}

// Empty every slot of this warp's cache (at the start of a replica).
__device__ __forceinline__ void cache_reset(const StencilCache& sc, int lane) {
  for (int i = lane; i < sc.S; i += 32) sc.key[i] = -1;
  __syncwarp();
}

__device__ __forceinline__ float3 ld3(const float* s, int i) {
  return make_float3(s[3 * i], s[3 * i + 1], s[3 * i + 2]);
}
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// cos(n phi) and sin(n phi) from cos phi and sin phi by n rotations in the
// complex plane (exact trigonometry, no angle): (c, s) <- (c, s) e^{i phi}.
__device__ __forceinline__ void multiple_angle(float cphi, float sphi, int n, float& cn, float& sn) {
  cn = 1.f;
  sn = 0.f;
  for (int k = 0; k < n; ++k) {
    const float c2 = fmaf(cn, cphi, -sn * sphi);
    sn = fmaf(sn, cphi, cn * sphi);
    cn = c2;
  }
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
    float sn, cn;
    multiple_angle(cphi, sphi, T.n, cn, sn);
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

// q <- q (x) (cos(a/2), sin(a/2) u), normalised.
__device__ __forceinline__ void quat_advance(float q[4], float ux, float uy, float uz, float ang) {
  float s, c;
  const float h = 0.5f * ang;
  if (fabsf(h) < 0.05f) {
    // Taylor series of sin and cos to h^5 and h^6: truncation below
    // h^7 / 5040 < 2e-13 (relative 4e-12) for |h| < 0.05
    const float h2 = h * h;
    s = h * (1.f - h2 * (1.f / 6.f) * (1.f - h2 * (1.f / 20.f)));
    c = 1.f - h2 * 0.5f * (1.f - h2 * (1.f / 12.f) * (1.f - h2 * (1.f / 30.f)));
  } else {
    sincosf(h, &s, &c);
  }
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

// Record of a replica's final evaluation (the one after which a relaxation
// makes no further move: its last iteration, convergence, or a non-finite
// value): rigid: pose (7) into last_x[7 r..], total force (lab frame) and
// body-frame torque into last_f[6 r..]; flexible: positions and forces of
// its atoms (rows off..off+n-1 of last_x, last_f).  One lane (rigid) or the
// warp (flexible) writes it, once per replica and call.
__device__ __forceinline__ void record_rigid(float* last_x, float* last_f, int r, const float c[3], const float q[4],
                                             const float Ft[3], const float tq[3]) {
  float* px = last_x + 7 * (size_t)r;
  float* pf = last_f + 6 * (size_t)r;
  for (int a = 0; a < 3; ++a) {
    px[a] = c[a];
    pf[a] = Ft[a];
    pf[3 + a] = tq[a];
  }
  for (int a = 0; a < 4; ++a) px[3 + a] = q[a];
}
__device__ __forceinline__ void record_flex(float* last_x, float* last_f, int off, int n, int lane, const float* sx,
                                            const float* sf) {
  for (int m = lane; m < 3 * n; m += 32) {
    last_x[3 * (size_t)off + m] = sx[m];
    last_f[3 * (size_t)off + m] = sf[m];
  }
}

// Forces of one flexible replica whose positions are in s.x: grid term
// (quads over atoms) + intramolecular terms; writes s.f and s.eg and
// returns this lane's share of the energy (the caller sums the warp),
// accumulated in Acc.
template <class Acc = double>
__device__ __forceinline__ Acc flex_forces(const GridView& g, bool use_grid, bool use_intra,
                                           const TemplateView& tv, int ab, int n, int lane, WarpState& s,
                                           int& flags, const StencilCache& sc) {
  __syncwarp();
  const int quad = lane >> 2, q = lane & 3;
  Acc e = Acc(0);
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
    if (use_grid) grid_quad(g, q, act, x, y, z, par, eg, fx, fy, fz, flags, sc, i);
    float ix = 0.f, iy = 0.f, iz = 0.f, ie = 0.f;
    if (use_intra && act) intra_quad(tv, ab, n, i, q, s.x, ix, iy, iz, ie);
    ix = qsum(ix);
    iy = qsum(iy);
    iz = qsum(iz);
    e += (Acc)ie;
    if (act && q == 0) {
      s.f[3 * i] = fx + ix;
      s.f[3 * i + 1] = fy + iy;
      s.f[3 * i + 2] = fz + iz;
      s.eg[i] = eg;
      e += (Acc)eg;
    }
  }
  __syncwarp();
  return e;
}

// Intramolecular forces of one flexible replica, each term evaluated once:
// the lanes split the terms and add every term's forces to its atoms in
// s_f (nonbonded pairs in the registers of the atoms' owner lanes, the
// reactions passed by shuffles; bonded terms with atomics).  Returns this
// lane's share of the energy.  Same terms as
// intra_quad (reduced UFF-like form; nonbonded on pairs more than two bonds
// apart), without the per-atom repetition.
__device__ __forceinline__ uint32_t pick4(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, int k) {
  return k == 0 ? w0 : k == 1 ? w1 : k == 2 ? w2 : w3;
}

// 2^x by the PTX instruction ex2.approx.ftz.f32 (relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kLog2e = 1.44269504088896341f;   // log2(e)

// Nonbonded force factor c (F_i = c d, d = x_i - x_j) and energy of one pair
// (Morse with mixed R_i + R_j and eps_i eps_j, plus Coulomb), from per-atom
// factors prepared once per replica: pi = {k_e q_i, a R_i, eps_i, -} for
// this lane's atom and pj = {q_j, a R_j, eps_j, -} for the partner, with
// a = alpha log2(e), so that e^{-alpha (r - R_i - R_j)} = 2^{a R_i + a R_j - a r}.
__device__ __forceinline__ void nb_pair(float3 d, float4 pi, float4 pj, float alpha, float a, float& c, float& e) {
  const float r2 = dot3(d, d);
  const float ir = rsqrtf(r2);
  const float r = r2 * ir;
  const float e1 = ex2_approx(fmaf(-a, r, pi.y + pj.y));
  const float ee = pi.z * pj.z;
  const float qr = pi.x * pj.x * ir;                      // k_e q_i q_j / r
  c = -(2.f * alpha * ee * e1 * (1.f - e1) - qr * ir) * ir;
  e = ee * e1 * (e1 - 2.f) + qr;
}

// f[3 i .. 3 i + 2] += (x, y, z) by atomic additions (f in shared memory).
__device__ __forceinline__ void sh_add3(float* f, int i, float x, float y, float z) {
  atomicAdd(f + 3 * i, x);
  atomicAdd(f + 3 * i + 1, y);
  atomicAdd(f + 3 * i + 2, z);
}

// Zero positions and nonbonded factors of the slots n .. (next multiple of
// 32) - 1, which the nonbonded pass reads for partners outside the molecule.
__device__ __forceinline__ void pad_pair_slots(float* s_x, float4* s_nb, int n, int lane) {
  for (int i = n + lane; i < ((n + 31) & ~31); i += 32) {
    s_x[3 * i] = s_x[3 * i + 1] = s_x[3 * i + 2] = 0.f;
    s_nb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Steps d = d0 .. d1 of one block pair of the nonbonded pass (below): the
// pair (this lane's atom, slot (lane + d) mod ring of the block at base) when
// bit d of act is set.  Slots from n to the next multiple of 32 hold zero
// positions and factors (written when the replica is loaded).  Adds the pair forces to fi and the energies to e;
// returns the reactions received on this lane's atom of the partner block.
template <bool DIAG>
__device__ __forceinline__ float3 nb_steps(const float* s_x, const float4* s_nb, float3 xi, float4 pi, float alpha,
                                           float a, uint32_t act, int lane, int base, int ring, int d0, int d1,
                                           float3& fi, float& e) {
  float3 g = make_float3(0.f, 0.f, 0.f);
  int sl = lane + d0, src = lane - d0;
  if (sl >= ring) sl -= ring;
  if (src < 0) src += ring;
#pragma unroll 2
  for (int d = d0; d <= d1; ++d) {
    const bool on = (act >> d) & 1u;
    const int j = base + sl;
    const float3 dv = sub3(xi, ld3(s_x, j));
    float c, ep;
    nb_pair(dv, pi, s_nb[j], alpha, a, c, ep);
    c = on ? c : 0.f;                      // slots past n hold zeros: dv stays finite
    const float cx = c * dv.x, cy = c * dv.y, cz = c * dv.z;
    e += on ? ep : 0.f;
    fi.x += cx;
    fi.y += cy;
    fi.z += cz;
    g.x -= __shfl_sync(kFull, cx, src);
    g.y -= __shfl_sync(kFull, cy, src);
    g.z -= __shfl_sync(kFull, cz, src);
    if (DIAG) {
      sl = sl + 1 == ring ? 0 : sl + 1;
      src = src == 0 ? ring - 1 : src - 1;
    } else {
      sl = (sl + 1) & 31;
      src = (src - 1) & 31;
    }
  }
  return g;
}

__device__ float intra_terms(const TemplateView& tv, int t, int lane, const float* s_x, float* s_f,
                             const float4* s_nb) {
  float e = 0.f;
  const float alpha = tv.alpha;
  const int n = tv.natoms[t], ab = tv.atom_off[t];
  // Nonbonded pairs, by blocks of 32 atoms: lane l owns atom 32 I + l of
  // every block I and keeps its force in registers.  Block pair I < J: the
  // pairs (32 I + l, 32 J + (l + d) mod 32), d = 0 .. 31, cover I x J once;
  // within a block of m atoms the pairs (l, (l + d) mod m), d = 1 .. m/2 (at
  // d = m/2 for even m only from l < m/2), cover it once.  At a given d the
  // partners of the lanes are distinct and the partner's owner receives the
  // reaction from lane (l - d) mod ring by a shuffle, so no lane writes
  // another lane's atom and the pass needs no synchronisation; s_f is
  // updated by the owners once per block pair.  Which steps d carry a pair
  // (partner inside the molecule, not excluded, counted from this atom) is
  // one 32-bit word per lane and block pair, computed before the steps.
  // Inactive steps read the partner's slot of s_x / s_nb (a real atom, or a
  // zeroed slot below the next multiple of 32) and add zero.
  const float a2 = alpha * kLog2e;
  const int nblk = (n + 31) >> 5;
  for (int I = 0; I < nblk; ++I) {
    const int i = 32 * I + lane;
    const bool own = i < n;
    const int ii = own ? i : 32 * I;
    const float3 xi = ld3(s_x, ii);
    float4 pi = s_nb[ii];
    pi.x *= GRIDFF_KE;
    const uint32_t* ex = tv.excl + 4 * (size_t)(ab + ii);
    float3 fi = make_float3(0.f, 0.f, 0.f);
    for (int J = I; J < nblk; ++J) {
      const int base = 32 * J, m = min(32, n - base);
      const bool diag = J == I;
      const int ring = diag ? m : 32;
      // partner slots with a pair, then bit d = slot (lane + d) mod ring
      const uint32_t ok = (m >= 32 ? 0xffffffffu : ((1u << m) - 1u)) & ~__ldg(&ex[J]);
      const unsigned long long dbl = (unsigned long long)ok | ((unsigned long long)ok << ring);
      uint32_t act = own ? (uint32_t)(dbl >> lane) : 0u;
      float3 gj;
      if (diag) {
        const int h = m >> 1;
        act &= ((2u << h) - 1u) & ~1u;                          // d = 1 .. m/2
        if (!(m & 1) && lane >= h) act &= ~(1u << h);           // d = m/2 counted from l < m/2
        gj = nb_steps<true>(s_x, s_nb, xi, pi, alpha, a2, act, lane, base, ring, 1, h, fi, e);
        fi.x += gj.x;
        fi.y += gj.y;
        fi.z += gj.z;
      } else {
        gj = nb_steps<false>(s_x, s_nb, xi, pi, alpha, a2, act, lane, base, 32, 0, 31, fi, e);
        if (base + lane < n) {
          float* f = s_f + 3 * (base + lane);
          f[0] += gj.x;
          f[1] += gj.y;
          f[2] += gj.z;
        }
      }
    }
    if (own) {
      s_f[3 * i] += fi.x;
      s_f[3 * i + 1] += fi.y;
      s_f[3 * i + 2] += fi.z;
    }
  }
  __syncwarp();
  // Bonded terms (few per atom): lanes take terms round-robin and add the
  // forces with shared-memory atomics.  Reciprocals come from rsqrtf
  // (1/x = rsqrt(x)^2), not from divisions.
  for (int b = tv.ub_off[t] + lane; b < tv.ub_off[t + 1]; b += 32) {
    const BondTerm B = tv.ub[b];
    const float3 d = sub3(ld3(s_x, B.i), ld3(s_x, B.j));
    const float r2 = dot3(d, d);
    const float ir = r2 > 0.f ? rsqrtf(r2) : 0.f;   // zero length: no direction, no force
    const float dr = r2 * ir - B.r0;
    const float c = -2.f * B.k * dr * ir;
    sh_add3(s_f, B.i, c * d.x, c * d.y, c * d.z);
    sh_add3(s_f, B.j, -c * d.x, -c * d.y, -c * d.z);
    e += B.k * dr * dr;
  }
  for (int a = tv.ua_off[t] + lane; a < tv.ua_off[t + 1]; a += 32) {
    const AngleRec A = tv.ua[a];
    const float3 u = sub3(ld3(s_x, A.a), ld3(s_x, A.b)), w = sub3(ld3(s_x, A.c), ld3(s_x, A.b));
    const float ru = rsqrtf(dot3(u, u)), rw = rsqrtf(dot3(w, w));
    const float inv = ru * rw, iu2 = ru * ru, iw2 = rw * rw;
    const float c = dot3(u, w) * inv;
    const float dEdc = 2.f * A.k * (c - A.cos0);
    const float cu = c * iu2, cw = c * iw2;
    const float3 ga = make_float3(w.x * inv - cu * u.x, w.y * inv - cu * u.y, w.z * inv - cu * u.z);
    const float3 gc = make_float3(u.x * inv - cw * w.x, u.y * inv - cw * w.y, u.z * inv - cw * w.z);
    sh_add3(s_f, A.a, -dEdc * ga.x, -dEdc * ga.y, -dEdc * ga.z);
    sh_add3(s_f, A.c, -dEdc * gc.x, -dEdc * gc.y, -dEdc * gc.z);
    sh_add3(s_f, A.b, dEdc * (ga.x + gc.x), dEdc * (ga.y + gc.y), dEdc * (ga.z + gc.z));
    e += A.k * (c - A.cos0) * (c - A.cos0);
  }
  for (int k = tv.ut_off[t] + lane; k < tv.ut_off[t + 1]; k += 32) {
    const TorsionRec T = tv.ut[k];
    const float3 xa = ld3(s_x, T.a), xb = ld3(s_x, T.b), xc = ld3(s_x, T.c), xd = ld3(s_x, T.d);
    const float3 F = sub3(xa, xb), G = sub3(xb, xc), H = sub3(xd, xc);
    const float3 A = cross3(F, G), B = cross3(H, G);
    const float A2 = dot3(A, A), B2 = dot3(B, B), G2 = dot3(G, G);
    if (A2 < 1e-12f || B2 < 1e-12f || G2 < 1e-12f) continue;   // collinear: no torque
    const float rA = rsqrtf(A2), rB = rsqrtf(B2), rG = rsqrtf(G2);
    const float iA2 = rA * rA, iB2 = rB * rB, Gn = G2 * rG;
    const float iAB = rA * rB;
    const float cphi = dot3(A, B) * iAB;
    const float sphi = dot3(cross3(B, A), G) * iAB * rG;
    float sn, cn;
    multiple_angle(cphi, sphi, T.n, cn, sn);
    const float dEdphi = 0.5f * T.V * T.cn0 * T.n * sn;
    const float FG = dot3(F, G) * iA2 * rG, HG = dot3(H, G) * iB2 * rG;
    const float ca = -Gn * iA2, cd = Gn * iB2;
    const float a1 = -ca + FG, b1 = -cd + HG;
    // gradients of phi with respect to the four atoms, times -dE/dphi
    const float m0 = -dEdphi * ca, m3 = -dEdphi * cd, m1 = -dEdphi * a1, m2 = -dEdphi * b1;
    const float h1 = dEdphi * HG, h2 = dEdphi * FG;
    sh_add3(s_f, T.a, m0 * A.x, m0 * A.y, m0 * A.z);
    sh_add3(s_f, T.b, m1 * A.x + h1 * B.x, m1 * A.y + h1 * B.y, m1 * A.z + h1 * B.z);
    sh_add3(s_f, T.c, m2 * B.x + h2 * A.x, m2 * B.y + h2 * A.y, m2 * B.z + h2 * A.z);
    sh_add3(s_f, T.d, m3 * B.x, m3 * B.y, m3 * B.z);
    e += 0.5f * T.V * (1.f - T.cn0 * cn);
  }
  return e;
}

// Forces of one flexible replica (positions in s.x) with the grid term by
// quads (stored per atom) followed by the unique-term intramolecular pass
// (added with shared-memory atomics).  Writes s.f, s.eg; returns this
// lane's share of the energy.
template <class Acc = double, int KIND = -1, class St = WarpState>
__device__ __forceinline__ Acc flex_forces_terms(const GridView& g, bool use_grid, bool use_intra,
                                                 const TemplateView& tv, int t, int ab, int n, int lane,
                                                 St& s, int& flags, const StencilCache& sc,
                                                 const float4* s_nb) {
  __syncwarp();
  const int quad = lane >> 2, q = lane & 3;
  Acc e = Acc(0);
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
    if (use_grid) grid_quad<false, KIND>(g, q, act, x, y, z, par, eg, fx, fy, fz, flags, sc, i);
    if (act && q == 0) {
      s.f[3 * i] = fx;
      s.f[3 * i + 1] = fy;
      s.f[3 * i + 2] = fz;
      store_eg(s, i, eg);
      e += (Acc)eg;
    }
  }
  __syncwarp();
  if (use_intra) e += (Acc)intra_terms(tv, t, lane, s.x, s.f, s_nb);
  __syncwarp();
  return e;
}

// Grid forces of a rigid replica: total force (lab) and body-frame torque
// (warp-reduced), and this lane's share of the energy (not reduced),
// accumulated per atom in Acc (double for the NVE energy trace, float for
// relaxations, where only the final value is reported).  Force, torque and
// energy are linear in the per-atom forces, so each lane accumulates its
// quad share of every atom and the warp sums once per step.
template <class Acc>
__device__ __forceinline__ void rigid_forces(const GridView& g, const TemplateView& tv, int ab, int n, int lane,
                                             const float c[3], const float Rm[9], float Ft[3], float tq[3],
                                             Acc& e, int& flags, const StencilCache& sc) {
  const int quad = lane >> 2, q = lane & 3;
  __syncwarp();   // cache keys written by one lane of a quad in the previous step
  for (int a = 0; a < 3; ++a) Ft[a] = tq[a] = 0.f;
  e = Acc(0);
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
    grid_quad<true>(g, q, act, px, py, pz, par, ei, fx, fy, fz, flags, sc, i);   // this lane's share
    if (act) {
      e += (Acc)ei;
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
    const StencilCache nocache{nullptr, nullptr, 0};
    double E = flex_forces(g, use_grid, use_intra && !rigid, tv, ab, n, lane, s, flags, nocache);
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

// Grid interpolation alone at independent points (steps a2-a6 of the path:
// fold, cell, weights, gather, contraction, channel combination): a quad
// per point, 8 points per warp per round, grid-stride over the points.
#ifndef GRIDFF_POINTS_MINB
#define GRIDFF_POINTS_MINB 1
#endif
template <int KIND>
__global__ void __launch_bounds__(256, GRIDFF_POINTS_MINB)
eval_points_kernel(GridView g, long long n, const float* __restrict__ xyz, const float* __restrict__ qpl,
                   float* __restrict__ E, float* __restrict__ F, int* __restrict__ st) {
  const int lane = threadIdx.x & 31, quad = lane >> 2, q = lane & 3;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const StencilCache nocache{nullptr, nullptr, 0};
  for (long long b = warp * kQuads; b < n; b += n_warps * kQuads) {   // uniform over the warp
    const long long i = b + quad;
    const bool act = i < n;
    float x = 0.f, y = 0.f, z = 0.f;
    float4 par = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act) {
      x = __ldg(&xyz[3 * i]);
      y = __ldg(&xyz[3 * i + 1]);
      z = __ldg(&xyz[3 * i + 2]);
      par = make_float4(__ldg(&qpl[3 * i]), __ldg(&qpl[3 * i + 1]), __ldg(&qpl[3 * i + 2]), 0.f);
    }
    // a non-finite position is reported and evaluates to zero
    const bool fin = finite3(x, y, z);
    int flags = fin ? 0 : GRIDFF_REP_NONFINITE;
    float e, fx, fy, fz;
    grid_quad<false, KIND>(g, q, act && fin, x, y, z, par, e, fx, fy, fz, flags, nocache, -1);
    if (act && q == 0) {
      E[i] = e;
      F[3 * i] = fx;
      F[3 * i + 1] = fy;
      F[3 * i + 2] = fz;
      if (st) st[i] = flags | (finite3(fx, fy, fz) && isfinite(e) ? 0 : GRIDFF_REP_NONFINITE);
    }
  }
}

// ---------------------------------------------------------------------------
// FIRE, rigid replicas
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
relax_rigid_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl, int n_rep,
                   float* pose, float* vel, float* fdt, float* falpha, int* fnp, int* status,
                   int* steps, double* energy, float* last_x, float* last_f, int nsteps, FireP fp, Control ctl,
                   int use_grid, int S) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31;
  const StencilCache sc = warp_cache(dyn_smem, S, threadIdx.x >> 5);
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t];
    const float4 rig = tv.rigid[t];
    const float rmax = tv.rmax[t];
    cache_reset(sc, lane);
    float c[3], q[4], v[3], w[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = pose[7 * (size_t)r + a];
      v[a] = vel[6 * (size_t)r + a];
      w[a] = vel[6 * (size_t)r + 3 + a];
    }
    for (int a = 0; a < 4; ++a) q[a] = pose[7 * (size_t)r + 3 + a];
    float dt = fdt[r], al = falpha[r];
    int np = fnp[r], st = status[r], evals = 0;
    float elane = 0.f;          // this lane's share of the last evaluated energy
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
      float e = 0.f;
      int flags = 0;
      if (use_grid) {
        rigid_forces(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags, sc);
      } else {
        for (int a = 0; a < 3; ++a) Ft[a] = tq[a] = 0.f;
      }
      st |= __reduce_or_sync(kFull, flags);
      ++evals;
      elane = e;
      const bool fin = finite3(Ft[0], Ft[1], Ft[2]) && finite3(tq[0], tq[1], tq[2]) && finite3(c[0], c[1], c[2]);
      float f2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2] + tq[0] * tq[0] + tq[1] * tq[1] +
                 tq[2] * tq[2];
      if (lane == 0 && (s == nsteps - 1 || !fin || f2 < fp.f_conv2)) record_rigid(last_x, last_f, r, c, q, Ft, tq);
      if (!fin) {
        st |= GRIDFF_REP_NONFINITE;
        break;
      }
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
    const double Etot = evals > 0 ? wsum((double)elane) : energy[r];
    if (evals > 0 && !isfinite(Etot)) st |= GRIDFF_REP_NONFINITE;
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
      energy[r] = Etot;
      report(ctl, n, evals, st, total);
    }
  }
}

// ---------------------------------------------------------------------------
// FIRE, rigid replicas, sub-warp form: each replica is handled by W lanes
// (W = 8, 16 or 32; 32/W replicas per warp), one lane per atom.  Per step
// and per round of W atoms: the lane places its atom and finds its cell;
// atoms whose cell is not in the stencil cache are refilled cooperatively
// (their cells are published in shared memory and the quads of the
// sub-warp serve all misses of the step from one queue, gathering the 16
// z-runs, lane q taking record q of each run, and storing the channel-
// combined node values); then every lane
// contracts its own atom's 64 cached values (16 z passes, 4 y, 1 x) with
// no work repeated across lanes.  Cache layout of a replica (S >= atoms
// slots): the 16 (x, y) runs (a, b) form 8 pairs p = 2a + (b >> 1); float4
// 2p + h of atom i (index (2p + h) * S + i) holds z-nodes 2h and 2h + 1 of
// the pair's two runs interleaved, (A_2h, B_2h, A_2h+1, B_2h+1), so the
// contraction runs on paired FP32 FMAs.
// ---------------------------------------------------------------------------
// Grid forces of the replica served by this sub-warp at pose (c, Rm): every
// lane locates its R atoms, the stencils that changed cell are refilled by
// the quads, every lane contracts its atoms; returns the total force and the
// body-frame torque summed over the sub-warp, this lane's share of the
// energy (Acc: float for relaxations, double for NVE) and the BELOW flag.
template <int W, int R, int KIND, class Acc>
__device__ __forceinline__ void sw_forces(const GridView& g, const StencilCache& sc, float* cval, int2* pub,
                                          const float4* __restrict__ par, int S, int sw, int l, int n, bool run,
                                          const float c[3], const float Rm[9], const float4 (&bk)[R],
                                          const float4 (&pk)[R], float Ft[3], float tq[3], Acc& e, int& flags) {
  for (int a = 0; a < 3; ++a) Ft[a] = tq[a] = 0.f;
  e = Acc(0);
  // locate every atom of the lane
  Cell cl[R];
  int key[R];
  unsigned miss_mask[R];
  float3 arm[R];   // R(q) b_i: the atom's lab-frame offset from the centre of mass
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = k * W + l;
    const bool act = run && i < n;
    const float4 b = bk[k];
    arm[k] = make_float3(Rm[0] * b.x + Rm[1] * b.y + Rm[2] * b.z, Rm[3] * b.x + Rm[4] * b.y + Rm[5] * b.z,
                         Rm[6] * b.x + Rm[7] * b.y + Rm[8] * b.z);
    const float px = arm[k].x + c[0], py = arm[k].y + c[1], pz = arm[k].z + c[2];
    cl[k] = locate(g, act, px, py, pz, flags);
    key[k] = (cl[k].ix * g.ny + cl[k].iy) * g.nz + cl[k].iz;
    const bool miss = cl[k].inside && sc.key[i < S ? i : 0] != key[k];
    unsigned msub = __ballot_sync(kFull, miss);
    if constexpr (W < 32) msub = (msub >> (sw * W)) & ((1u << (W & 31)) - 1u);
    miss_mask[k] = msub;
  }
  // refill the stencils that changed cell.  Each lane publishes the cells
  // of its atoms that missed; the misses of all rounds k form one queue
  // (bit k W + l = atom index), served W/4 atoms at a time (one per quad)
  // with one copy of the gather code
#pragma unroll
  for (int k = 0; k < R; ++k)
    if ((miss_mask[k] >> l) & 1u) pub[k * W + l] = make_int2(cl[k].ix | (cl[k].iy << 16), cl[k].iz);
  __syncwarp();
  constexpr int kPerWord = 64 / W;   // rounds k whose miss bits share one 64-bit word
#pragma unroll
  for (int k0 = 0; k0 < R; k0 += kPerWord) {
    unsigned long long mm = 0;
#pragma unroll
    for (int k = k0; k < R && k < k0 + kPerWord; ++k) mm |= (unsigned long long)miss_mask[k] << ((k - k0) * W);
#pragma unroll 1
    while (__any_sync(kFull, mm != 0)) {
      const int qd = l >> 2, qq = l & 3;
      unsigned long long m = mm;
      for (int j = 0; j < qd && m; ++j) m &= m - 1;
      if (m) {
        const int slot = k0 * W + __ffsll((long long)m) - 1;
        const int2 pc = pub[slot];
        const int oix = (int)((unsigned)pc.x & 0xffffu), oiy = (int)((unsigned)pc.x >> 16), oiz = pc.y;
        float cv[16];
        gather_runs<KIND>(g, ((long long)oix * g.nyp + oiy) * g.nzp + oiz + qq, __ldg(&par[slot]), cv);
        // run mm = 4a + b, z-node qq goes to float4 2p + (qq >> 1) of
        // run pair p = 2a + (b >> 1), component 2 (qq & 1) + (b & 1)
#pragma unroll
        for (int r2 = 0; r2 < 16; ++r2) {
          const int a = r2 >> 2, bq = r2 & 3;
          const int f4 = 2 * (2 * a + (bq >> 1)) + (qq >> 1);
          cval[((size_t)f4 * S + slot) * 4 + 2 * (qq & 1) + (bq & 1)] = cv[r2];
        }
        if (qq == 0) sc.key[slot] = (oix * g.ny + oiy) * g.nz + oiz;
      }
      for (int j = 0; j < W / 4 && mm; ++j) mm &= mm - 1;
    }
  }
  __syncwarp();
  // contract every atom of the lane (independent chains, no branch between
  // them: an atom outside the grid or beyond n reads a valid slot and its
  // results are dropped by selection)
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = min(k * W + l, S - 1);
    const bool in = cl[k].inside;
    {
      float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
      bspline_weights(cl[k].tx, wx, dwx);
      bspline_weights(cl[k].ty, wy, dwy);
      bspline_weights(cl[k].tz, wz, dwz);
      // two (x, y) runs at a time with paired FP32 FMAs: the cache
      // holds run pairs interleaved, so (run A, run B) values of one
      // z-node form an operand pair
      float2 WZ[4], DZ[4];
#pragma unroll
      for (int cz = 0; cz < 4; ++cz) {
        WZ[cz] = make_float2(wz[cz], wz[cz]);
        DZ[cz] = make_float2(dwz[cz], dwz[cz]);
      }
      float ev = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        float2 yv = make_float2(0.f, 0.f), yy = yv, yz = yv;
#pragma unroll
        for (int pb = 0; pb < 2; ++pb) {
          const int pr = 2 * a + pb;
          const float4 F0 = sc.val[(2 * pr) * S + i], F1 = sc.val[(2 * pr + 1) * S + i];
          const float2 z0 = make_float2(F0.x, F0.y), z1 = make_float2(F0.z, F0.w);
          const float2 z2 = make_float2(F1.x, F1.y), z3 = make_float2(F1.z, F1.w);
          float2 zv = __fmul2_rn(WZ[3], z3), zd = __fmul2_rn(DZ[3], z3);
          zv = __ffma2_rn(WZ[2], z2, zv);
          zd = __ffma2_rn(DZ[2], z2, zd);
          zv = __ffma2_rn(WZ[1], z1, zv);
          zd = __ffma2_rn(DZ[1], z1, zd);
          zv = __ffma2_rn(WZ[0], z0, zv);
          zd = __ffma2_rn(DZ[0], z0, zd);
          const float2 WY = make_float2(wy[2 * pb], wy[2 * pb + 1]);
          const float2 DY = make_float2(dwy[2 * pb], dwy[2 * pb + 1]);
          yv = __ffma2_rn(WY, zv, yv);
          yy = __ffma2_rn(DY, zv, yy);
          yz = __ffma2_rn(WY, zd, yz);
        }
        const float sv = yv.x + yv.y, sy = yy.x + yy.y, sz = yz.x + yz.y;
        ev = fmaf(wx[a], sv, ev);
        gx = fmaf(dwx[a], sv, gx);
        gy = fmaf(wx[a], sy, gy);
        gz = fmaf(wx[a], sz, gz);
      }
      const float fx = in ? -gx * g.inv_dx : 0.f, fy = in ? -gy * g.inv_dy : 0.f, fz = in ? -gz * g.inv_dz : 0.f;
      e += in ? ev : 0.f;
      Ft[0] += fx;
      Ft[1] += fy;
      Ft[2] += fz;
      // lab-frame torque (R b) x f; turned into the body frame once per step
      const float3 a = arm[k];
      tq[0] += a.y * fz - a.z * fy;
      tq[1] += a.z * fx - a.x * fz;
      tq[2] += a.x * fy - a.y * fx;
    }
  }
  {
    // body-frame torque R^T tau_lab (linear: the per-lane partial sums
    // may be rotated before the sub-warp sum)
    const float t0 = tq[0], t1 = tq[1], t2 = tq[2];
    tq[0] = Rm[0] * t0 + Rm[3] * t1 + Rm[6] * t2;
    tq[1] = Rm[1] * t0 + Rm[4] * t1 + Rm[7] * t2;
    tq[2] = Rm[2] * t0 + Rm[5] * t1 + Rm[8] * t2;
  }
  // sums over the sub-warp (xor offsets below W stay inside it); the
  // only flag locate() raises is BELOW: one ballot instead of a sum
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Ft[a] += __shfl_xor_sync(kFull, Ft[a], o);
      tq[a] += __shfl_xor_sync(kFull, tq[a], o);
    }
  }
  {
    unsigned bb = __ballot_sync(kFull, (flags & GRIDFF_REP_BELOW) != 0);
    if constexpr (W < 32) bb = (bb >> (sw * W)) & ((1u << (W & 31)) - 1u);
    flags = bb ? GRIDFF_REP_BELOW : 0;
  }
}

// Time-sliced schedule of the sub-warp relaxation.  A warp task is the
// 32 / W replicas one warp relaxes together; all run the same iteration
// count, so when the tasks outnumber the resident warps by a non-integer
// factor, whole tasks per warp leave the last round partly idle (4096
// replicas on 1216 warps: 1.68 rounds take 2).  Instead the P x nsteps grid
// of (task, iteration) is cut into equal contiguous ranges, one per warp
// (McNaughton's wrap-around rule for preemptive scheduling).  A range starts
// inside task p0 and ends inside task p1; the warp runs first the head of p1
// (iterations from 0), then the whole tasks between, and last the tail of p0,
// whose head the previous warp ran first.  A task's two parts never overlap
// in time when every range holds at least nsteps iterations, which the
// 5/4 condition below guarantees with a margin of a quarter of a task.  The
// head's final state goes through global memory (the same arrays a call
// reads and writes) and a per-task flag; the tail's wait is bounded.
//
// Part j of warp `warp`'s work: task p (p < 0: no part j), iterations
// [it_b, it_e), and whether it is a head (hands its state on) or a tail
// (waits for the head).  Not inlined: the schedule is recomputed per part
// instead of holding registers through the relaxation loop.
struct SwPart {
  int p, it_b, it_e;
  int role;   // 0 whole task, 1 head, 2 tail
};

__device__ __noinline__ SwPart sw_part(int warp, int n_warps, int P, int nsteps, int j) {
  SwPart s{-1, 0, nsteps, 0};
  if (4LL * P < 5LL * n_warps || nsteps < 64) {
    const long long p = warp + (long long)j * n_warps;
    if (p < P) s.p = (int)p;
    return s;
  }
  const long long T = (long long)P * nsteps, D = (T + n_warps - 1) / n_warps;
  const long long rb = min(T, (long long)warp * D), re = min(T, rb + D);
  if (rb >= re) return s;
  const int p_tail = (int)(rb / nsteps), it_tail = (int)(rb % nsteps);
  const int p_head = (int)(re / nsteps), it_head = (int)(re % nsteps);
  const int has_head = it_head > 0, has_tail = it_tail > 0;
  const int p_first = has_tail ? p_tail + 1 : p_tail;
  const int n_parts = has_head + (p_head - p_first) + has_tail;
  if (j >= n_parts) return s;
  if (has_head && j == 0) {
    s.p = p_head;
    s.it_e = it_head;
    s.role = 1;
  } else if (has_tail && j == n_parts - 1) {
    s.p = p_tail;
    s.it_b = it_tail;
    s.role = 2;
  } else {
    s.p = p_first + j - has_head;
  }
  return s;
}

// Bound of the wait for a hand-off flag: one second of %globaltimer time,
// after which the part is skipped and the call returns GRIDFF_ETIMEOUT.
// The poll count is only a backstop that ends the loop should the timer
// not advance (polls are about a microsecond apart: an acquire load from
// L2 and a requested 1 us sleep).  A head finishes a quarter of a task
// before its tail starts, so a working launch never waits long.
constexpr unsigned long long kHandoffWaitNs = 1000000000ull;
constexpr int kHandoffPolls = 1 << 23;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The hand-off flag's value once it is set, or 0 when the bounded wait ran
// out (one lane calls it).
__device__ __noinline__ int wait_handoff(const int* flag) {
  const unsigned long long deadline = gtimer() + kHandoffWaitNs;
  int hv = 0;
  for (int k = 0; k < kHandoffPolls; ++k) {
    hv = ld_acquire(flag);
    if (hv != 0 || gtimer() > deadline) break;
    __nanosleep(1000);
  }
  return hv;
}

template <int W, int R, int WPB, int MINB, int KIND>
__global__ void __launch_bounds__(32 * WPB, MINB)
relax_rigid_sw_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl, int n_rep,
                      float* pose, float* vel, float* fdt, float* falpha, int* fnp, int* status,
                      int* steps, double* energy, float* last_x, float* last_f, int* handoff, int queued,
                      int publish, int nsteps, FireP fp, Control ctl, int S) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  constexpr int RPW = 32 / W;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int sw = lane / W, l = lane % W;
  unsigned char* const wbase = dyn_smem + (size_t)(wib * RPW + sw) * sw_cache_bytes(S);
  StencilCache sc;
  sc.val = (float4*)wbase;
  sc.key = (int*)(wbase + (size_t)S * 256);
  sc.S = S;
  int2* const pub = (int2*)(wbase + cache_bytes(S));
  float* const cval = (float*)sc.val;
  const int warp = blockIdx.x * WPB + wib;
  const int n_warps = gridDim.x * WPB;
  const unsigned long long t0 = gtimer();
  // Relaxations that may stop early (f_conv > 0) have unknown lengths:
  // there the warps take whole tasks from an atomic queue (greedy list
  // scheduling) instead of the time-sliced ranges.
  const int n_tasks = (n_rep + RPW - 1) / RPW;
  for (int j = 0;; ++j) {      // uniform over the warp
    SwPart part;
    if (queued) {
      int next = 0;
      if (lane == 0) next = atomicAdd(&ctl.res->next, 1);
      next = __shfl_sync(kFull, next, 0);
      part = SwPart{next < n_tasks ? next : -1, 0, nsteps, 0};
    } else {
      part = sw_part(warp, n_warps, n_tasks, nsteps, j);
    }
    if (part.p < 0) break;
    const int p = part.p, it_b = part.it_b, it_e = part.it_e;
    const bool head = part.role == 1, tail = part.role == 2;
    // flag value of a finished head: bit 0 set, bit 1 + s set when the
    // abort flag or the clock budget stopped replica s of the task
    int hv = 1;
    if (tail) {
      // wait until the previous warp has written the head of this task
      if (lane == 0) {
        hv = wait_handoff(handoff + p);
        if (hv == 0) atomicAdd(&ctl.res->handoff_timeouts, 1);
      }
      hv = __shfl_sync(kFull, hv, 0);
      __syncwarp();
      if (hv == 0) continue;
    }
    const int r = p * RPW + sw;
    const bool valid = r < n_rep;
    int n = 0, ab = 0;
    float4 rig = make_float4(1.f, 1.f, 1.f, 1.f);
    float rmax = 1.f;
    float c[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f};
    float dt = 0.f, al = 0.f;
    int np = 0, st = 0, evals = 0;
    if (valid) {
      const int t = rep_tmpl[r];
      n = tv.natoms[t];
      ab = tv.atom_off[t];
      rig = tv.rigid[t];
      rmax = tv.rmax[t];
      // L2 loads: a tail part reads what another SM wrote in this launch
      for (int a = 0; a < 3; ++a) {
        c[a] = __ldcg(&pose[7 * (size_t)r + a]);
        v[a] = __ldcg(&vel[6 * (size_t)r + a]);
        w[a] = __ldcg(&vel[6 * (size_t)r + 3 + a]);
      }
      for (int a = 0; a < 4; ++a) q[a] = __ldcg(&pose[7 * (size_t)r + 3 + a]);
      dt = __ldcg(&fdt[r]);
      al = __ldcg(&falpha[r]);
      np = __ldcg(&fnp[r]);
      st = __ldcg(&status[r]);
    }
    // this lane's atoms i = k W + l, k < R (R W >= atoms): body coordinates
    // and grid factors stay in registers for the whole relaxation
    float4 bk[R], pk[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = k * W + l;
      bk[k] = pk[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid && i < n) {
        bk[k] = __ldg(&tv.body[ab + i]);
        pk[k] = __ldg(&tv.par[ab + i]);
      }
    }
    for (int i = l; i < S; i += W) sc.key[i] = -1;
    __syncwarp();
    const float inv_m = 1.f / rig.x;
    const float3 inv_I = make_float3(1.f / rig.y, 1.f / rig.z, 1.f / rig.w);
    const float ang_cap = fp.d_max / rmax;
    float elane = 0.f;
    // a tail whose head was stopped stops too (the head's state is final)
    bool done = !valid || ((hv >> (1 + sw)) & 1);
    bool stopped = false;
    for (int it = it_b; it < it_e; ++it) {
      if ((it & 31) == 0) {
        int sb = 0;
        if (l == 0 && !done) {
          if (*ctl.abort_flag) sb |= GRIDFF_REP_ABORTED;
          if (ctl.budget_ns && gtimer() - t0 > ctl.budget_ns) sb |= GRIDFF_REP_STEPLIMIT;
        }
        sb = __shfl_sync(kFull, sb, sw * W);
        if (sb) {
          st |= sb;
          done = true;
          stopped = true;
        }
      }
      if (st & (GRIDFF_REP_CONVERGED | GRIDFF_REP_NONFINITE)) done = true;
      if (!__any_sync(kFull, !done)) break;
      const bool run = !done;
      float Rm[9];
      quat_rot(q[0], q[1], q[2], q[3], Rm);
      float Ft[3], tq[3];
      float e = 0.f;
      int flags = 0;
      sw_forces<W, R, KIND, float>(g, sc, cval, pub, tv.par + ab, S, sw, l, n, run, c, Rm, bk, pk, Ft, tq, e,
                                    flags);
      if (!run) continue;
      st |= flags;
      ++evals;
      elane = e;
      const float f2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2] + tq[0] * tq[0] + tq[1] * tq[1] +
                       tq[2] * tq[2];
      // a NaN or infinity in any force or torque component reaches f2
      const bool fin = isfinite(f2) && isfinite(c[0] + c[1] + c[2]);
      if (l == 0 && (it == nsteps - 1 || !fin || f2 < fp.f_conv2)) record_rigid(last_x, last_f, r, c, q, Ft, tq);
      if (!fin) {
        st |= GRIDFF_REP_NONFINITE;
        continue;
      }
      if (f2 < fp.f_conv2) {
        st |= GRIDFF_REP_CONVERGED;
        continue;
      }
      // FIRE decision (identical in every lane of the sub-warp).  The
      // serial part of each iteration: norms by reciprocal square roots,
      // reciprocal masses and moments precomputed, no divisions.
      const float P = Ft[0] * v[0] + Ft[1] * v[1] + Ft[2] * v[2] + tq[0] * w[0] + tq[1] * w[1] + tq[2] * w[2];
      if (P > 0.f) {
        const float F2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2];
        const float T2 = tq[0] * tq[0] + tq[1] * tq[1] + tq[2] * tq[2];
        const float V2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const float W2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        // al |v| / |F| and al |w| / |tau|
        const float sf = F2 > 0.f && V2 > 0.f ? al * V2 * rsqrtf(V2) * rsqrtf(F2) : 0.f;
        const float sw_ = T2 > 0.f && W2 > 0.f ? al * W2 * rsqrtf(W2) * rsqrtf(T2) : 0.f;
        for (int a = 0; a < 3; ++a) {
          v[a] = (1.f - al) * v[a] + sf * Ft[a];
          w[a] = (1.f - al) * w[a] + sw_ * tq[a];
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
      const float adt = GRIDFF_ACC * dt;
      v[0] += adt * inv_m * Ft[0];
      v[1] += adt * inv_m * Ft[1];
      v[2] += adt * inv_m * Ft[2];
      w[0] += adt * inv_I.x * tq[0];
      w[1] += adt * inv_I.y * tq[1];
      w[2] += adt * inv_I.z * tq[2];
      const float dr[3] = {v[0] * dt, v[1] * dt, v[2] * dt};
      const float dn2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
      const float scl = dn2 > fp.d_max * fp.d_max ? fp.d_max * rsqrtf(dn2) : 1.f;
      for (int a = 0; a < 3; ++a) c[a] += dr[a] * scl;
      const float wn2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
      if (wn2 > 0.f) {
        const float iw = rsqrtf(wn2);
        const float ang = fminf(wn2 * iw * dt, ang_cap);
        quat_advance(q, w[0] * iw, w[1] * iw, w[2] * iw, ang);
      }
    }
    // energy of the last evaluation: sum over the sub-warp in FP64
    double et = (double)elane;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) et += __shfl_xor_sync(kFull, et, o);
    if (valid && l == 0) {
      const double Etot = evals > 0 ? et : __ldcg(&energy[r]);
      if (evals > 0 && !isfinite(Etot)) st |= GRIDFF_REP_NONFINITE;
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
      const int total = __ldcg(&steps[r]) + evals;
      steps[r] = total;
      energy[r] = Etot;
      // a head part counts its evaluations; convergence is counted once,
      // by the part that ends the task
      report(ctl, n, evals, head ? (st & ~GRIDFF_REP_CONVERGED) : st, total);
    }
    if (head && publish) {
      // publish the head's state to the warp that runs the tail
      const unsigned sm = __ballot_sync(kFull, stopped && l == 0);
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        int v = 1;
        for (int s2 = 0; s2 < RPW; ++s2)
          if ((sm >> (s2 * W)) & 1u) v |= 2 << s2;
        st_release(handoff + p, v);
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// FIRE, flexible replicas
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSM)
relax_flex_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl,
                  const int* __restrict__ rep_off, int n_rep, float* xs, float* vs, float* fdt,
                  float* falpha, int* fnp, int* status, int* steps, double* energy, float* last_x,
                  float* last_f, int nsteps, FireP fp, Control ctl, int use_grid, int use_intra, int S) {
  __shared__ WarpState s_all[kWarpsPerBlock];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpState& s = s_all[wib];
  const StencilCache sc = warp_cache(dyn_smem, S, wib);
  const int warp = blockIdx.x * kWarpsPerBlock + wib;
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    __syncwarp();
    cache_reset(sc, lane);
    for (int k = lane; k < 3 * n; k += 32) {
      s.x[k] = xs[3 * (size_t)off + k];
      s.v[k] = vs[3 * (size_t)off + k];
    }
    float dt = fdt[r], al = falpha[r];
    int np = fnp[r], st = status[r], evals = 0;
    float elane = 0.f;          // this lane's share of the last evaluated energy
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
      const float e = flex_forces<float>(g, use_grid, use_intra, tv, ab, n, lane, s, flags, sc);
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
      st |= __reduce_or_sync(kFull, flags);
      ++evals;
      elane = e;
      if (it == nsteps - 1 || (st & GRIDFF_REP_NONFINITE) || !(f2 >= fp.f_conv2))
        record_flex(last_x, last_f, off, n, lane, s.x, s.f);
      if ((st & GRIDFF_REP_NONFINITE) || !isfinite(f2)) {
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
    const double Etot = evals > 0 ? wsum((double)elane) : energy[r];
    if (evals > 0 && !isfinite(Etot)) st |= GRIDFF_REP_NONFINITE;
    if (lane == 0) {
      fdt[r] = dt;
      falpha[r] = al;
      fnp[r] = np;
      status[r] = st;
      int total = steps[r] + evals;
      steps[r] = total;
      energy[r] = Etot;
      report(ctl, n, evals, st, total);
    }
  }
}

// ---------------------------------------------------------------------------
// FIRE, flexible replicas of uneven size: unique-term intramolecular pass,
// WPB warps per block, replicas handed out by a work queue in decreasing
// cost order (order != nullptr) or statically (order == nullptr).  Same
// iteration as relax_flex_kernel.
// ---------------------------------------------------------------------------
#ifndef GRIDFF_FLEX_WARPS_PER_SM
#define GRIDFF_FLEX_WARPS_PER_SM 32    // register budget: 65536 / (32 * 32) = 64 per thread
#endif
// GC: the stencils of every atom are cached in global memory (gval, gkey:
// the replica's atoms from 16 rep_off[r] float4s and rep_off[r] keys, the
// layout of the shared-memory cache with one slot per atom), S = 0.
template <int WPB, int KIND, bool GC>
__global__ void __launch_bounds__(32 * WPB, GRIDFF_FLEX_WARPS_PER_SM / WPB)
relax_flex_terms_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl,
                        const int* __restrict__ rep_off, const int* __restrict__ order, int n_rep, float* xs,
                        float* vs, float* fdt, float* falpha, int* fnp, int* status, int* steps, double* energy,
                        float* last_x, float* last_f, int nsteps, FireP fp, Control ctl, int use_grid,
                        int use_intra, int S, float4* gval, int* gkey) {
  __shared__ WarpStateXF s_all[WPB];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpStateXF& s = s_all[wib];
  // per-warp dynamic shared memory: stencil cache, then the template's
  // nonbonded parameters {q, R, eps, 0}
  unsigned char* wbase = dyn_smem + (size_t)wib * flex_terms_warp_bytes(S);
  StencilCache sc;
  sc.val = (float4*)wbase;
  sc.key = (int*)(wbase + (size_t)S * 256);
  sc.S = S;
  float4* s_nb = (float4*)(wbase + cache_bytes(S));
  const int warp = blockIdx.x * WPB + wib;
  const int n_warps = gridDim.x * WPB;
  const unsigned long long t0 = gtimer();
  for (int k = warp;; k += n_warps) {
    if (order) {
      int next = 0;
      if (lane == 0) next = atomicAdd(&ctl.res->next, 1);
      k = __shfl_sync(kFull, next, 0);
    }
    if (k >= n_rep) break;
    const int r = order ? order[k] : k;
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    __syncwarp();
    if (GC && use_grid) {
      sc.val = gval + 16 * (size_t)off;
      sc.key = gkey + off;
      sc.S = n;
    }
    cache_reset(sc, lane);
    float* const v_r = vs + 3 * (size_t)off;   // this replica's velocities (global memory)
    for (int m = lane; m < 3 * n; m += 32) s.x[m] = xs[3 * (size_t)off + m];
    // nonbonded factors {q, alpha log2(e) R, eps} and the inverse mass in
    // the free fourth slot; zeros up to the next multiple of 32 atoms
    for (int i = lane; i < n; i += 32) {
      float4 p = __ldg(&tv.nb[ab + i]);
      p.y *= tv.alpha * kLog2e;
      p.w = 1.f / __ldg(&tv.body[ab + i]).w;
      s_nb[i] = p;
    }
    pad_pair_slots(s.x, s_nb, n, lane);
    float dt = fdt[r], al = falpha[r];
    int np = fnp[r], st = status[r], evals = 0;
    float elane = 0.f;
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
      const float e = flex_forces_terms<float, KIND>(g, use_grid, use_intra, tv, t, ab, n, lane, s, flags, sc,
                                                     s_nb);
      float f2 = 0.f, P = 0.f, v2 = 0.f;
      for (int m = lane; m < 3 * n; m += 32) {
        float f = s.f[m], v = v_r[m];
        f2 = fmaf(f, f, f2);
        P = fmaf(f, v, P);
        v2 = fmaf(v, v, v2);
      }
      f2 = wsum(f2);
      P = wsum(P);
      v2 = wsum(v2);
      st |= __reduce_or_sync(kFull, flags);
      ++evals;
      elane = e;
      if (it == nsteps - 1 || (st & GRIDFF_REP_NONFINITE) || !(f2 >= fp.f_conv2))
        record_flex(last_x, last_f, off, n, lane, s.x, s.f);
      if ((st & GRIDFF_REP_NONFINITE) || !isfinite(f2)) {
        st |= GRIDFF_REP_NONFINITE;
        break;
      }
      if (f2 < fp.f_conv2) {
        st |= GRIDFF_REP_CONVERGED;
        break;
      }
      float keep, mixf;
      if (P > 0.f) {
        keep = 1.f - al;
        mixf = f2 > 0.f && v2 > 0.f ? al * v2 * rsqrtf(v2) * rsqrtf(f2) : 0.f;   // al |v| / |F|
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
      const float adt = GRIDFF_ACC * dt, dmax2 = fp.d_max * fp.d_max;
      for (int i = lane; i < n; i += 32) {
        const float im = s_nb[i].w;
        float d[3];
        for (int a = 0; a < 3; ++a) {
          float f = s.f[3 * i + a];
          float vv = keep * v_r[3 * i + a] + mixf * f;
          vv += adt * im * f;
          v_r[3 * i + a] = vv;
          d[a] = vv * dt;
        }
        const float dn2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const float scl = dn2 > dmax2 ? fp.d_max * rsqrtf(dn2) : 1.f;
        for (int a = 0; a < 3; ++a) s.x[3 * i + a] += d[a] * scl;
      }
    }
    __syncwarp();
    for (int m = lane; m < 3 * n; m += 32) xs[3 * (size_t)off + m] = s.x[m];
    const double Etot = evals > 0 ? wsum((double)elane) : energy[r];
    if (evals > 0 && !isfinite(Etot)) st |= GRIDFF_REP_NONFINITE;
    if (lane == 0) {
      fdt[r] = dt;
      falpha[r] = al;
      fnp[r] = np;
      status[r] = st;
      int total = steps[r] + evals;
      steps[r] = total;
      energy[r] = Etot;
      report(ctl, n, evals, st, total);
    }
  }
}

// ---------------------------------------------------------------------------
// Langevin dynamics of flexible replicas (the thermalisation of minima
// hopping, Sec. 7), BAOAB splitting: half kick, half drift, exact
// Ornstein-Uhlenbeck velocity update v <- c1 v + c2 sqrt(kT/m) xi, half
// drift, forces, half kick; c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2).
// xi of replica r, global step s, component m = 3 i + a:
//   normal_of(splitmix64(splitmix64(seed ^ splitmix64(r)) ^ (512 s + m))).
// Layout as relax_flex_terms_kernel (warp per replica, work queue, GC: the
// global stencil cache).
// ---------------------------------------------------------------------------
template <int WPB, int KIND, bool GC>
__global__ void __launch_bounds__(32 * WPB, GRIDFF_FLEX_WARPS_PER_SM / WPB)
langevin_flex_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl,
                     const int* __restrict__ rep_off, const int* __restrict__ order, int n_rep, float* xs,
                     float* vs, int* status, double* energy, int nsteps, float dt, float c1, float c2,
                     float kT_acc, unsigned long long seed, long long step0, Control ctl, int use_grid,
                     int use_intra, int S, float4* gval, int* gkey) {
  __shared__ WarpState s_all[WPB];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpState& s = s_all[wib];
  unsigned char* wbase = dyn_smem + (size_t)wib * flex_terms_warp_bytes(S);
  StencilCache sc;
  sc.val = (float4*)wbase;
  sc.key = (int*)(wbase + (size_t)S * 256);
  sc.S = S;
  float4* s_nb = (float4*)(wbase + cache_bytes(S));
  const int warp = blockIdx.x * WPB + wib;
  const int n_warps = gridDim.x * WPB;
  const unsigned long long t0 = gtimer();
  const float hdt = 0.5f * dt;
  const float sq_kT = sqrtf(kT_acc);
  for (int k = warp;; k += n_warps) {
    if (order) {
      int next = 0;
      if (lane == 0) next = atomicAdd(&ctl.res->next, 1);
      k = __shfl_sync(kFull, next, 0);
    }
    if (k >= n_rep) break;
    const int r = order ? order[k] : k;
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    const unsigned long long key = splitmix64(seed ^ splitmix64((unsigned long long)r));
    __syncwarp();
    if (GC && use_grid) {
      sc.val = gval + 16 * (size_t)off;
      sc.key = gkey + off;
      sc.S = n;
    }
    cache_reset(sc, lane);
    for (int m = lane; m < 3 * n; m += 32) {
      s.x[m] = xs[3 * (size_t)off + m];
      s.v[m] = vs[3 * (size_t)off + m];
    }
    // nonbonded factors {q, alpha log2(e) R, eps} and 1/sqrt(m) in the
    // free fourth slot; zeros up to the next multiple of 32 atoms
    for (int i = lane; i < n; i += 32) {
      float4 p = __ldg(&tv.nb[ab + i]);
      p.y *= tv.alpha * kLog2e;
      p.w = rsqrtf(__ldg(&tv.body[ab + i]).w);
      s_nb[i] = p;
    }
    pad_pair_slots(s.x, s_nb, n, lane);
    int st = status[r] & ~(GRIDFF_REP_CONVERGED | GRIDFF_REP_ABORTED | GRIDFF_REP_STEPLIMIT);
    int flags = 0, steps_done = 0;
    float elane = flex_forces_terms<float, KIND>(g, use_grid, use_intra, tv, t, ab, n, lane, s, flags, sc, s_nb);
    for (int it = 0; it < nsteps && !(st & GRIDFF_REP_NONFINITE); ++it) {
      if ((it & 31) == 0) {
        const int sb = stop_bits(ctl, t0, lane);
        if (sb) {
          st |= sb;
          break;
        }
      }
      const unsigned long long sstep = (unsigned long long)(step0 + it) * 512ull;
      for (int m = lane; m < 3 * n; m += 32) {
        const float rsm = s_nb[m / 3].w;   // 1 / sqrt(m_i)
        float v = s.v[m] + hdt * GRIDFF_ACC * s.f[m] * (rsm * rsm);
        float x = s.x[m] + hdt * v;
        const float xi = normal_of(splitmix64(key ^ (sstep + (unsigned long long)m)));
        v = c1 * v + c2 * sq_kT * rsm * xi;
        s.x[m] = x + hdt * v;
        s.v[m] = v;
      }
      elane = flex_forces_terms<float, KIND>(g, use_grid, use_intra, tv, t, ab, n, lane, s, flags, sc, s_nb);
      float f2 = 0.f;
      for (int m = lane; m < 3 * n; m += 32) {
        const float rsm = s_nb[m / 3].w;
        s.v[m] += hdt * GRIDFF_ACC * s.f[m] * (rsm * rsm);
        f2 = fmaf(s.f[m], s.f[m], f2);
      }
      f2 = wsum(f2);
      st |= __reduce_or_sync(kFull, flags);
      ++steps_done;
      if (!isfinite(f2)) st |= GRIDFF_REP_NONFINITE;
    }
    __syncwarp();
    for (int m = lane; m < 3 * n; m += 32) {
      xs[3 * (size_t)off + m] = s.x[m];
      vs[3 * (size_t)off + m] = s.v[m];
    }
    const double Etot = wsum((double)elane);
    if (!isfinite(Etot)) st |= GRIDFF_REP_NONFINITE;
    if (lane == 0) {
      status[r] = st;
      energy[r] = Etot;
      report(ctl, n, steps_done + 1, st, steps_done);
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
                int use_grid, int use_intra, int S) {
  __shared__ WarpState s_all[kWarpsPerBlock];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpState& s = s_all[wib];
  const StencilCache sc = warp_cache(dyn_smem, S, wib);
  const int warp = blockIdx.x * kWarpsPerBlock + wib;
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    __syncwarp();
    cache_reset(sc, lane);
    for (int k = lane; k < 3 * n; k += 32) {
      s.x[k] = xs[3 * (size_t)off + k];
      s.v[k] = vs[3 * (size_t)off + k];
    }
    int st = status[r] & ~(GRIDFF_REP_ABORTED | GRIDFF_REP_STEPLIMIT);
    int flags = 0, evals = 0;
    double e = flex_forces(g, use_grid, use_intra, tv, ab, n, lane, s, flags, sc);
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
      e = flex_forces(g, use_grid, use_intra, tv, ab, n, lane, s, flags, sc);
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

// inv4I = 1 / (4 I_k).  Rotation angles of one step are small: below 0.05
// rad the sine and cosine come from their Taylor series (truncation below
// 2e-13, far under FP32 rounding), above from sincosf.
__device__ __forceinline__ void free_rot(int k, float h, float inv4I, float q[4], float p[4]) {
  float Pq[4], Pp[4];
  perm(k, q, Pq);
  perm(k, p, Pp);
  const float zeta = h * (p[0] * Pq[0] + p[1] * Pq[1] + p[2] * Pq[2] + p[3] * Pq[3]) * inv4I;
  float sz, cz;
  if (fabsf(zeta) < 0.05f) {
    const float z2 = zeta * zeta;
    sz = zeta * (1.f - z2 * (1.f / 6.f) * (1.f - z2 * (1.f / 20.f)));
    cz = 1.f - z2 * 0.5f * (1.f - z2 * (1.f / 12.f) * (1.f - z2 * (1.f / 30.f)));
  } else {
    sincosf(zeta, &sz, &cz);
  }
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
                 int rec_every, double* trace, Control ctl, int S) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31;
  const StencilCache sc = warp_cache(dyn_smem, S, threadIdx.x >> 5);
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int n_warps = gridDim.x * kWarpsPerBlock;
  const unsigned long long t0 = gtimer();
  for (int r = warp; r < n_rep; r += n_warps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t];
    const float4 rig = tv.rigid[t];
    const float I[3] = {rig.y, rig.z, rig.w};
    const float i4I[3] = {0.25f / rig.y, 0.25f / rig.z, 0.25f / rig.w};
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
    cache_reset(sc, lane);
    rigid_forces(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags, sc);
    e = wsum(e);
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
      free_rot(3, h, i4I[2], q, p);
      free_rot(2, h, i4I[1], q, p);
      free_rot(1, dt, i4I[0], q, p);
      free_rot(2, h, i4I[1], q, p);
      free_rot(3, h, i4I[2], q, p);
      quat_rot(q[0], q[1], q[2], q[3], Rm);
      rigid_forces(g, tv, ab, n, lane, c, Rm, Ft, tq, e, flags, sc);
      e = wsum(e);
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

// NVE of rigid replicas with the sub-warp layout of relax_rigid_sw_kernel
// (W lanes per replica, R atoms per lane, the stencil cache, sw_forces) and
// the NO_SQUISH splitting of run_rigid_kernel.  The energy is accumulated
// per lane in FP64 and summed over the sub-warp only when it is recorded.
template <int W, int R, int WPB, int MINB, int KIND>
__global__ void __launch_bounds__(32 * WPB, MINB)
run_rigid_sw_kernel(GridView g, TemplateView tv, const int* __restrict__ rep_tmpl, int n_rep, float* pose, float* vel,
                    int* status, double* energy, int* handoff, float4* handoff_p, int nsteps, float dt,
                    int rec_every, double* trace, Control ctl, int S) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  constexpr int RPW = 32 / W;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int sw = lane / W, l = lane % W;
  unsigned char* const wbase = dyn_smem + (size_t)(wib * RPW + sw) * sw_cache_bytes(S);
  StencilCache sc;
  sc.val = (float4*)wbase;
  sc.key = (int*)(wbase + (size_t)S * 256);
  sc.S = S;
  int2* const pub = (int2*)(wbase + cache_bytes(S));
  float* const cval = (float*)sc.val;
  const int warp = blockIdx.x * WPB + wib;
  const int n_warps = gridDim.x * WPB;
  const unsigned long long t0 = gtimer();
  // the time-sliced schedule of the relaxation kernel; a head hands on the
  // quaternion momentum exactly (handoff_p) besides the state arrays
  for (int j = 0;; ++j) {      // uniform over the warp
    const SwPart part = sw_part(warp, n_warps, (n_rep + RPW - 1) / RPW, nsteps, j);
    if (part.p < 0) break;
    const int it_b = part.it_b, it_e = part.it_e;
    const bool head = part.role == 1, tail = part.role == 2;
    int hv = 1;
    if (tail) {
      if (lane == 0) {
        hv = wait_handoff(handoff + part.p);
        if (hv == 0) atomicAdd(&ctl.res->handoff_timeouts, 1);
      }
      hv = __shfl_sync(kFull, hv, 0);
      __syncwarp();
      if (hv == 0) continue;
    }
    const int r = part.p * RPW + sw;
    // a replica whose head was stopped keeps the head's final state
    const bool valid = r < n_rep && !((hv >> (1 + sw)) & 1);
    int n = 0, ab = 0;
    float4 rig = make_float4(1.f, 1.f, 1.f, 1.f);
    float c[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f}, p[4] = {0.f, 0.f, 0.f, 0.f};
    int st = 0;
    if (valid) {
      const int t = rep_tmpl[r];
      n = tv.natoms[t];
      ab = tv.atom_off[t];
      rig = tv.rigid[t];
      for (int a = 0; a < 3; ++a) {
        c[a] = __ldcg(&pose[7 * (size_t)r + a]);
        v[a] = __ldcg(&vel[6 * (size_t)r + a]);
      }
      for (int a = 0; a < 4; ++a) q[a] = __ldcg(&pose[7 * (size_t)r + 3 + a]);
      if (tail) {
        const float4 pp = __ldcg(&handoff_p[r]);
        p[0] = pp.x;
        p[1] = pp.y;
        p[2] = pp.z;
        p[3] = pp.w;
        st = __ldcg(&status[r]);
      } else {
        const float L[3] = {rig.y * vel[6 * (size_t)r + 3], rig.z * vel[6 * (size_t)r + 4],
                            rig.w * vel[6 * (size_t)r + 5]};
        p[0] = 2.f * (-q[1] * L[0] - q[2] * L[1] - q[3] * L[2]);
        p[1] = 2.f * (q[0] * L[0] - q[3] * L[1] + q[2] * L[2]);
        p[2] = 2.f * (q[3] * L[0] + q[0] * L[1] - q[1] * L[2]);
        p[3] = 2.f * (-q[2] * L[0] + q[1] * L[1] + q[0] * L[2]);
        st = status[r] & ~(GRIDFF_REP_ABORTED | GRIDFF_REP_STEPLIMIT);
      }
    }
    const float I[3] = {rig.y, rig.z, rig.w};
    const float i4I[3] = {0.25f / I[0], 0.25f / I[1], 0.25f / I[2]};
    float4 bk[R], pk[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = k * W + l;
      bk[k] = pk[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid && i < n) {
        bk[k] = __ldg(&tv.body[ab + i]);
        pk[k] = __ldg(&tv.par[ab + i]);
      }
    }
    for (int i = l; i < S; i += W) sc.key[i] = -1;
    __syncwarp();
    const float ham = 0.5f * dt * GRIDFF_ACC / rig.x;
    auto sub_sum = [&](double x) {
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      return x;
    };
    auto total = [&](double epot) {
      float L[3];
      body_L(q, p, L);
      double ke = 0.5 * rig.x * (double)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      for (int a = 0; a < 3; ++a) ke += 0.5 * (double)L[a] * (double)L[a] / (double)I[a];
      return epot + ke / (double)GRIDFF_ACC;
    };
    float Rm[9];
    quat_rot(q[0], q[1], q[2], q[3], Rm);
    float Ft[3], tq[3];
    double e = 0.0;
    int flags = 0, evals = 0;
    bool run = valid, stopped = false;
    // forces at the start of the part (a tail recomputes those its head
    // ended with: the same values)
    sw_forces<W, R, KIND, double>(g, sc, cval, pub, tv.par + ab, S, sw, l, n, run, c, Rm, bk, pk, Ft, tq, e,
                                  flags);
    if (it_b == 0) {
      const double e0 = sub_sum(e);
      if (trace && valid && l == 0) trace[r] = total(e0);
    }
    for (int it = it_b; it < it_e; ++it) {
      if ((it & 31) == 0) {
        int sb = 0;
        if (l == 0 && run) {
          if (*ctl.abort_flag) sb |= GRIDFF_REP_ABORTED;
          if (ctl.budget_ns && gtimer() - t0 > ctl.budget_ns) sb |= GRIDFF_REP_STEPLIMIT;
        }
        sb = __shfl_sync(kFull, sb, sw * W);
        if (sb) {
          st |= sb;
          run = false;
          stopped = true;
        }
      }
      if (!__any_sync(kFull, run)) break;
      if (run) {
        const float h = 0.5f * dt;
        for (int a = 0; a < 3; ++a) v[a] += ham * Ft[a];
        const float tb[3] = {GRIDFF_ACC * tq[0], GRIDFF_ACC * tq[1], GRIDFF_ACC * tq[2]};
        kick_rot(p, q, tb, h);
        for (int a = 0; a < 3; ++a) c[a] += dt * v[a];
        free_rot(3, h, i4I[2], q, p);
        free_rot(2, h, i4I[1], q, p);
        free_rot(1, dt, i4I[0], q, p);
        free_rot(2, h, i4I[1], q, p);
        free_rot(3, h, i4I[2], q, p);
      }
      quat_rot(q[0], q[1], q[2], q[3], Rm);
      int f2 = 0;
      sw_forces<W, R, KIND, double>(g, sc, cval, pub, tv.par + ab, S, sw, l, n, run, c, Rm, bk, pk, Ft, tq, e,
                                    f2);
      if (run) {
        flags |= f2;
        ++evals;
        for (int a = 0; a < 3; ++a) v[a] += ham * Ft[a];
        const float tb[3] = {GRIDFF_ACC * tq[0], GRIDFF_ACC * tq[1], GRIDFF_ACC * tq[2]};
        kick_rot(p, q, tb, 0.5f * dt);
      }
      if (rec_every > 0 && (it + 1) % rec_every == 0) {
        const double et = sub_sum(e);
        if (trace && valid && run && l == 0) trace[(size_t)((it + 1) / rec_every) * n_rep + r] = total(et);
      }
    }
    const double et = sub_sum(e);
    if (valid && l == 0) {
      st |= flags;
      if (!isfinite(et)) st |= GRIDFF_REP_NONFINITE;
      float L[3];
      body_L(q, p, L);
      for (int a = 0; a < 3; ++a) {
        pose[7 * (size_t)r + a] = c[a];
        vel[6 * (size_t)r + a] = v[a];
        vel[6 * (size_t)r + 3 + a] = L[a] / I[a];
      }
      for (int a = 0; a < 4; ++a) pose[7 * (size_t)r + 3 + a] = q[a];
      if (head) handoff_p[r] = make_float4(p[0], p[1], p[2], p[3]);
      status[r] = st;
      energy[r] = et;
      report(ctl, n, evals, st & ~GRIDFF_REP_CONVERGED, it_b + evals);
    }
    if (head) {
      const unsigned sm = __ballot_sync(kFull, stopped && l == 0);
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        int hvv = 1;
        for (int s2 = 0; s2 < RPW; ++s2)
          if ((sm >> (s2 * W)) & 1u) hvv |= 2 << s2;
        st_release(handoff + part.p, hvv);
      }
    }
    __syncwarp();
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

#ifndef GRIDFF_BLOCK_CAP
#define GRIDFF_BLOCK_CAP 0
#endif
#ifndef GRIDFF_CACHE_CAP
#define GRIDFF_CACHE_CAP 128
#endif

// Stencil-cache slots per warp: every atom of the largest template, up to a
// cap (rigid kernels keep no other per-warp shared state; flexible kernels
// also hold positions, velocities and forces).
int cache_slots(const gridff_replicas* R, bool rigid) {
  int cap = rigid ? GRIDFF_CACHE_CAP : (GRIDFF_CACHE_CAP < 48 ? GRIDFF_CACHE_CAP : 48);
  return R->max_natoms < cap ? R->max_natoms : cap;
}

#ifndef GRIDFF_SW_WARPS
#define GRIDFF_SW_WARPS 4
#endif
#ifndef GRIDFF_SW_MINB
#define GRIDFF_SW_MINB 2
#endif
constexpr int kSwWarps = GRIDFF_SW_WARPS;
constexpr int kSwMinBlocks = GRIDFF_SW_MINB;
#ifndef GRIDFF_RIGID_SUBWARP
#define GRIDFF_RIGID_SUBWARP -1      // -1: chosen from the molecule size; 0: quad kernel
#endif
// Sub-warp width of the rigid relaxation kernel (0 = the quad kernel, used
// when the cache would not fit): among W = 8, 16, 32 with R = ceil(n / W)
// atoms per lane, prefer R <= 3 (R = 4 costs registers), then the fewest
// idle lane slots (n / (W R) largest), then the smaller W.  Measured on
// GB300 for 10, 24, 38 and 60 atoms this picks the fastest width each time.
int rigid_subwarp_width(const gridff_replicas* R) {
  if (GRIDFF_RIGID_SUBWARP >= 0) return GRIDFF_RIGID_SUBWARP;
  const int n = R->max_natoms;
  int best = 0;
  double best_score = -1.0;
  for (int W : {8, 16, 32}) {
    const int rounds = (n + W - 1) / W;
    if (rounds > 4) continue;
    const double score = (rounds <= 3 ? 2.0 : 0.0) + (double)n / (W * rounds);
    if (score > best_score + 1e-12) {
      best_score = score;
      best = W;
    }
  }
  if (best == 0) return 0;
  return sw_cache_bytes(n) * kSwWarps * (32 / best) <= 200 * 1024 ? best : 0;
}

// Allow `bytes` of dynamic shared memory (needed whenever static plus
// dynamic shared memory exceeds 48 KB).
cudaError_t set_dyn_smem(const void* kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
int persistent_blocks(gridff_ctx* ctx, const void* kernel, int n_rep, size_t dyn_smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, dyn_smem);
  if (per_sm < 1) per_sm = 1;
  if (GRIDFF_BLOCK_CAP > 0 && per_sm > GRIDFF_BLOCK_CAP) per_sm = GRIDFF_BLOCK_CAP;
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

__global__ void fire_reset_kernel(int n, float dt0, float a0, float* dt, float* al, int* np, int* st, int* steps) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  dt[r] = dt0;
  al[r] = a0;
  np[r] = 0;
  st[r] = 0;
  steps[r] = 0;
}

using SwFn = void (*)(GridView, TemplateView, const int*, int, float*, float*, float*, float*, int*, int*, int*,
                     double*, float*, float*, int*, int, int, int, FireP, Control, int);

// Sub-warp rigid kernel for W lanes per replica and R atoms per lane; FP32
// four-slot grids get a build without the other record kinds' code.
SwFn rigid_sw_fn(int W, int R, int kind) {
#define GRIDFF_SW(w, r)                                                                     \
  if (W == w && R == r)                                                                     \
    return kind == REC_F32x4 ? relax_rigid_sw_kernel<w, r, kSwWarps, kSwMinBlocks, REC_F32x4> \
                             : relax_rigid_sw_kernel<w, r, kSwWarps, kSwMinBlocks, -1>;
  GRIDFF_SW(8, 1) GRIDFF_SW(8, 2) GRIDFF_SW(8, 3) GRIDFF_SW(8, 4)
  GRIDFF_SW(16, 1) GRIDFF_SW(16, 2) GRIDFF_SW(16, 3) GRIDFF_SW(16, 4)
  GRIDFF_SW(32, 1) GRIDFF_SW(32, 2) GRIDFF_SW(32, 3) GRIDFF_SW(32, 4)
#undef GRIDFF_SW
  return nullptr;
}
int sw_rounds(const gridff_replicas* R, int W) { return (R->max_natoms + W - 1) / W; }

using RunSwFn = void (*)(GridView, TemplateView, const int*, int, float*, float*, int*, double*, int*, float4*, int,
                         float, int, double*, Control, int);
// NVE sub-warp kernel for W lanes per replica and R atoms per lane.
RunSwFn run_sw_fn(int W, int R, int kind) {
#define GRIDFF_RSW(w, r)                                                                  \
  if (W == w && R == r)                                                                   \
    return kind == REC_F32x4 ? run_rigid_sw_kernel<w, r, kSwWarps, kSwMinBlocks, REC_F32x4> \
                             : run_rigid_sw_kernel<w, r, kSwWarps, kSwMinBlocks, -1>;
  GRIDFF_RSW(8, 1) GRIDFF_RSW(8, 2) GRIDFF_RSW(8, 3) GRIDFF_RSW(8, 4)
  GRIDFF_RSW(16, 1) GRIDFF_RSW(16, 2) GRIDFF_RSW(16, 3) GRIDFF_RSW(16, 4)
  GRIDFF_RSW(32, 1) GRIDFF_RSW(32, 2) GRIDFF_RSW(32, 3) GRIDFF_RSW(32, 4)
#undef GRIDFF_RSW
  return nullptr;
}
// FP32 four-slot grids get their own instances (the record kind known at
// compile time); other kinds dispatch at run time.
using FlexTermsFn = void (*)(GridView, TemplateView, const int*, const int*, const int*, int, float*, float*, float*,
                             float*, int*, int*, int*, double*, float*, float*, int, FireP, Control, int, int, int,
                             float4*, int*);
template <int K, bool GC>
FlexTermsFn flex_terms_fn_k(int wpb) {
  return wpb == 2 ? relax_flex_terms_kernel<2, K, GC> : wpb == 8 ? relax_flex_terms_kernel<8, K, GC>
                                                                 : relax_flex_terms_kernel<4, K, GC>;
}
FlexTermsFn flex_terms_fn(int wpb, int kind, bool gc) {
  if (gc) return kind == REC_F32x4 ? flex_terms_fn_k<REC_F32x4, true>(wpb) : flex_terms_fn_k<-1, true>(wpb);
  return kind == REC_F32x4 ? flex_terms_fn_k<REC_F32x4, false>(wpb) : flex_terms_fn_k<-1, false>(wpb);
}
const void* flex_terms_ptr(int wpb, int kind, bool gc) { return (const void*)flex_terms_fn(wpb, kind, gc);
}

struct KernelShape {
  const void* fn;
  int threads;
  int units_per_block;   // replicas resident per block
  size_t dyn;            // dynamic shared memory
};

// Kernel, block shape and dynamic shared memory of configuration c, or
// fn == nullptr when c does not apply to R.
KernelShape shape_of(const gridff_replicas* R, const LaunchCfg& c, int kind) {
  KernelShape k{nullptr, 0, 0, 0};
  switch (c.kernel) {
    case GRIDFF_KERNEL_RIGID_SUBWARP: {
      if (!R->rigid || (c.W != 8 && c.W != 16 && c.W != 32) || c.S < R->max_natoms) return k;
      const SwFn fn = rigid_sw_fn(c.W, sw_rounds(R, c.W), kind);
      if (!fn) return k;
      return {(const void*)fn, 32 * kSwWarps, kSwWarps * (32 / c.W), sw_cache_bytes(c.S) * kSwWarps * (32 / c.W)};
    }
    case GRIDFF_KERNEL_RIGID_QUAD:
      if (!R->rigid || c.wpb != kWarpsPerBlock) return k;
      return {(const void*)relax_rigid_kernel, kThreads, kWarpsPerBlock, cache_bytes(c.S) * kWarpsPerBlock};
    case GRIDFF_KERNEL_FLEX_QUAD:
      if (R->rigid || c.wpb != kWarpsPerBlock) return k;
      return {(const void*)relax_flex_kernel, kThreads, kWarpsPerBlock, cache_bytes(c.S) * kWarpsPerBlock};
    case GRIDFF_KERNEL_FLEX_TERMS:
      if (R->rigid || (c.wpb != 2 && c.wpb != 4 && c.wpb != 8) || (c.gcache && c.S != 0)) return k;
      return {flex_terms_ptr(c.wpb, kind, c.gcache != 0), 32 * c.wpb, c.wpb, flex_terms_warp_bytes(c.S) * c.wpb};
    default:
      return k;
  }
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
  if (hres->handoff_timeouts)
    return set_err(ctx, GRIDFF_ETIMEOUT, "%d split relaxations did not receive their first part in time",
                   hres->handoff_timeouts);
  return GRIDFF_OK;
}

}  // namespace

LaunchCfg default_launch_cfg(const gridff_replicas* R, bool use_grid) {
  LaunchCfg c;
  if (R->rigid) {
    const int W = rigid_subwarp_width(R);
    if (use_grid && W > 0) {
      c.kernel = GRIDFF_KERNEL_RIGID_SUBWARP;
      c.W = W;
      c.wpb = kSwWarps;
      c.S = R->max_natoms;
    } else {
      c.kernel = GRIDFF_KERNEL_RIGID_QUAD;
      c.wpb = kWarpsPerBlock;
      c.S = cache_slots(R, true);
    }
  } else {
    // measured on 16384 replicas of 10-120 atoms: the unique-term kernel
    // with the work queue and the stencils cached in global memory is
    // fastest (shared-memory staging costs more occupancy than it saves)
    c.kernel = GRIDFF_KERNEL_FLEX_TERMS;
    c.wpb = 8;
    c.S = 0;
    c.queue = 1;
    c.gcache = use_grid ? 1 : 0;
  }
  return c;
}

gridff_status check_fire_params(gridff_ctx* ctx, const gridff_fire_params& P) {
  if (!(P.dt_start > 0) || !(P.dt_max > 0) || !(P.d_max > 0) || P.f_conv < 0)
    return set_err(ctx, GRIDFF_EINVAL, "bad FIRE parameters");
  return GRIDFF_OK;
}

// The global stencil cache of a flexible replica set: one 256-byte stencil
// and a key per atom, allocated at the first use and kept with the set.
static gridff_status ensure_gcache(gridff_ctx* ctx, gridff_replicas* R) {
  if (R->gval) return GRIDFF_OK;
  if (cudaMalloc(&R->gval, (size_t)R->n_atoms * 256) != cudaSuccess ||
      cudaMalloc(&R->gkey, (size_t)R->n_atoms * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(R->gval);
    R->gval = nullptr;
    return set_err(ctx, GRIDFF_ENOMEM, "global stencil cache of %d atoms", R->n_atoms);
  }
  return GRIDFF_OK;
}

gridff_status prepare_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, const LaunchCfg& c,
                            int flags, int* blocks_out) {
  const KernelShape k = shape_of(R, c, grid ? grid->kind : REC_F32x4);
  if (!k.fn) return set_err(ctx, GRIDFF_EINVAL, "launch configuration (kernel %d) does not apply", c.kernel);
  if (c.S < 0 || c.S > GRIDFF_MAX_ATOMS) return set_err(ctx, GRIDFF_EINVAL, "cache slots %d", c.S);
  if (c.kernel == GRIDFF_KERNEL_RIGID_SUBWARP && (flags & GRIDFF_NO_GRID))
    return set_err(ctx, GRIDFF_EINVAL, "the sub-warp rigid kernel needs the grid term");
  cudaFuncAttributes fa{};
  GRIDFF_CUDA(ctx, cudaFuncGetAttributes(&fa, k.fn));
  int optin = 0;
  GRIDFF_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  if (fa.sharedSizeBytes + k.dyn > (size_t)optin)
    return set_err(ctx, GRIDFF_EINVAL, "launch configuration needs %zu B of shared memory per block (limit %d)",
                   fa.sharedSizeBytes + k.dyn, optin);
  GRIDFF_CUDA(ctx, set_dyn_smem(k.fn, k.dyn));
  int per_sm = 0;
  GRIDFF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.threads, k.dyn));
  if (per_sm < 1) return set_err(ctx, GRIDFF_EINVAL, "launch configuration does not fit on an SM");
  if (GRIDFF_BLOCK_CAP > 0 && per_sm > GRIDFF_BLOCK_CAP) per_sm = GRIDFF_BLOCK_CAP;
  if (c.blocks < 0) return set_err(ctx, GRIDFF_EINVAL, "block cap %d", c.blocks);
  if (c.queue < 0 || c.queue > (c.kernel == GRIDFF_KERNEL_RIGID_SUBWARP ? 2 : 1))
    return set_err(ctx, GRIDFF_EINVAL, "queue mode %d", c.queue);
  if ((c.gcache != 0 && c.gcache != 1) || (c.gcache && c.kernel != GRIDFF_KERNEL_FLEX_TERMS))
    return set_err(ctx, GRIDFF_EINVAL, "cache_global %d with kernel %d", c.gcache, c.kernel);
  if (c.gcache) {
    const gridff_status gs = ensure_gcache(ctx, R);
    if (gs != GRIDFF_OK) return gs;
  }
  const int need = (R->n_rep + k.units_per_block - 1) / k.units_per_block;
  *blocks_out = need < per_sm * ctx->n_sm ? need : per_sm * ctx->n_sm;
  if (c.blocks > 0 && *blocks_out > c.blocks) *blocks_out = c.blocks;
  if (c.l2win && grid && !(flags & GRIDFF_NO_GRID)) {   // the window holds the grid: none without it
    int max_persist = 0, max_win = 0;
    GRIDFF_CUDA(ctx, cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device));
    GRIDFF_CUDA(ctx, cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device));
    if (max_persist <= 0 || max_win <= 0) return set_err(ctx, GRIDFF_ENOTSUP, "no persisting L2 on this device");
    if (!ctx->l2_limit_set) {
      GRIDFF_CUDA(ctx, cudaDeviceGetLimit(&ctx->l2_prev_limit, cudaLimitPersistingL2CacheSize));
      ctx->l2_limit_set = 1;
    }
    const size_t want = grid->rec_bytes < (size_t)max_persist ? grid->rec_bytes : (size_t)max_persist;
    size_t cur = 0;
    GRIDFF_CUDA(ctx, cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
    if (cur < want) GRIDFF_CUDA(ctx, cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
  }
  return GRIDFF_OK;
}

namespace {

template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*fn)(KArgs...), int blocks, int threads, size_t dyn, cudaStream_t s,
                      const cudaAccessPolicyWindow* win, Args... args) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(blocks);
  lc.blockDim = dim3(threads);
  lc.dynamicSmemBytes = dyn;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  if (win) {
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow = *win;
    lc.attrs = attr;
    lc.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&lc, fn, args...);
}

}  // namespace

gridff_status enqueue_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, const LaunchCfg& c,
                            int blocks, int nsteps, const gridff_fire_params& P, int flags) {
  cudaStream_t s = ctx->stream;
  if (!(flags & GRIDFF_CONTINUE)) {
    fire_reset_kernel<<<(R->n_rep + 255) / 256, 256, 0, s>>>(R->n_rep, P.dt_start, P.alpha_start, R->fire_dt,
                                                             R->fire_alpha, R->fire_nplus, R->status, R->steps);
    GRIDFF_CUDA(ctx, cudaGetLastError());
  }
  // without CONTINUE the FIRE scalars, status and counters start afresh; a
  // continued relaxation keeps them (converged/non-finite replicas stay
  // frozen, stop bits of the previous call stay visible)
  GRIDFF_CUDA(ctx, cudaMemsetAsync(ctx->result_dev, 0, sizeof(DevResult), s));
  FireP fp{P.dt_start, P.dt_max, P.f_inc, P.f_dec, P.alpha_start, P.f_alpha, P.d_max,
           P.f_conv * P.f_conv, P.n_min};
  Control ctl{ctx->ctrl_dev, (unsigned long long)(P.clock_budget_s > 0 ? P.clock_budget_s * 1e9 : 0),
              (DevResult*)ctx->result_dev};
  GridView gv = grid ? grid->view() : empty_view();
  const int use_grid = !(flags & GRIDFF_NO_GRID), use_intra = !(flags & GRIDFF_NO_INTRA);
  const int kind = grid ? grid->kind : REC_F32x4;
  const KernelShape k = shape_of(R, c, kind);
  cudaAccessPolicyWindow win{};
  const cudaAccessPolicyWindow* wp = nullptr;
  if (c.l2win && grid && use_grid) {
    int max_win = 0;
    size_t lim = 0;
    cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device);
    cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize);
    win.base_ptr = (void*)grid->rec;
    win.num_bytes = grid->rec_bytes < (size_t)max_win ? grid->rec_bytes : (size_t)max_win;
    win.hitRatio = win.num_bytes > 0 && lim < win.num_bytes ? (float)lim / (float)win.num_bytes : 1.f;
    win.hitProp = cudaAccessPropertyPersisting;
    win.missProp = cudaAccessPropertyStreaming;
    wp = &win;
  }
  cudaError_t e = cudaSuccess;
  switch (c.kernel) {
    case GRIDFF_KERNEL_RIGID_SUBWARP:
      // hand-off flags of the time-sliced schedule, cleared for this launch
      GRIDFF_CUDA(ctx, cudaMemsetAsync(R->handoff, 0, R->n_rep * sizeof(int), s));
      e = launch_ex(rigid_sw_fn(c.W, sw_rounds(R, c.W), kind), blocks, k.threads, k.dyn, s, wp, gv, R->tv,
                    (const int*)R->rep_tmpl, R->n_rep, R->x, R->v, R->fire_dt, R->fire_alpha, R->fire_nplus,
                    R->status, R->steps, R->energy, R->last_x, R->last_f, R->handoff,
                    (int)(c.queue == 1 || (c.queue == 0 && P.f_conv > 0)), (int)!(flags & GRIDFF_TEST_NO_HANDOFF),
                    nsteps, fp, ctl, c.S);
      break;
    case GRIDFF_KERNEL_RIGID_QUAD:
      e = launch_ex(relax_rigid_kernel, blocks, k.threads, k.dyn, s, wp, gv, R->tv, (const int*)R->rep_tmpl,
                    R->n_rep, R->x, R->v, R->fire_dt, R->fire_alpha, R->fire_nplus, R->status, R->steps, R->energy,
                    R->last_x, R->last_f, nsteps, fp, ctl, use_grid, c.S);
      break;
    case GRIDFF_KERNEL_FLEX_QUAD:
      e = launch_ex(relax_flex_kernel, blocks, k.threads, k.dyn, s, wp, gv, R->tv, (const int*)R->rep_tmpl,
                    (const int*)R->rep_off, R->n_rep, R->x, R->v, R->fire_dt, R->fire_alpha, R->fire_nplus,
                    R->status, R->steps, R->energy, R->last_x, R->last_f, nsteps, fp, ctl, use_grid, use_intra, c.S);
      break;
    case GRIDFF_KERNEL_FLEX_TERMS: {
      const int* ord = c.queue ? (const int*)R->order : nullptr;
      e = launch_ex(flex_terms_fn(c.wpb, kind, c.gcache != 0), blocks, k.threads, k.dyn, s, wp, gv, R->tv,
                    (const int*)R->rep_tmpl, (const int*)R->rep_off, ord, R->n_rep, R->x, R->v, R->fire_dt,
                    R->fire_alpha, R->fire_nplus, R->status, R->steps, R->energy, R->last_x, R->last_f, nsteps, fp,
                    ctl, use_grid, use_intra, c.S, R->gval, R->gkey);
      break;
    }
    default:
      return set_err(ctx, GRIDFF_EINVAL, "unknown kernel %d", c.kernel);
  }
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "relaxation launch: %s", cudaGetErrorString(e));
  return GRIDFF_OK;
}

// host entry points (traced with NVTX ranges)
#include "trace.h"

extern "C" {

gridff_status gridff_eval(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int flags,
                          double* E_out, float* F_out, float* Ea_out, int32_t* st_out) {
  NvtxRange nvtx_range("gridff_eval");
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

gridff_status gridff_eval_points(gridff_ctx* ctx, const gridff_grid* grid, int64_t n, const float* xyz,
                                 const float* qpl, float* E, float* F, int32_t* status, int flags) {
  NvtxRange nvtx_range("gridff_eval_points");
  if (!ctx) return GRIDFF_EINVAL;
  if (!grid || n < 0 || (n > 0 && (!xyz || !qpl || !E || !F)))
    return set_err(ctx, GRIDFF_EINVAL, "null argument or negative count");
  if (n == 0) return GRIDFF_OK;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const bool dev = flags & GRIDFF_DEVICE_PTRS;
  const size_t n3 = 3 * (size_t)n * sizeof(float), n1 = (size_t)n * sizeof(float);
  Staging stg(ctx);
  const float *dx = xyz, *dq = qpl;
  float *dE = E, *dF = F;
  int* dS = status;
  if (!dev) {
    GRIDFF_CUDA(ctx, cudaMallocAsync(&stg.ptr, 3 * n3 + 2 * n1 + 64, s));
    char* p = (char*)stg.ptr;
    float* hx = (float*)p;
    float* hq = (float*)(p + n3);
    dF = (float*)(p + 2 * n3);
    dE = (float*)(p + 3 * n3);
    dS = status ? (int*)(p + 3 * n3 + n1) : nullptr;
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(hx, xyz, n3, cudaMemcpyHostToDevice, s));
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(hq, qpl, n3, cudaMemcpyHostToDevice, s));
    dx = hx;
    dq = hq;
  }
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
  if (flags & GRIDFF_POINTS_BINNED) {
    const gridff_status bst = enqueue_eval_points_binned(ctx, grid, n, dx, dq, dE, dF, dS);
    if (bst != GRIDFF_OK) return bst;
  } else {
    const GridView gv = grid->view();
    const void* fn = grid->kind == REC_F32x4 ? (const void*)eval_points_kernel<REC_F32x4>
                                             : (const void*)eval_points_kernel<-1>;
    int per_sm = 0;
    GRIDFF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0));
    const long long need = (n + 63) / 64;   // 8 warps x 8 points per block round
    const long long cap = (long long)(per_sm > 0 ? per_sm : 1) * ctx->n_sm;
    const int blocks = (int)(need < cap ? need : cap);
    if (grid->kind == REC_F32x4)
      eval_points_kernel<REC_F32x4><<<blocks, 256, 0, s>>>(gv, (long long)n, dx, dq, dE, dF, dS);
    else
      eval_points_kernel<-1><<<blocks, 256, 0, s>>>(gv, (long long)n, dx, dq, dE, dF, dS);
    GRIDFF_CUDA(ctx, cudaGetLastError());
  }
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev1, s));
  if (!dev) {
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(E, dE, n1, cudaMemcpyDeviceToHost, s));
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(F, dF, n3, cudaMemcpyDeviceToHost, s));
    if (status) GRIDFF_CUDA(ctx, cudaMemcpyAsync(status, dS, n1, cudaMemcpyDeviceToHost, s));
  }
  if (!(dev && (flags & GRIDFF_ASYNC))) {
    GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) ctx->last_ms = ms;
  }
  return GRIDFF_OK;
}

gridff_status gridff_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int32_t nsteps,
                           const gridff_fire_params* prm, int flags, gridff_relax_result* result) {
  NvtxRange nvtx_range("gridff_relax");
  gridff_status st = check_common(ctx, grid, R, flags);
  if (st != GRIDFF_OK) return st;
  if (nsteps < 0) return set_err(ctx, GRIDFF_EINVAL, "nsteps < 0");
  gridff_fire_params def;
  gridff_fire_params_default(&def);
  const gridff_fire_params& P = prm ? *prm : def;
  if ((st = check_fire_params(ctx, P)) != GRIDFF_OK) return st;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const bool use_grid = !(flags & GRIDFF_NO_GRID);
  const LaunchCfg c = R->cfg.kernel >= 0 ? R->cfg : default_launch_cfg(R, use_grid);
  int blocks = 0;
  if ((st = prepare_relax(ctx, grid, R, c, flags, &blocks)) != GRIDFF_OK) return st;
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  if ((st = enqueue_relax(ctx, grid, R, c, blocks, nsteps, P, flags)) != GRIDFF_OK) return st;
  DevResult h{};
  gridff_status rs = finish_launch(ctx, &h);
  if (result) {
    result->atom_evals = (int64_t)h.atom_evals;
    result->n_converged = h.n_converged;
    result->max_steps = h.max_steps;
  }
  return rs;
}

gridff_status gridff_langevin(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int32_t nsteps,
                              const gridff_langevin_params* prm, int flags) {
  NvtxRange nvtx_range("gridff_langevin");
  gridff_status st = check_common(ctx, grid, R, flags);
  if (st != GRIDFF_OK) return st;
  if (!prm || !(prm->dt > 0) || !(prm->temperature >= 0) || !(prm->gamma >= 0) || nsteps < 0 || prm->step0 < 0)
    return set_err(ctx, GRIDFF_EINVAL, "bad Langevin parameters");
  if (R->rigid) return set_err(ctx, GRIDFF_ENOTSUP, "Langevin dynamics is implemented for flexible replicas");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  GRIDFF_CUDA(ctx, cudaMemsetAsync(ctx->result_dev, 0, sizeof(DevResult), s));
  Control ctl{ctx->ctrl_dev, (unsigned long long)(prm->clock_budget_s > 0 ? prm->clock_budget_s * 1e9 : 0),
              (DevResult*)ctx->result_dev};
  GridView gv = grid ? grid->view() : empty_view();
  const int use_grid = !(flags & GRIDFF_NO_GRID), use_intra = !(flags & GRIDFF_NO_INTRA);
  const double c1 = exp(-(double)prm->gamma * prm->dt);
  const double c2 = sqrt(1.0 - c1 * c1);
  const double kB = 8.617333262e-5;   // eV/K
  const float kT_acc = (float)(kB * prm->temperature * GRIDFF_ACC);
  // layout: the replica set's unique-term configuration if it has one
  const LaunchCfg c = R->cfg.kernel == GRIDFF_KERNEL_FLEX_TERMS ? R->cfg : default_launch_cfg(R, true);
  const int wpb = c.kernel == GRIDFF_KERNEL_FLEX_TERMS ? c.wpb : 8;
  const int S = c.kernel == GRIDFF_KERNEL_FLEX_TERMS ? c.S : 0;
  const bool gc = c.kernel == GRIDFF_KERNEL_FLEX_TERMS && c.gcache && S == 0 && use_grid;
  if (gc) {
    const gridff_status gs = ensure_gcache(ctx, R);
    if (gs != GRIDFF_OK) return gs;
  }
  using LangevinFn = void (*)(GridView, TemplateView, const int*, const int*, const int*, int, float*, float*, int*,
                              double*, int, float, float, float, float, unsigned long long, long long, Control, int,
                              int, int, float4*, int*);
  const bool f32 = !grid || grid->kind == REC_F32x4;
  const LangevinFn lf =
      gc ? (f32 ? (wpb == 2 ? langevin_flex_kernel<2, REC_F32x4, true>
                            : wpb == 4 ? langevin_flex_kernel<4, REC_F32x4, true> : langevin_flex_kernel<8, REC_F32x4, true>)
                : (wpb == 2 ? langevin_flex_kernel<2, -1, true>
                            : wpb == 4 ? langevin_flex_kernel<4, -1, true> : langevin_flex_kernel<8, -1, true>))
         : (f32 ? (wpb == 2 ? langevin_flex_kernel<2, REC_F32x4, false>
                            : wpb == 4 ? langevin_flex_kernel<4, REC_F32x4, false>
                                       : langevin_flex_kernel<8, REC_F32x4, false>)
                : (wpb == 2 ? langevin_flex_kernel<2, -1, false>
                            : wpb == 4 ? langevin_flex_kernel<4, -1, false> : langevin_flex_kernel<8, -1, false>));
  const void* fn = (const void*)lf;
  const size_t dyn = flex_terms_warp_bytes(S) * wpb;
  GRIDFF_CUDA(ctx, set_dyn_smem(fn, dyn));
  int per_sm = 0;
  GRIDFF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * wpb, dyn));
  if (per_sm < 1) return set_err(ctx, GRIDFF_EINVAL, "Langevin launch does not fit on an SM");
  const int need = (R->n_rep + wpb - 1) / wpb;
  const int blocks = need < per_sm * ctx->n_sm ? need : per_sm * ctx->n_sm;
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
  lf<<<blocks, 32 * wpb, dyn, s>>>(gv, R->tv, R->rep_tmpl, R->rep_off, R->order, R->n_rep, R->x, R->v, R->status,
                                   R->energy, nsteps, prm->dt, (float)c1, (float)c2, kT_acc,
                                   (unsigned long long)prm->seed, (long long)prm->step0, ctl, use_grid, use_intra, S,
                                   R->gval, R->gkey);
  DevResult h{};
  return finish_launch(ctx, &h);
}

gridff_status gridff_run(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, int32_t nsteps,
                         const gridff_md_params* prm, int flags, double* energy_trace) {
  NvtxRange nvtx_range("gridff_run");
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
    const int W = rigid_subwarp_width(R);
    const RunSwFn fn = W > 0 ? run_sw_fn(W, sw_rounds(R, W), grid->kind) : nullptr;
    if (fn) {
      // the sub-warp layout of the relaxation, every atom cached
      const int S = R->max_natoms;
      const size_t dyn = sw_cache_bytes(S) * kSwWarps * (32 / W);
      GRIDFF_CUDA(ctx, set_dyn_smem((const void*)fn, dyn));
      const int per_block = kSwWarps * (32 / W);
      int per_sm = 0;
      GRIDFF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, 32 * kSwWarps, dyn));
      if (per_sm < 1) per_sm = 1;
      const int need = (R->n_rep + per_block - 1) / per_block;
      int blocks = need < per_sm * ctx->n_sm ? need : per_sm * ctx->n_sm;
      if (R->cfg.blocks > 0 && blocks > R->cfg.blocks) blocks = R->cfg.blocks;
      GRIDFF_CUDA(ctx, cudaMemsetAsync(R->handoff, 0, R->n_rep * sizeof(int), s));
      fn<<<blocks, 32 * kSwWarps, dyn, s>>>(gv, R->tv, R->rep_tmpl, R->n_rep, R->x, R->v, R->status, R->energy,
                                            R->handoff, R->handoff_p, nsteps, prm->dt, rec_every, dtrace, ctl, S);
      DevResult h{};
      gridff_status rs = finish_launch(ctx, &h);
      if (energy_trace && !dev) {
        GRIDFF_CUDA(ctx, cudaMemcpyAsync(energy_trace, dtrace, tbytes, cudaMemcpyDeviceToHost, s));
        GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
      }
      return rs;
    }
    const int S = cache_slots(R, true);
    const size_t dyn = cache_bytes(S) * kWarpsPerBlock;
    GRIDFF_CUDA(ctx, set_dyn_smem((const void*)run_rigid_kernel, dyn));
    int blocks = persistent_blocks(ctx, (const void*)run_rigid_kernel, R->n_rep, dyn);
    run_rigid_kernel<<<blocks, kThreads, dyn, s>>>(gv, R->tv, R->rep_tmpl, R->n_rep, R->x, R->v, R->status,
                                                   R->energy, nsteps, prm->dt, rec_every, dtrace, ctl, S);
  } else {
    const int S = cache_slots(R, false);
    const size_t dyn = cache_bytes(S) * kWarpsPerBlock;
    GRIDFF_CUDA(ctx, set_dyn_smem((const void*)run_flex_kernel, dyn));
    int blocks = persistent_blocks(ctx, (const void*)run_flex_kernel, R->n_rep, dyn);
    run_flex_kernel<<<blocks, kThreads, dyn, s>>>(gv, R->tv, R->rep_tmpl, R->rep_off, R->n_rep, R->x, R->v,
                                                  R->status, R->energy, nsteps, prm->dt, rec_every, dtrace, ctl,
                                                  use_grid, use_intra, S);
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
