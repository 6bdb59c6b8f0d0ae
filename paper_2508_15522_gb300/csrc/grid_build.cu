// Substrate grid construction on the GPU (Sec. 3, 4, 5 of the paper):
//   node values of V^C (3D Ewald, slab dipole correction), V^P, V^L
//   -> exact cubic B-spline coefficients (separable 1D line solves)
//   -> padded float4 records read by the interpolation kernels.
// Everything before the final packing runs in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kKe = 14.399645;  // eV*A/e^2

struct alignas(32) D4 {   // x, y, z, charge
  double x, y, z, w;
};

struct RowInfo {      // one row of in-plane reciprocal vectors: fixed m1, m2 in [lo, hi]
  int m1, lo, hi, goff;
};

struct BuildParams {
  int nx, ny, nz;
  double x0, y0, z0, dx, dy, dz;
  double A1x, A1y, A2x, A2y, Lz;    // cell
  int n_img1, n_img2;               // in-plane image range
  double alpha, rcut2, ercut2, beta;
  int morse;                        // compute V^P, V^L
  int coulomb;                      // compute V^C
  int slotP, slotL, slotC;          // output channel slots (-1 = absent)
  double bg;                        // -pi Q / (beta^2 V)
  double dip;                       // 4 pi M_z / V
  double B1x, B1y, B2x, B2y;        // in-plane reciprocal vectors
  int n_rows;
  int nzk;                          // z samples in the G table (= nz)
};

// --------------------------------------------------------------------------
// reciprocal-space tables
// --------------------------------------------------------------------------
// AS[k2][m3] = A_k S(k) for k = m1 B1 + m2 B2 + m3 B3 (A_k = 4 pi e^{-k^2/4b^2}/(V k^2),
// S(k) = sum_j q_j e^{-i k.r_j}); zero outside the sphere |k| < kmax or at k = 0.
__global__ void k_struct_kernel(const D4* __restrict__ atoms, int n_atoms,
                                const int2* __restrict__ k2_m, int n_k2, int M3, double B1x,
                                double B1y, double B2x, double B2y, double B3z, double kmax2,
                                double beta, double vol, double2* __restrict__ AS) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nm3 = 2 * M3 + 1;
  if (idx >= n_k2 * nm3) return;
  int k2 = idx / nm3, m3 = idx % nm3 - M3;
  int2 m = k2_m[k2];
  double kx = m.x * B1x + m.y * B2x, ky = m.x * B1y + m.y * B2y, kz = m3 * B3z;
  double k2n = kx * kx + ky * ky + kz * kz;
  double2 out = make_double2(0.0, 0.0);
  if (k2n > 0.0 && k2n < kmax2) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < n_atoms; ++j) {
      D4 a = atoms[j];
      double s, c;
      sincos(kx * a.x + ky * a.y + kz * a.z, &s, &c);
      re += a.w * c;
      im -= a.w * s;
    }
    double A = 4.0 * kPi / vol * exp(-k2n / (4.0 * beta * beta)) / k2n;
    out = make_double2(A * re, A * im);
  }
  AS[idx] = out;
}

// G[k2][l] = sum_m3 AS[k2][m3] e^{i kz(m3) z_l}
__global__ void k_zsum_kernel(const double2* __restrict__ AS, int n_k2, int M3, double B3z,
                              double z0, double dz, int nz, double2* __restrict__ G) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_k2 * nz) return;
  int k2 = idx / nz, l = idx % nz;
  double z = z0 + l * dz;
  int nm3 = 2 * M3 + 1;
  double re = 0.0, im = 0.0;
  for (int t = 0; t < nm3; ++t) {
    double2 as = AS[(size_t)k2 * nm3 + t];
    if (as.x == 0.0 && as.y == 0.0) continue;
    double s, c;
    sincos((t - M3) * B3z * z, &s, &c);
    re += as.x * c - as.y * s;
    im += as.x * s + as.y * c;
  }
  G[idx] = make_double2(re, im);
}

// --------------------------------------------------------------------------
// node values: one thread per node, z fastest
// --------------------------------------------------------------------------
constexpr int kNodeThreads = 256;

__global__ void __launch_bounds__(kNodeThreads)
node_values_kernel(BuildParams p, const D4* __restrict__ atoms,
                   const double2* __restrict__ Reps, int n_atoms,
                   const RowInfo* __restrict__ rows, const double2* __restrict__ G,
                   double* __restrict__ vals) {
  __shared__ D4 s_at[kNodeThreads];
  __shared__ double2 s_re[kNodeThreads];
  size_t n_nodes = (size_t)p.nx * p.ny * p.nz;
  size_t node = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool live = node < n_nodes;
  size_t nn = live ? node : 0;
  int iz = (int)(nn % p.nz);
  int iy = (int)((nn / p.nz) % p.ny);
  int ix = (int)(nn / ((size_t)p.nz * p.ny));
  double x = p.x0 + ix * p.dx, y = p.y0 + iy * p.dy, z = p.z0 + iz * p.dz;

  double vP = 0.0, vL = 0.0, phi = 0.0;
  for (int base = 0; base < n_atoms; base += kNodeThreads) {
    int j = base + threadIdx.x;
    if (j < n_atoms) {
      s_at[threadIdx.x] = atoms[j];
      s_re[threadIdx.x] = Reps[j];
    }
    __syncthreads();
    int cnt = min(kNodeThreads, n_atoms - base);
    if (live) {
      for (int t = 0; t < cnt; ++t) {
        D4 a = s_at[t];
        double2 re = s_re[t];
        double ddz = z - a.z, dz2 = ddz * ddz;
        for (int n1 = -p.n_img1; n1 <= p.n_img1; ++n1) {
          for (int n2 = -p.n_img2; n2 <= p.n_img2; ++n2) {
            double ddx = x - (a.x + n1 * p.A1x + n2 * p.A2x);
            double ddy = y - (a.y + n1 * p.A1y + n2 * p.A2y);
            double d2 = ddx * ddx + ddy * ddy + dz2;
            if (p.morse && d2 < p.rcut2) {
              double d = sqrt(d2);
              double e1 = exp(-p.alpha * (d - re.x));
              vL += re.y * e1;
              vP += re.y * e1 * e1;
            }
            if (p.coulomb && d2 < p.ercut2 && a.w != 0.0) {
              double d = sqrt(d2);
              phi += a.w * erfc(p.beta * d) / d;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if (!live) return;
  if (p.coulomb) {
    // reciprocal part: sum over in-plane rows of Re(G[k2][l] e^{i k.rho})
    double rec = 0.0;
    double th2 = p.B2x * x + p.B2y * y;
    double s2, c2;
    sincos(th2, &s2, &c2);
    for (int r = 0; r < p.n_rows; ++r) {
      RowInfo ri = rows[r];
      double th = ri.m1 * (p.B1x * x + p.B1y * y) + ri.lo * th2;
      double ps, pc;
      sincos(th, &ps, &pc);
      const double2* g = G + (size_t)ri.goff * p.nzk + iz;
      for (int m2 = ri.lo; m2 <= ri.hi; ++m2) {
        double2 gv = g[(size_t)(m2 - ri.lo) * p.nzk];
        rec += gv.x * pc - gv.y * ps;
        double npc = pc * c2 - ps * s2;
        ps = ps * c2 + pc * s2;
        pc = npc;
      }
    }
    phi += rec + p.bg + p.dip * z;
    vals[(size_t)p.slotC * n_nodes + node] = kKe * phi;
  }
  if (p.morse) {
    vals[(size_t)p.slotP * n_nodes + node] = vP;
    vals[(size_t)p.slotL * n_nodes + node] = vL;
  }
}

// --------------------------------------------------------------------------
// B-spline line solves (FP64, in place)
// --------------------------------------------------------------------------
// Tridiagonal matrix with constant off-diagonals 1/6 and diagonal bd[k]:
// forward sweep d'_k = (d_k - d'_{k-1}/6) inv[k], back substitution
// y_k = d'_k - cp[k] y_{k+1}.  Cyclic systems add the Sherman-Morrison
// correction x = y - fac (y_0 + (1/6)/gamma y_{n-1}) zc.
struct LineTables {
  const double* inv;
  const double* cp;
  const double* zc;      // nullptr: not cyclic
  double fac, a_over_gamma;
};

__global__ void line_solve_kernel(double* __restrict__ data, int n, long long stride,
                                  long long n_lines, int inner, long long inner_stride,
                                  long long outer_stride, LineTables t) {
  long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= n_lines) return;
  long long o = line / inner, i = line % inner;
  double* d = data + o * outer_stride + i * inner_stride;
  const double a = 1.0 / 6.0;
  double prev = 0.0;
  for (int k = 0; k < n; ++k) {
    double v = (d[k * stride] - a * prev) * t.inv[k];
    d[k * stride] = v;
    prev = v;
  }
  double next = d[(long long)(n - 1) * stride];
  for (int k = n - 2; k >= 0; --k) {
    double v = d[k * stride] - t.cp[k] * next;
    d[k * stride] = v;
    next = v;
  }
  if (t.zc) {
    double s = t.fac * (d[0] + t.a_over_gamma * d[(long long)(n - 1) * stride]);
    for (int k = 0; k < n; ++k) d[k * stride] -= s * t.zc[k];
  }
}

void host_tables(int n, bool cyclic, std::vector<double>& out, double& fac, double& aog) {
  const double a = 1.0 / 6.0, c = 1.0 / 6.0, b = 2.0 / 3.0;
  std::vector<double> bd(n, b);
  double gamma = -b;
  if (cyclic) {
    bd[0] = b - gamma;
    bd[n - 1] = b - a * c / gamma;
  } else {
    bd[0] = b + a;        // clamped end: the index -1 reads b_0
    bd[n - 1] = b + c;    // index n reads b_{n-1}
  }
  std::vector<double> inv(n), cp(n);
  inv[0] = 1.0 / bd[0];
  cp[0] = c * inv[0];
  for (int k = 1; k < n; ++k) {
    double den = bd[k] - a * cp[k - 1];
    inv[k] = 1.0 / den;
    cp[k] = c * inv[k];
  }
  std::vector<double> zc(n, 0.0);
  fac = 0.0;
  aog = 0.0;
  if (cyclic) {
    std::vector<double> u(n, 0.0);
    u[0] = gamma;
    u[n - 1] = c;
    double prev = 0.0;
    for (int k = 0; k < n; ++k) {
      zc[k] = (u[k] - a * prev) * inv[k];
      prev = zc[k];
    }
    for (int k = n - 2; k >= 0; --k) zc[k] -= cp[k] * zc[k + 1];
    aog = a / gamma;
    fac = 1.0 / (1.0 + zc[0] + aog * zc[n - 1]);
  }
  out.clear();
  out.insert(out.end(), inv.begin(), inv.end());
  out.insert(out.end(), cp.begin(), cp.end());
  out.insert(out.end(), zc.begin(), zc.end());
}

// --------------------------------------------------------------------------
// packing into padded records
// --------------------------------------------------------------------------
// Round x to the nearest value with `bits` significant bits (ties to even),
// quantum at least 2^min_exp: the value an FP16 (11, -24) or BF16 (8, -133)
// number nearest to x has; computed exactly in FP64 (x / q is exact for a
// power of two q, rint rounds to even).
__device__ double round_sig(double x, int bits, int min_exp) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  frexp(x, &e);
  const int qe = e - bits > min_exp ? e - bits : min_exp;
  const double q = ldexp(1.0, qe);
  return rint(x / q) * q;
}

template <int KIND>
__global__ void pack_kernel(const double* __restrict__ coefs, int nx, int ny, int nz, int nyp, int nzp,
                            long long n_rec, int slotC, int slotP, int slotL, double iC, double iP, double iL,
                            void* __restrict__ out) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rec) return;
  int pz = (int)(r % nzp);
  int py = (int)((r / nzp) % nyp);
  int px = (int)(r / ((long long)nzp * nyp));
  int ix = (px - 1 + nx) % nx, iy = (py - 1 + ny) % ny;
  int iz = min(max(pz - 1, 0), nz - 1);
  size_t n_nodes = (size_t)nx * ny * nz;
  size_t node = ((size_t)ix * ny + iy) * nz + iz;
  // coefficient / scale (the scales are powers of two: exact)
  const double c = slotC >= 0 ? coefs[(size_t)slotC * n_nodes + node] * iC : 0.0;
  const double p = slotP >= 0 ? coefs[(size_t)slotP * n_nodes + node] * iP : 0.0;
  const double l = slotL >= 0 ? coefs[(size_t)slotL * n_nodes + node] * iL : 0.0;
  if (KIND == REC_F32x4) {
    ((float4*)out)[r] = make_float4((float)c, (float)p, (float)l, 0.f);
  } else if (KIND == REC_F32x2) {
    ((float2*)out)[r] = make_float2((float)p, (float)l);
  } else if (KIND == REC_F16x4 || KIND == REC_F16x2) {
    const __half hc = __double2half(round_sig(c, 11, -24)), hp = __double2half(round_sig(p, 11, -24));
    const __half hl = __double2half(round_sig(l, 11, -24));
    if (KIND == REC_F16x4) {
      ((__half2*)out)[2 * r] = __halves2half2(hc, hp);
      ((__half2*)out)[2 * r + 1] = __halves2half2(hl, __double2half(0.0));
    } else {
      ((__half2*)out)[r] = __halves2half2(hp, hl);
    }
  } else {
    const __nv_bfloat16 bc = __double2bfloat16(round_sig(c, 8, -133));
    const __nv_bfloat16 bp = __double2bfloat16(round_sig(p, 8, -133));
    const __nv_bfloat16 bl = __double2bfloat16(round_sig(l, 8, -133));
    if (KIND == REC_BF16x4) {
      ((__nv_bfloat162*)out)[2 * r] = __halves2bfloat162(bc, bp);
      ((__nv_bfloat162*)out)[2 * r + 1] = __halves2bfloat162(bl, __double2bfloat16(0.0));
    } else {
      ((__nv_bfloat162*)out)[r] = __halves2bfloat162(bp, bl);
    }
  }
}

// max |coefficient| of each channel (bit patterns of non-negative doubles
// order like the values)
__global__ void absmax_kernel(const double* __restrict__ coefs, size_t n_nodes, int n_ch,
                              unsigned long long* __restrict__ out) {
  for (int ch = 0; ch < n_ch; ++ch) {
    double m = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (size_t)gridDim.x * blockDim.x)
      m = fmax(m, fabs(coefs[(size_t)ch * n_nodes + i]));
    if (m > 0.0) atomicMax(&out[ch], (unsigned long long)__double_as_longlong(m));
  }
}

struct DevFree {
  std::vector<void*> ptrs;
  ~DevFree() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t alloc(T** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  void release(void* p) { ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end()); }
};

void channel_slots(int channels, int& sC, int& sP, int& sL, int& n_ch) {
  n_ch = 0;
  sC = sP = sL = -1;
  if (channels & GRIDFF_CH_C) sC = n_ch++;
  if (channels & GRIDFF_CH_P) sP = n_ch++;
  if (channels & GRIDFF_CH_L) sL = n_ch++;
}

// Allocate grid->rec for the grid's storage layout and pack FP64
// coefficients ([C][nx][ny][nz], device) into it.  FP16/BF16: per-channel
// scale 2^(e - 15) with max |coef| < 2^e, so that |coef| / scale < 2^15.
gridff_status pack_records(gridff_ctx* ctx, gridff_grid* g, const double* data) {
  int nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
  cudaStream_t s = ctx->stream;
  g->nxp = nx + 3;
  g->nyp = ny + 3;
  g->nzp = nz + 2;
  int sC, sP, sL, nch;
  channel_slots(g->channels, sC, sP, sL, nch);
  const bool two = sC < 0;     // no Coulomb channel: {P, L} records
  g->kind = g->storage == GRIDFF_STORE_F16 ? (two ? REC_F16x2 : REC_F16x4)
          : g->storage == GRIDFF_STORE_BF16 ? (two ? REC_BF16x2 : REC_BF16x4)
                                            : (two ? REC_F32x2 : REC_F32x4);
  double inv[3] = {1.0, 1.0, 1.0};
  g->scale[0] = g->scale[1] = g->scale[2] = 1.f;
  if (g->storage != GRIDFF_STORE_F32) {
    unsigned long long* mx = nullptr;
    GRIDFF_CUDA(ctx, cudaMallocAsync((void**)&mx, 3 * sizeof(unsigned long long), s));
    cudaError_t e = cudaMemsetAsync(mx, 0, 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      absmax_kernel<<<4 * ctx->n_sm, 256, 0, s>>>(data, (size_t)nx * ny * nz, nch, mx);
      e = cudaGetLastError();
    }
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, mx, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(mx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "channel maxima: %s", cudaGetErrorString(e));
    const int slot_of[3] = {sC, sP, sL};
    for (int c = 0; c < 3; ++c) {
      if (slot_of[c] < 0) continue;
      double m;
      memcpy(&m, &h[slot_of[c]], sizeof(double));
      int ex = 0;
      if (m > 0.0) frexp(m, &ex);
      g->scale[c] = (float)ldexp(1.0, ex - 15);
      inv[c] = ldexp(1.0, 15 - ex);
    }
  }
  long long n_rec = (long long)g->nxp * g->nyp * g->nzp;
  g->rec_bytes = (size_t)n_rec * rec_bytes_of(g->kind);
  GRIDFF_CUDA(ctx, cudaMalloc(&g->rec, g->rec_bytes));
  const unsigned blocks = (unsigned)((n_rec + 255) / 256);
#define GRIDFF_PACK(K)                                                                                \
  pack_kernel<K><<<blocks, 256, 0, s>>>(data, nx, ny, nz, g->nyp, g->nzp, n_rec, sC, sP, sL, inv[0], \
                                         inv[1], inv[2], g->rec)
  switch (g->kind) {
    case REC_F32x4: GRIDFF_PACK(REC_F32x4); break;
    case REC_F32x2: GRIDFF_PACK(REC_F32x2); break;
    case REC_F16x4: GRIDFF_PACK(REC_F16x4); break;
    case REC_F16x2: GRIDFF_PACK(REC_F16x2); break;
    case REC_BF16x4: GRIDFF_PACK(REC_BF16x4); break;
    default: GRIDFF_PACK(REC_BF16x2); break;
  }
#undef GRIDFF_PACK
  GRIDFF_CUDA(ctx, cudaGetLastError());
  return GRIDFF_OK;
}

bool storage_ok(int st) {
  return st == GRIDFF_STORE_F32 || st == GRIDFF_STORE_F16 || st == GRIDFF_STORE_BF16;
}

// Fit coefficients in place (3 passes) and pack them into grid->rec.
gridff_status fit_and_pack(gridff_ctx* ctx, gridff_grid* g, double* data, DevFree& df) {
  int nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
  int n_ch = g->n_ch;
  cudaStream_t s = ctx->stream;
  // tables for the three axes
  std::vector<double> tz, ty, tx;
  double fz, ay, fy, ax, fx, az;
  host_tables(nz, false, tz, fz, az);
  host_tables(ny, true, ty, fy, ay);
  host_tables(nx, true, tx, fx, ax);
  std::vector<double> all;
  all.insert(all.end(), tz.begin(), tz.end());
  all.insert(all.end(), ty.begin(), ty.end());
  all.insert(all.end(), tx.begin(), tx.end());
  double* dt = nullptr;
  GRIDFF_CUDA(ctx, df.alloc(&dt, all.size() * sizeof(double)));
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(dt, all.data(), all.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
  double* pz = dt;
  double* py = dt + tz.size();
  double* px = py + ty.size();
  long long N = (long long)nx * ny * nz;
  const int TB = 128;
  // z: lines (c, ix, iy), contiguous
  {
    LineTables t{pz, pz + nz, nullptr, 0.0, 0.0};
    long long lines = (long long)n_ch * nx * ny;
    line_solve_kernel<<<(unsigned)((lines + TB - 1) / TB), TB, 0, s>>>(data, nz, 1, lines, 1, 0,
                                                                      nz, t);
  }
  // y: lines (c, ix, iz): outer = c*nx + ix (stride ny*nz), inner = iz
  {
    LineTables t{py, py + ny, py + 2 * ny, fy, ay};
    long long lines = (long long)n_ch * nx * nz;
    line_solve_kernel<<<(unsigned)((lines + TB - 1) / TB), TB, 0, s>>>(
        data, ny, nz, lines, nz, 1, (long long)ny * nz, t);
  }
  // x: lines (c, iy, iz): outer = c (stride N), inner = iy*nz + iz
  {
    LineTables t{px, px + nx, px + 2 * nx, fx, ax};
    long long lines = (long long)n_ch * ny * nz;
    line_solve_kernel<<<(unsigned)((lines + TB - 1) / TB), TB, 0, s>>>(
        data, nx, (long long)ny * nz, lines, ny * nz, 1, N, t);
  }
  GRIDFF_CUDA(ctx, cudaGetLastError());
  return pack_records(ctx, g, data);
}

bool dims_ok(const int* d) { return d[0] >= 4 && d[1] >= 4 && d[2] >= 4; }

// --------------------------------------------------------------------------
// Allocation-free coefficient fit (gridff_fit_coefs_noalloc)
// --------------------------------------------------------------------------
// The per-axis line-solve tables live in this file-scope device array
// instead of memory allocated per call.  Layout per axis a (0 = x, 1 = y,
// 2 = z): inv[n], cp[n], zc[n], then fac and a_over_gamma, at a * kNoAllocStride.
constexpr int kNoAllocMaxN = 4096;
constexpr int kNoAllocStride = 3 * kNoAllocMaxN + 2;
__device__ __align__(256) double g_noalloc_tables[3 * kNoAllocStride];

// One thread per axis builds that axis' tables (same recurrences as host_tables).
__global__ void noalloc_tables_kernel(double* tab, int nx, int ny, int nz) {
  int a = threadIdx.x;
  if (a > 2) return;
  int n = a == 0 ? nx : a == 1 ? ny : nz;
  bool cyclic = a < 2;
  double* inv = tab + (size_t)a * kNoAllocStride;
  double* cp = inv + kNoAllocMaxN;
  double* zc = cp + kNoAllocMaxN;
  double* scal = zc + kNoAllocMaxN;
  const double lo = 1.0 / 6.0, up = 1.0 / 6.0, b = 2.0 / 3.0, gamma = -b;
  for (int k = 0; k < n; ++k) {
    double bd = b;
    if (k == 0) bd = cyclic ? b - gamma : b + lo;
    if (k == n - 1) bd = cyclic ? b - lo * up / gamma : b + up;
    double den = k == 0 ? bd : bd - lo * cp[k - 1];
    inv[k] = 1.0 / den;
    cp[k] = up * inv[k];
  }
  scal[0] = 0.0;
  scal[1] = 0.0;
  if (cyclic) {
    double prev = 0.0;
    for (int k = 0; k < n; ++k) {
      double u = k == 0 ? gamma : (k == n - 1 ? up : 0.0);
      zc[k] = (u - lo * prev) * inv[k];
      prev = zc[k];
    }
    for (int k = n - 2; k >= 0; --k) zc[k] -= cp[k] * zc[k + 1];
    scal[1] = lo / gamma;
    scal[0] = 1.0 / (1.0 + zc[0] + scal[1] * zc[n - 1]);
  }
}

// Line solve that reads its tables (and the cyclic correction scalars) from
// device memory; `cyclic` selects the Sherman-Morrison correction.
__global__ void noalloc_line_kernel(double* __restrict__ data, int n, long long stride, long long n_lines,
                                    int inner, long long inner_stride, long long outer_stride,
                                    const double* __restrict__ tab, int cyclic) {
  long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= n_lines) return;
  const double* inv = tab;
  const double* cp = tab + kNoAllocMaxN;
  const double* zc = cp + kNoAllocMaxN;
  const double* scal = zc + kNoAllocMaxN;
  long long o = line / inner, i = line % inner;
  double* d = data + o * outer_stride + i * inner_stride;
  const double a = 1.0 / 6.0;
  double prev = 0.0;
  for (int k = 0; k < n; ++k) {
    double v = (d[k * stride] - a * prev) * inv[k];
    d[k * stride] = v;
    prev = v;
  }
  double next = d[(long long)(n - 1) * stride];
  for (int k = n - 2; k >= 0; --k) {
    double v = d[k * stride] - cp[k] * next;
    d[k * stride] = v;
    next = v;
  }
  if (cyclic) {
    double s = scal[0] * (d[0] + scal[1] * d[(long long)(n - 1) * stride]);
    for (int k = 0; k < n; ++k) d[k * stride] -= s * zc[k];
  }
}

// Device address of g_noalloc_tables, looked up once per device (the host
// symbol g_noalloc_tables is only a stand-in, never a device address).
double* noalloc_tables_address(int device, cudaError_t* err) {
  static std::mutex mu;
  static double* addr[64] = {nullptr};
  *err = cudaSuccess;
  if (device < 0 || device >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_tables);
    if (*err != cudaSuccess) return nullptr;
    addr[device] = (double*)p;
  }
  return addr[device];
}

}  // namespace

GridView gridff_grid::view() const {
  GridView v;
  v.rec = rec;
  v.kind = kind;
  v.sC = scale[0];
  v.sP = scale[1];
  v.sL = scale[2];
  v.nx = dims[0];
  v.ny = dims[1];
  v.nz = dims[2];
  v.nyp = nyp;
  v.nzp = nzp;
  v.sx = (long long)nyp * nzp;
  v.x0 = (float)origin[0];
  v.y0 = (float)origin[1];
  v.z0 = (float)origin[2];
  v.inv_dx = (float)(1.0 / spacing[0]);
  v.inv_dy = (float)(1.0 / spacing[1]);
  v.inv_dz = (float)(1.0 / spacing[2]);
  v.Lx = (float)(spacing[0] * dims[0]);
  v.Ly = (float)(spacing[1] * dims[1]);
  v.inv_Lx = (float)(1.0 / (spacing[0] * dims[0]));
  v.inv_Ly = (float)(1.0 / (spacing[1] * dims[1]));
  v.uzf = (float)ghost;
  return v;
}

extern "C" {

gridff_status gridff_build_grid(gridff_ctx* ctx, const gridff_substrate* sub,
                                const gridff_grid_opts* opts, gridff_grid** out) {
  NvtxRange nvtx_range("gridff_build_grid");
  if (!ctx || !sub || !opts || !out) return set_err(ctx, GRIDFF_EINVAL, "null argument");
  *out = nullptr;
  if (sub->n_atoms <= 0 || !sub->xyz || !sub->q || !sub->R || !sub->eps)
    return set_err(ctx, GRIDFF_EINVAL, "substrate needs n_atoms > 0 and all arrays");
  if (!storage_ok(opts->storage)) return set_err(ctx, GRIDFF_ENOTSUP, "storage not supported");
  if (!(opts->spacing > 0) || !(opts->length[0] > 0) || !(opts->length[1] > 0) ||
      !(opts->length[2] > 0))
    return set_err(ctx, GRIDFF_EINVAL, "grid box lengths and spacing must be > 0");
  const double* C = sub->cell;
  if (C[2] != 0.0 || C[5] != 0.0 || C[6] != 0.0 || C[7] != 0.0 || !(C[8] > 0))
    return set_err(ctx, GRIDFF_EINVAL, "cell rows must be A1, A2 in-plane and A3 = (0, 0, Lz)");
  double area = C[0] * C[4] - C[1] * C[3];
  if (!(fabs(area) > 1e-6)) return set_err(ctx, GRIDFF_EINVAL, "degenerate in-plane cell");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));

  gridff_grid* g = new gridff_grid();
  g->ctx = ctx;
  g->device = ctx->device;
  g->storage = opts->storage;
  bool charged = false;
  double Qtot = 0.0, Mz = 0.0;
  double zmin = 1e300, zmax = -1e300;
  for (int j = 0; j < sub->n_atoms; ++j) {
    charged |= sub->q[j] != 0.0;
    Qtot += sub->q[j];
    Mz += sub->q[j] * sub->xyz[3 * j + 2];
    zmin = std::min(zmin, sub->xyz[3 * j + 2]);
    zmax = std::max(zmax, sub->xyz[3 * j + 2]);
  }
  int chans = opts->channels ? opts->channels : (GRIDFF_CH_C | GRIDFF_CH_P | GRIDFF_CH_L);
  if (!charged) chans &= ~GRIDFF_CH_C;
  if (!(chans & (GRIDFF_CH_P | GRIDFF_CH_L)) && !(chans & GRIDFF_CH_C)) {
    delete g;
    return set_err(ctx, GRIDFF_EINVAL, "no channel to build");
  }
  // Morse channels come in pairs
  if (chans & (GRIDFF_CH_P | GRIDFF_CH_L)) chans |= GRIDFF_CH_P | GRIDFF_CH_L;
  g->channels = chans;
  int sC, sP, sL;
  channel_slots(chans, sC, sP, sL, g->n_ch);
  if (opts->ghost_below < 0 || opts->ghost_below > 64) {
    delete g;
    return set_err(ctx, GRIDFF_EINVAL, "ghost_below = %d outside 0..64", opts->ghost_below);
  }
  for (int a = 0; a < 3; ++a) {
    g->dims[a] = (int)ceil(opts->length[a] / opts->spacing - 1e-9);
    g->spacing[a] = opts->length[a] / g->dims[a];
    g->origin[a] = opts->origin[a];
  }
  // ghost planes: nodes also below the box; the floor stays at its face
  g->ghost = opts->ghost_below;
  g->floor_z = opts->origin[2];
  g->dims[2] += g->ghost;
  g->origin[2] = opts->origin[2] - g->ghost * g->spacing[2];
  if (!dims_ok(g->dims)) {
    delete g;
    return set_err(ctx, GRIDFF_EINVAL, "grid needs at least 4 nodes per axis");
  }
  if (g->ghost > 0 && !(g->origin[2] > zmax + 0.1)) {
    const double low = g->origin[2];
    delete g;
    return set_err(ctx, GRIDFF_EINVAL,
                   "ghost planes reach z = %g, not above the substrate's highest atom (z = %g) by 0.1 A", low, zmax);
  }
  double alpha = opts->alpha > 0 ? opts->alpha : 1.5;
  double rcut = opts->rcut > 0 ? opts->rcut : 17.0;
  double tol = opts->ewald_tol > 0 ? opts->ewald_tol : 1e-10;
  double ercut = opts->ewald_rcut > 0 ? opts->ewald_rcut : 12.0;
  double s_tol = sqrt(-log(tol));
  double beta = s_tol / ercut;
  double kmax = 2.0 * beta * s_tol;
  double Lz = C[8];
  double ztop = g->origin[2] + g->spacing[2] * (g->dims[2] - 1);
  double zspan = std::max(ztop, zmax) - std::min(g->origin[2], zmin);
  if (charged && Lz - zspan < ercut) {
    delete g;
    return set_err(ctx, GRIDFF_EINVAL,
                   "Ewald height Lz = %g too small: needs >= %g (z span %g + real-space cutoff)",
                   Lz, zspan + ercut, zspan);
  }

  DevFree df;
  cudaStream_t s = ctx->stream;
  size_t n_nodes = (size_t)g->dims[0] * g->dims[1] * g->dims[2];
  double* vals = nullptr;
  const size_t vals_bytes = n_nodes * g->n_ch * sizeof(double);
  if (df.alloc(&vals, vals_bytes) != cudaSuccess) {
    delete g;
    return set_err(ctx, GRIDFF_ENOMEM, "cannot allocate %zu bytes of node values", vals_bytes);
  }
  auto bail = [&](gridff_status st) {
    gridff_grid_destroy(g);
    return st;
  };
  // substrate upload
  std::vector<D4> h_at(sub->n_atoms);
  std::vector<double2> h_re(sub->n_atoms);
  for (int j = 0; j < sub->n_atoms; ++j) {
    h_at[j] = D4{sub->xyz[3 * j], sub->xyz[3 * j + 1], sub->xyz[3 * j + 2], sub->q[j]};
    h_re[j] = make_double2(sub->R[j], sub->eps[j]);
  }
  D4* d_at = nullptr;
  double2* d_re = nullptr;
  if (df.alloc(&d_at, h_at.size() * sizeof(D4)) != cudaSuccess ||
      df.alloc(&d_re, h_re.size() * sizeof(double2)) != cudaSuccess)
    return bail(set_err(ctx, GRIDFF_ENOMEM, "substrate upload"));
  if (cudaMemcpyAsync(d_at, h_at.data(), h_at.size() * sizeof(D4), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(d_re, h_re.data(), h_re.size() * sizeof(double2), cudaMemcpyHostToDevice, s))
    return bail(set_err(ctx, GRIDFF_ECUDA, "substrate upload failed"));

  BuildParams p{};
  p.nx = g->dims[0];
  p.ny = g->dims[1];
  p.nz = g->dims[2];
  p.x0 = g->origin[0];
  p.y0 = g->origin[1];
  p.z0 = g->origin[2];
  p.dx = g->spacing[0];
  p.dy = g->spacing[1];
  p.dz = g->spacing[2];
  p.A1x = C[0];
  p.A1y = C[1];
  p.A2x = C[3];
  p.A2y = C[4];
  p.Lz = Lz;
  // in-plane image range: every image within (max node-atom in-plane distance + cutoff)
  {
    double xs[2] = {g->origin[0], g->origin[0] + opts->length[0]};
    double ys[2] = {g->origin[1], g->origin[1] + opts->length[1]};
    double dmax = 0.0;
    for (int j = 0; j < sub->n_atoms; ++j)
      for (double xx : xs)
        for (double yy : ys)
          dmax = std::max(dmax, hypot(xx - sub->xyz[3 * j], yy - sub->xyz[3 * j + 1]));
    double reach = dmax + std::max(rcut, charged ? ercut : 0.0);
    double h1 = fabs(area) / hypot(C[3], C[4]);   // distance between A1 lattice lines
    double h2 = fabs(area) / hypot(C[0], C[1]);
    p.n_img1 = (int)ceil(reach / h1);
    p.n_img2 = (int)ceil(reach / h2);
  }
  p.alpha = alpha;
  p.rcut2 = rcut * rcut;
  p.ercut2 = ercut * ercut;
  p.beta = beta;
  p.morse = (chans & GRIDFF_CH_P) ? 1 : 0;
  p.coulomb = (chans & GRIDFF_CH_C) ? 1 : 0;
  p.slotC = sC;
  p.slotP = sP;
  p.slotL = sL;
  double vol = fabs(area) * Lz;
  p.bg = -kPi * Qtot / (beta * beta * vol);
  p.dip = 4.0 * kPi * Mz / vol;
  // reciprocal lattice: B = 2 pi inv(cell)^T; for this cell B3 = (0, 0, 2 pi / Lz)
  double inv_area = 1.0 / area;
  p.B1x = 2 * kPi * C[4] * inv_area;
  p.B1y = -2 * kPi * C[3] * inv_area;
  p.B2x = -2 * kPi * C[1] * inv_area;
  p.B2y = 2 * kPi * C[0] * inv_area;
  double B3z = 2 * kPi / Lz;
  p.nzk = p.nz;

  RowInfo* d_rows = nullptr;
  double2* d_G = nullptr;
  if (p.coulomb) {
    int M1 = (int)ceil(kmax * hypot(C[0], C[1]) / (2 * kPi)) + 1;
    int M2 = (int)ceil(kmax * hypot(C[3], C[4]) / (2 * kPi)) + 1;
    int M3 = (int)ceil(kmax * Lz / (2 * kPi)) + 1;
    std::vector<RowInfo> rows;
    std::vector<int2> k2m;
    for (int m1 = -M1; m1 <= M1; ++m1) {
      int lo = 1 << 30, hi = -(1 << 30);
      for (int m2 = -M2; m2 <= M2; ++m2) {
        double kx = m1 * p.B1x + m2 * p.B2x, ky = m1 * p.B1y + m2 * p.B2y;
        if (kx * kx + ky * ky < kmax * kmax) {
          lo = std::min(lo, m2);
          hi = std::max(hi, m2);
        }
      }
      if (lo > hi) continue;
      rows.push_back(RowInfo{m1, lo, hi, (int)k2m.size()});
      for (int m2 = lo; m2 <= hi; ++m2) k2m.push_back(make_int2(m1, m2));
    }
    p.n_rows = (int)rows.size();
    int n_k2 = (int)k2m.size();
    int2* d_k2m = nullptr;
    double2* d_AS = nullptr;
    size_t n_as = (size_t)n_k2 * (2 * M3 + 1);
    if (df.alloc(&d_rows, rows.size() * sizeof(RowInfo)) != cudaSuccess ||
        df.alloc(&d_k2m, k2m.size() * sizeof(int2)) != cudaSuccess ||
        df.alloc(&d_AS, n_as * sizeof(double2)) != cudaSuccess ||
        df.alloc(&d_G, (size_t)n_k2 * p.nz * sizeof(double2)) != cudaSuccess)
      return bail(set_err(ctx, GRIDFF_ENOMEM, "reciprocal tables"));
    if (cudaMemcpyAsync(d_rows, rows.data(), rows.size() * sizeof(RowInfo), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_k2m, k2m.data(), k2m.size() * sizeof(int2), cudaMemcpyHostToDevice, s))
      return bail(set_err(ctx, GRIDFF_ECUDA, "table upload"));
    k_struct_kernel<<<(unsigned)((n_as + 127) / 128), 128, 0, s>>>(
        d_at, sub->n_atoms, d_k2m, n_k2, M3, p.B1x, p.B1y, p.B2x, p.B2y, B3z, kmax * kmax, beta,
        vol, d_AS);
    size_t n_g = (size_t)n_k2 * p.nz;
    k_zsum_kernel<<<(unsigned)((n_g + 127) / 128), 128, 0, s>>>(d_AS, n_k2, M3, B3z, p.z0, p.dz,
                                                                p.nz, d_G);
    if (cudaGetLastError() != cudaSuccess) return bail(set_err(ctx, GRIDFF_ECUDA, "reciprocal kernels"));
  }
  node_values_kernel<<<(unsigned)((n_nodes + kNodeThreads - 1) / kNodeThreads), kNodeThreads, 0,
                       s>>>(p, d_at, d_re, sub->n_atoms, d_rows, d_G, vals);
  if (cudaGetLastError() != cudaSuccess) return bail(set_err(ctx, GRIDFF_ECUDA, "node kernel launch"));
  if (opts->keep_f64) {
    if (cudaMalloc(&g->f64_values, n_nodes * g->n_ch * sizeof(double)) != cudaSuccess)
      return bail(set_err(ctx, GRIDFF_ENOMEM, "kept node values"));
    if (cudaMemcpyAsync(g->f64_values, vals, n_nodes * g->n_ch * sizeof(double),
                        cudaMemcpyDeviceToDevice, s))
      return bail(set_err(ctx, GRIDFF_ECUDA, "copy of node values"));
  }
  gridff_status st = fit_and_pack(ctx, g, vals, df);
  if (st != GRIDFF_OK) return bail(st);
  if (opts->keep_f64) {
    g->f64_coefs = vals;
    df.release(vals);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(set_err(ctx, GRIDFF_ECUDA, "grid build: %s", cudaGetErrorString(e)));
  *out = g;
  return GRIDFF_OK;
}

gridff_status gridff_grid_from_coefs(gridff_ctx* ctx, const double origin[3], const double spacing[3],
                                     const int32_t dims[3], int32_t channels, const double* coefs,
                                     int32_t storage, gridff_grid** out) {
  NvtxRange nvtx_range("gridff_grid_from_coefs");
  if (!ctx || !origin || !spacing || !dims || !coefs || !out)
    return set_err(ctx, GRIDFF_EINVAL, "null argument");
  *out = nullptr;
  if (!storage_ok(storage)) return set_err(ctx, GRIDFF_ENOTSUP, "storage not supported");
  if (!dims_ok(dims)) return set_err(ctx, GRIDFF_EINVAL, "grid needs at least 4 nodes per axis");
  if (!(channels & 7) || (channels & ~7)) return set_err(ctx, GRIDFF_EINVAL, "bad channel mask");
  for (int a = 0; a < 3; ++a)
    if (!(spacing[a] > 0)) return set_err(ctx, GRIDFF_EINVAL, "spacing must be > 0");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  gridff_grid* g = new gridff_grid();
  g->ctx = ctx;
  g->device = ctx->device;
  g->channels = channels;
  g->storage = storage;
  int sC, sP, sL;
  channel_slots(channels, sC, sP, sL, g->n_ch);
  for (int a = 0; a < 3; ++a) {
    g->dims[a] = dims[a];
    g->origin[a] = origin[a];
    g->spacing[a] = spacing[a];
  }
  g->floor_z = origin[2];
  size_t n = (size_t)dims[0] * dims[1] * dims[2] * g->n_ch;
  DevFree df;
  double* d = nullptr;
  if (df.alloc(&d, n * sizeof(double)) != cudaSuccess) {
    delete g;
    return set_err(ctx, GRIDFF_ENOMEM, "coefficient upload");
  }
  if (cudaMemcpyAsync(d, coefs, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
    delete g;
    return set_err(ctx, GRIDFF_ECUDA, "coefficient upload");
  }
  // reuse the packing step only (coefficients are given)
  gridff_status pst = pack_records(ctx, g, d);
  if (pst != GRIDFF_OK) {
    gridff_grid_destroy(g);
    return pst;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    gridff_grid_destroy(g);
    return set_err(ctx, GRIDFF_ECUDA, "pack: %s", cudaGetErrorString(e));
  }
  *out = g;
  return GRIDFF_OK;
}

gridff_status gridff_fit_coefs_noalloc(gridff_ctx* ctx, const double* values, double* coefs,
                                       const int32_t dims[3], int32_t n_channels, int flags) {
  NvtxRange nvtx_range("gridff_fit_coefs_noalloc");
  if (!ctx || !values || !coefs || !dims) return set_err(ctx, GRIDFF_EINVAL, "null argument");
  if (n_channels < 1) return set_err(ctx, GRIDFF_EINVAL, "n_channels must be >= 1");
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 4 || dims[a] > kNoAllocMaxN)
      return set_err(ctx, GRIDFF_EINVAL,
                     "gridff_fit_coefs_noalloc: dims[%d] = %d outside 4..%d (the size of its fixed "
                     "device table)", a, dims[a], kNoAllocMaxN);
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)dims[0] * dims[1] * dims[2] * n_channels * sizeof(double);
  // both arrays must be memory of this context's device (a host pointer
  // handed to the line-solve kernels would be an out-of-bounds access)
  for (const void* p : {(const void*)values, (const void*)coefs}) {
    cudaPointerAttributes pa{};
    const cudaError_t pe = cudaPointerGetAttributes(&pa, p);
    if (pe != cudaSuccess) cudaGetLastError();
    if (pe != cudaSuccess || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
        (pa.type == cudaMemoryTypeDevice && pa.device != ctx->device))
      return set_err(ctx, GRIDFF_EINVAL, "gridff_fit_coefs_noalloc: %s is not memory of device %d",
                     p == (const void*)values ? "values" : "coefs", ctx->device);
  }
  {
    // in place (equal pointers) is allowed; partly overlapping ranges are not
    const char *v0 = (const char*)values, *c0 = (const char*)coefs;
    if (v0 != c0 && v0 < c0 + bytes && c0 < v0 + bytes)
      return set_err(ctx, GRIDFF_EINVAL, "gridff_fit_coefs_noalloc: values and coefs overlap without being equal");
  }
  cudaError_t e;
  double* tab = noalloc_tables_address(ctx->device, &e);
  if (!tab) return set_err(ctx, GRIDFF_ECUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
  cudaStream_t s = ctx->stream;
  int nx = dims[0], ny = dims[1], nz = dims[2];
  long long N = (long long)nx * ny * nz;
  if (values != coefs)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(coefs, values, (size_t)N * n_channels * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
  noalloc_tables_kernel<<<1, 32, 0, s>>>(tab, nx, ny, nz);
  const int TB = 128;
  long long lines = (long long)n_channels * nx * ny;   // z: contiguous lines
  noalloc_line_kernel<<<(unsigned)((lines + TB - 1) / TB), TB, 0, s>>>(
      coefs, nz, 1, lines, 1, 0, nz, tab + 2 * kNoAllocStride, 0);
  lines = (long long)n_channels * nx * nz;             // y
  noalloc_line_kernel<<<(unsigned)((lines + TB - 1) / TB), TB, 0, s>>>(
      coefs, ny, nz, lines, nz, 1, (long long)ny * nz, tab + kNoAllocStride, 1);
  lines = (long long)n_channels * ny * nz;             // x
  noalloc_line_kernel<<<(unsigned)((lines + TB - 1) / TB), TB, 0, s>>>(
      coefs, nx, (long long)ny * nz, lines, ny * nz, 1, N, tab, 1);
  GRIDFF_CUDA(ctx, cudaGetLastError());
  if (!(flags & GRIDFF_ASYNC)) GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

gridff_status gridff_grid_floor(const gridff_grid* g, double* z_floor) {
  if (!g || !z_floor) return GRIDFF_EINVAL;
  *z_floor = g->floor_z;
  return GRIDFF_OK;
}

gridff_status gridff_grid_storage(const gridff_grid* g, int32_t* storage, float scales[3]) {
  if (!g) return GRIDFF_EINVAL;
  if (storage) *storage = g->storage;
  if (scales)
    for (int c = 0; c < 3; ++c) scales[c] = g->scale[c];
  return GRIDFF_OK;
}

gridff_status gridff_grid_info(const gridff_grid* g, int32_t dims[3], double origin[3],
                               double spacing[3], int32_t* channels, size_t* device_bytes) {
  if (!g) return GRIDFF_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (dims) dims[a] = g->dims[a];
    if (origin) origin[a] = g->origin[a];
    if (spacing) spacing[a] = g->spacing[a];
  }
  if (channels) *channels = g->channels;
  if (device_bytes) *device_bytes = g->rec_bytes;
  return GRIDFF_OK;
}

gridff_status gridff_grid_download_f64(const gridff_grid* g, int what, double* host_out) {
  if (!g || !host_out) return GRIDFF_EINVAL;
  const double* src = what == 0 ? g->f64_values : what == 1 ? g->f64_coefs : nullptr;
  if (!src) return set_err(g->ctx, GRIDFF_EINVAL, "FP64 data not kept (set keep_f64 at build)");
  size_t n = (size_t)g->dims[0] * g->dims[1] * g->dims[2] * g->n_ch;
  GRIDFF_CUDA(g->ctx, cudaSetDevice(g->ctx->device));
  GRIDFF_CUDA(g->ctx, cudaMemcpyAsync(host_out, src, n * sizeof(double), cudaMemcpyDeviceToHost,
                                      g->ctx->stream));
  GRIDFF_CUDA(g->ctx, cudaStreamSynchronize(g->ctx->stream));
  return GRIDFF_OK;
}

void gridff_grid_destroy(gridff_grid* g) {
  if (!g) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(g->device);
  if (g->rec) cudaFree(g->rec);
  if (g->f64_values) cudaFree(g->f64_values);
  if (g->f64_coefs) cudaFree(g->f64_coefs);
  cudaSetDevice(prev);
  cudaGetLastError();   // leave no error of this teardown behind
  delete g;
}

}  // extern "C"
