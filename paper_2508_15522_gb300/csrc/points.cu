// Grid interpolation alone at independent points, binned by cell (the
// GRIDFF_POINTS_BINNED path of gridff_eval_points): steps a2-a6 of the path
// (fold into the tile, cell and fractional coordinates, cubic B-spline
// weights, gather of the 4x4x4 stencil, contraction, channel combination;
// Sec. 4, Sec. 5, Eqs. E, E_Coulomb, V_Morse) for points in no particular
// order.
//
// Points arrive in arbitrary order; gathered directly, every evaluation
// reads 16 scattered 64-byte runs and the L1 data path that receives those
// sectors limits the rate.  Here the points are first put in the order of
// their cell (a counting sort on the device), so the 32 points of a warp lie
// in a few neighbouring cells of one grid column and each warp-wide load of
// a stencil record touches one or two cache lines instead of 32.  Then one
// lane evaluates one point: it walks the 16 (x, y) runs of its stencil
// (four consecutive records along z each), combines the channels per node
// with the point's factors (Q, P, L), contracts along z (value and
// z-derivative), then along y and x (the 16/4/1 passes of Sec. 5).
//
// Sort: bin = (x cell, y cell, z cell / 4) in the records' memory order
// (z fastest), plus one bin for points above the grid (no gather).
//   1. count: every point adds itself to its bin (its rank = the count
//      before it);
//   2. exclusive scan of the bin counts (three passes: tile sums, scan of
//      the tile sums in one block, scan inside each tile);
//   3. scatter: the point's position, factors and index go to sorted
//      position = start of the bin + rank (one 32-byte record);
//   4. evaluate the records in order, results written at the original index.
#include <math.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "interp.cuh"

namespace {

constexpr int kZBin = 4;            // z cells per bin
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 4 * kScanThreads;   // counts per scan tile
constexpr int kEvalThreads = 256;

// Bin of a point: cells (ix, iy, iz / kZBin) in x-major, z-fastest order;
// points above the grid or with a non-finite coordinate go to the last bin,
// nx ny nzb, and gather nothing.
__device__ __forceinline__ int bin_of(const GridView& g, int nzb, float x, float y, float z) {
  int fl = 0;
  const bool fin = isfinite(x) && isfinite(y) && isfinite(z);
  const Cell c = locate(g, fin, x, y, z, fl);
  if (!c.inside) return g.nx * g.ny * nzb;
  return (c.ix * g.ny + c.iy) * nzb + c.iz / kZBin;
}

__global__ void bin_count_kernel(GridView g, int nzb, int n, const float* __restrict__ xyz, int* __restrict__ counts,
                                 int2* __restrict__ keyrank) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int key = bin_of(g, nzb, __ldg(&xyz[3 * (size_t)i]), __ldg(&xyz[3 * (size_t)i + 1]),
                         __ldg(&xyz[3 * (size_t)i + 2]));
  keyrank[i] = make_int2(key, atomicAdd(&counts[key], 1));
}

// Exclusive prefix sum over the block (kScanThreads threads) of one value
// per thread; returns this thread's prefix and sets *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    int x = s_warp[lane];
    int xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    s_warp[lane] = xi - x;        // exclusive prefix of warp `lane`
    if (lane == 31) s_warp[32] = xi;
  }
  __syncthreads();
  const int out = s_warp[w] + inc - v;
  *total = s_warp[32];
  __syncthreads();                // s_warp may be reused by the caller
  return out;
}

// Pass 1: sum of every tile of kScanTile counts.
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int* __restrict__ counts, int nb,
                                                                   int* __restrict__ tile_sums) {
  __shared__ int s_warp[33];
  const int base = blockIdx.x * kScanTile + 4 * threadIdx.x;
  int v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (base + k < nb) v += counts[base + k];
  int total;
  block_exclusive_scan(v, s_warp, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Pass 2 (one block): exclusive scan of the tile sums in place.
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(int* __restrict__ tile_sums, int n_tiles) {
  __shared__ int s_warp[33];
  const int per = (n_tiles + kScanThreads - 1) / kScanThreads;
  const int b = threadIdx.x * per;
  int v = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < n_tiles) v += tile_sums[b + k];
  int total;
  int run = block_exclusive_scan(v, s_warp, &total);
  for (int k = 0; k < per; ++k)
    if (b + k < n_tiles) {
      const int t = tile_sums[b + k];
      tile_sums[b + k] = run;
      run += t;
    }
}

// Pass 3: exclusive scan inside every tile, offset by the tile's prefix.
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int* __restrict__ counts, int nb,
                                                                   const int* __restrict__ tile_prefix,
                                                                   int* __restrict__ start) {
  __shared__ int s_warp[33];
  const int base = blockIdx.x * kScanTile + 4 * threadIdx.x;
  int c[4], v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c[k] = base + k < nb ? counts[base + k] : 0;
    v += c[k];
  }
  int total;
  int run = block_exclusive_scan(v, s_warp, &total) + tile_prefix[blockIdx.x];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (base + k < nb) {
      start[base + k] = run;
      run += c[k];
    }
}

// A point in sorted order: position and charge, then the two Morse factors
// and the point's original index (32 bytes, one sector).
struct SortedPoint {
  float4 xyzq;
  float4 pli;   // P, L, index (bit pattern), unused
};

__global__ void bin_scatter_kernel(int n, const int2* __restrict__ keyrank, const int* __restrict__ start,
                                   const float* __restrict__ xyz, const float* __restrict__ qpl,
                                   SortedPoint* __restrict__ sorted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 kr = keyrank[i];
  SortedPoint p;
  p.xyzq = make_float4(xyz[3 * (size_t)i], xyz[3 * (size_t)i + 1], xyz[3 * (size_t)i + 2], qpl[3 * (size_t)i]);
  p.pli = make_float4(qpl[3 * (size_t)i + 1], qpl[3 * (size_t)i + 2], __int_as_float(i), 0.f);
  sorted[start[kr.x] + kr.y] = p;
}

// Channel-combined values of one z-run (four consecutive records from
// `base`) for the grid's record kind, with the point's factors (channel
// scales folded in): c_k = fc C_k + fp P_k + fl L_k.
template <int KIND>
__device__ __forceinline__ void run_values(const GridView& g, long long base, float fc, float fp, float fl,
                                           float c[4]) {
  switch (KIND >= 0 ? KIND : g.kind) {
    case REC_F32x4: {
      const float4* p = (const float4*)g.rec + base;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 r = __ldg(p + k);
        c[k] = fmaf(fc, r.x, fmaf(fp, r.y, fl * r.z));
      }
      break;
    }
    case REC_F32x2: {
      const float2* p = (const float2*)g.rec + base;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 r = __ldg(p + k);
        c[k] = fmaf(fp, r.x, fl * r.y);
      }
      break;
    }
    case REC_F16x4:
    case REC_BF16x4: {
      const uint2* p = (const uint2*)g.rec + base;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint2 r = __ldg(p + k);
        float2 a, b;
        if (g.kind == REC_F16x4) {
          a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
          b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
        } else {
          a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
          b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
        }
        c[k] = fmaf(fc, a.x, fmaf(fp, a.y, fl * b.x));
      }
      break;
    }
    default: {   // REC_F16x2, REC_BF16x2
      const unsigned* p = (const unsigned*)g.rec + base;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned r = __ldg(p + k);
        const float2 a = g.kind == REC_F16x2 ? __half22float2(*reinterpret_cast<const __half2*>(&r))
                                             : __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r));
        c[k] = fmaf(fp, a.x, fl * a.y);
      }
      break;
    }
  }
}

#ifndef GRIDFF_SORTED_MINB
#define GRIDFF_SORTED_MINB 4
#endif
// One lane per point, points taken in sorted order (contiguous records),
// results written at the point's own index.
template <int KIND>
__global__ void __launch_bounds__(kEvalThreads, GRIDFF_SORTED_MINB)
eval_sorted_kernel(GridView g, int n, const SortedPoint* __restrict__ sorted, float* __restrict__ E,
                   float* __restrict__ F, int* __restrict__ st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float4 a4 = __ldg(&sorted[j].xyzq), b4 = __ldg(&sorted[j].pli);
  const int i = __float_as_int(b4.z);
  const float x = a4.x, y = a4.y, z = a4.z;
  const float fc = a4.w * g.sC, fp = b4.x * g.sP, fl = b4.y * g.sL;
  // a non-finite position is reported and evaluates to zero
  const bool fin = isfinite(x) && isfinite(y) && isfinite(z);
  int flags = fin ? 0 : GRIDFF_REP_NONFINITE;
  const Cell cl = locate(g, fin, x, y, z, flags);
  float e = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  if (cl.inside) {
    float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
    bspline_weights(cl.tx, wx, dwx);
    bspline_weights(cl.ty, wy, dwy);
    bspline_weights(cl.tz, wz, dwz);
    // padded record (ix, iy, iz) holds logical node (ix - 1, iy - 1, iz - 1):
    // the first record of the stencil's run (a, b) is base + a sx + b nzp
    const long long base = ((long long)cl.ix * g.nyp + cl.iy) * g.nzp + cl.iz;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float sv = 0.f, sdy = 0.f, sdz = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float c[4];
        run_values<KIND>(g, base + a * g.sx + b * g.nzp, fc, fp, fl, c);
        // 16 passes along z (value and z-derivative of run (a, b)) ...
        const float zv = fmaf(wz[0], c[0], fmaf(wz[1], c[1], fmaf(wz[2], c[2], wz[3] * c[3])));
        const float zd = fmaf(dwz[0], c[0], fmaf(dwz[1], c[1], fmaf(dwz[2], c[2], dwz[3] * c[3])));
        // ... 4 along y ...
        sv = fmaf(wy[b], zv, sv);
        sdy = fmaf(dwy[b], zv, sdy);
        sdz = fmaf(wy[b], zd, sdz);
      }
      // ... 1 along x
      e = fmaf(wx[a], sv, e);
      gx = fmaf(dwx[a], sv, gx);
      gy = fmaf(wx[a], sdy, gy);
      gz = fmaf(wx[a], sdz, gz);
    }
  }
  const float fx = -gx * g.inv_dx, fy = -gy * g.inv_dy, fz = -gz * g.inv_dz;
  E[i] = e;
  F[3 * (size_t)i] = fx;
  F[3 * (size_t)i + 1] = fy;
  F[3 * (size_t)i + 2] = fz;
  if (st)
    st[i] = flags | (isfinite(fx) && isfinite(fy) && isfinite(fz) && isfinite(e) ? 0 : GRIDFF_REP_NONFINITE);
}

}  // namespace

// Enqueue the binned evaluation of n points (device arrays) on the
// context stream; scratch comes from the stream-ordered pool and is
// released on the stream.  Called by gridff_eval_points.
gridff_status enqueue_eval_points_binned(gridff_ctx* ctx, const gridff_grid* grid, int64_t n, const float* xyz,
                                         const float* qpl, float* E, float* F, int32_t* status) {
  const GridView g = grid->view();
  const int nzb = (g.nz - 1 + kZBin - 1) / kZBin;   // z cells 0 .. nz - 2
  const long long nb_ll = (long long)g.nx * g.ny * nzb + 1;
  if (n >= (1LL << 31) || nb_ll >= (1LL << 30))
    return set_err(ctx, GRIDFF_ENOTSUP, "binned point evaluation: %lld points / %lld bins exceed its index range",
                   (long long)n, nb_ll);
  const int nb = (int)nb_ll, ni = (int)n;
  const int n_tiles = (nb + kScanTile - 1) / kScanTile;
  cudaStream_t s = ctx->stream;
  const size_t b_counts = ((size_t)nb * 4 + 255) & ~size_t(255), b_tiles = ((size_t)n_tiles * 4 + 255) & ~size_t(255),
               b_kr = ((size_t)ni * 8 + 255) & ~size_t(255), b_sorted = (size_t)ni * sizeof(SortedPoint);
  char* scratch = nullptr;
  GRIDFF_CUDA(ctx, cudaMallocAsync((void**)&scratch, 2 * b_counts + b_tiles + b_kr + b_sorted, s));
  int* counts = (int*)scratch;
  int* start = (int*)(scratch + b_counts);
  int* tiles = (int*)(scratch + 2 * b_counts);
  int2* keyrank = (int2*)(scratch + 2 * b_counts + b_tiles);
  SortedPoint* sorted = (SortedPoint*)(scratch + 2 * b_counts + b_tiles + b_kr);
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nb * 4, s);
  const int pb = (ni + 255) / 256;
  if (e == cudaSuccess) {
    bin_count_kernel<<<pb, 256, 0, s>>>(g, nzb, ni, xyz, counts, keyrank);
    scan_tiles_kernel<<<n_tiles, kScanThreads, 0, s>>>(counts, nb, tiles);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(tiles, n_tiles);
    scan_apply_kernel<<<n_tiles, kScanThreads, 0, s>>>(counts, nb, tiles, start);
    bin_scatter_kernel<<<pb, 256, 0, s>>>(ni, keyrank, start, xyz, qpl, sorted);
    const int eb = (ni + kEvalThreads - 1) / kEvalThreads;
    if (grid->kind == REC_F32x4)
      eval_sorted_kernel<REC_F32x4><<<eb, kEvalThreads, 0, s>>>(g, ni, sorted, E, F, status);
    else
      eval_sorted_kernel<-1><<<eb, kEvalThreads, 0, s>>>(g, ni, sorted, E, F, status);
    e = cudaGetLastError();
  }
  const cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "binned point evaluation: %s", cudaGetErrorString(e));
  return GRIDFF_OK;
}
