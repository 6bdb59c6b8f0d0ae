// Sampling support around the relaxation: random starting poses of rigid
// replicas (Sec. 7: molecules start from random placements over the
// surface) and the RMSD uniqueness filter of relaxed minima (Sec. 7: two
// minima are the same structure when their RMSD is below a threshold,
// 0.1 A in the paper, which covers conformation, site and orientation).
#include <math.h>

#include "internal.h"
#include "trace.h"

namespace {

// Uniform [0, 1) draw j of row r (24 bits).
__device__ __forceinline__ float uniform01(unsigned long long seed, int r, int j) {
  return uniform_of(splitmix64(seed ^ splitmix64((unsigned long long)r * 64 + j)));
}

// One warp per replica: centre of mass uniform over the tile and over
// [z_lo, z_hi), orientation uniform on SO(3) (Shoemake's subgroup
// algorithm), then lifted so that the lowest atom is at least z_floor.
__global__ void random_poses_kernel(TemplateView tv, const int* __restrict__ rep_tmpl, int n_rep,
                                    unsigned long long seed, float ox, float oy, float Lx, float Ly, float z_lo,
                                    float z_hi, float z_floor, float* __restrict__ pose, float* __restrict__ vel) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_rep) return;
  const float u1 = uniform01(seed, r, 0), u2 = uniform01(seed, r, 1), u3 = uniform01(seed, r, 2);
  const float a = sqrtf(1.f - u1), b = sqrtf(u1);
  float s2, c2, s3, c3;
  sincospif(2.f * u2, &s2, &c2);
  sincospif(2.f * u3, &s3, &c3);
  const float qw = b * c3, qx = a * s2, qy = a * c2, qz = b * s3;
  float Rm[9];
  quat_rot(qw, qx, qy, qz, Rm);
  const float cx = ox + Lx * uniform01(seed, r, 3);
  const float cy = oy + Ly * uniform01(seed, r, 4);
  float cz = z_lo + (z_hi - z_lo) * uniform01(seed, r, 5);
  const int t = rep_tmpl[r];
  const int n = tv.natoms[t], ab = tv.atom_off[t];
  float lowest = INFINITY;
  for (int i = lane; i < n; i += 32) {
    const float4 bp = tv.body[ab + i];
    lowest = fminf(lowest, Rm[6] * bp.x + Rm[7] * bp.y + Rm[8] * bp.z);
  }
  for (int o = 16; o; o >>= 1) lowest = fminf(lowest, __shfl_xor_sync(0xffffffffu, lowest, o));
  if (lane == 0) {
    cz = fmaxf(cz, z_floor - lowest);
    float* p = pose + 7 * (size_t)r;
    p[0] = cx; p[1] = cy; p[2] = cz;
    p[3] = qw; p[4] = qx; p[5] = qy; p[6] = qz;
    float* v = vel + 6 * (size_t)r;
    for (int k = 0; k < 6; ++k) v[k] = 0.f;
  }
}

// Body-frame moments of a template: mean position bbar and second moment
// S = (1/n) sum b b^T.  For rigid poses (c1, R1) and (c2, R2) with
// D = R1 - R2 and dc = c1 - c2 the mean squared atom displacement is
//   |dc|^2 + 2 dc . (D bbar) + sum_kl (D^T D)_kl S_kl.
struct Moments {
  float bbar[3];
  float S[9];
};

__global__ void moments_kernel(TemplateView tv, int t, Moments* out) {
  const int lane = threadIdx.x;
  const int n = tv.natoms[t], ab = tv.atom_off[t];
  float m[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = lane; i < n; i += 32) {
    const float4 b = tv.body[ab + i];
    const float v[3] = {b.x, b.y, b.z};
    for (int k = 0; k < 3; ++k) {
      m[k] += v[k];
      for (int l = 0; l < 3; ++l) m[3 + 3 * k + l] += v[k] * v[l];
    }
  }
  for (int k = 0; k < 12; ++k)
    for (int o = 16; o; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
  if (lane == 0) {
    for (int k = 0; k < 3; ++k) out->bbar[k] = m[k] / n;
    for (int k = 0; k < 9; ++k) out->S[k] = m[3 + k] / n;
  }
}

// dup_of[i] = smallest j < i with msd(i, j) < thr2 (centre of mass by the
// minimum image in x, y), else -1.  One warp per i; lane l tests j = j0 + l.
__global__ void dedupe_kernel(const Moments* __restrict__ mom, const float* __restrict__ pose, int n, float Lx,
                              float Ly, float thr2, int* __restrict__ dup_of) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const Moments M = *mom;
  const float* pi = pose + 7 * (size_t)i;
  float Ri[9];
  {
    const float w = pi[3], x = pi[4], y = pi[5], z = pi[6];
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    quat_rot(w * inv, x * inv, y * inv, z * inv, Ri);
  }
  int found = -1;
  for (int j0 = 0; j0 < i && found < 0; j0 += 32) {
    const int j = j0 + lane;
    bool hit = false;
    if (j < i) {
      const float* pj = pose + 7 * (size_t)j;
      float Rj[9];
      const float w = pj[3], x = pj[4], y = pj[5], z = pj[6];
      const float inv = rsqrtf(w * w + x * x + y * y + z * z);
      quat_rot(w * inv, x * inv, y * inv, z * inv, Rj);
      float dc[3] = {pi[0] - pj[0], pi[1] - pj[1], pi[2] - pj[2]};
      dc[0] -= Lx * rintf(dc[0] / Lx);
      dc[1] -= Ly * rintf(dc[1] / Ly);
      float D[9];
      for (int k = 0; k < 9; ++k) D[k] = Ri[k] - Rj[k];
      float msd = dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2];
      for (int k = 0; k < 3; ++k) {
        const float db = D[3 * k] * M.bbar[0] + D[3 * k + 1] * M.bbar[1] + D[3 * k + 2] * M.bbar[2];
        msd += 2.f * dc[k] * db;
      }
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          const float dtd = D[k] * D[l] + D[3 + k] * D[3 + l] + D[6 + k] * D[6 + l];
          msd += dtd * M.S[3 * k + l];
        }
      hit = msd < thr2;
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if (b) found = j0 + __ffs(b) - 1;
  }
  if (lane == 0) dup_of[i] = found;
}

// Mean x, y of each structure (for the minimum-image shift).
__global__ void centers_kernel(const float* __restrict__ xyz, int na, int n, float2* __restrict__ cen) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = xyz + (size_t)i * na * 3;
  float sx = 0.f, sy = 0.f;
  for (int a = 0; a < na; ++a) {
    sx += p[3 * a];
    sy += p[3 * a + 1];
  }
  cen[i] = make_float2(sx / na, sy / na);
}

// dup_of[i] = smallest j < i whose mean squared atom displacement from i,
// after shifting j by whole tile periods toward i's mean position, is below
// thr2; else -1.  One warp per i; lane l tests j = j0 + l over all atoms.
__global__ void dedupe_xyz_kernel(const float* __restrict__ xyz, const float2* __restrict__ cen, int na, int n,
                                  float Lx, float Ly, float thr2, int* __restrict__ dup_of) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float* pi = xyz + (size_t)i * na * 3;
  const float2 ci = cen[i];
  const float lim = thr2 * na;
  int found = -1;
  for (int j0 = 0; j0 < i && found < 0; j0 += 32) {
    const int j = j0 + lane;
    bool hit = false;
    if (j < i) {
      const float2 cj = cen[j];
      const float tx = Lx * rintf((ci.x - cj.x) / Lx), ty = Ly * rintf((ci.y - cj.y) / Ly);
      const float* pj = xyz + (size_t)j * na * 3;
      float ss = 0.f;
      for (int a = 0; a < na && ss < lim; ++a) {
        const float dx = pi[3 * a] - pj[3 * a] - tx, dy = pi[3 * a + 1] - pj[3 * a + 1] - ty;
        const float dz = pi[3 * a + 2] - pj[3 * a + 2];
        ss += dx * dx + dy * dy + dz * dz;
      }
      hit = ss < lim;
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if (b) found = j0 + __ffs(b) - 1;
  }
  if (lane == 0) dup_of[i] = found;
}

}  // namespace

extern "C" {

gridff_status gridff_random_poses(gridff_replicas* R, uint64_t seed, const double origin_xy[2],
                                  const double tile_xy[2], double z_lo, double z_hi, double z_floor) {
  NvtxRange nvtx_range("gridff_random_poses");
  if (!R || !origin_xy || !tile_xy) return GRIDFF_EINVAL;
  gridff_ctx* ctx = R->ctx;
  if (!R->rigid) return set_err(ctx, GRIDFF_ENOTSUP, "random poses are drawn for rigid replicas");
  if (!(tile_xy[0] > 0 && tile_xy[1] > 0 && z_hi >= z_lo))
    return set_err(ctx, GRIDFF_EINVAL, "tile must be positive and z_hi >= z_lo");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const int threads = 128;
  const unsigned blocks = (unsigned)(((long long)R->n_rep * 32 + threads - 1) / threads);
  random_poses_kernel<<<blocks, threads, 0, ctx->stream>>>(
      R->tv, R->rep_tmpl, R->n_rep, (unsigned long long)seed, (float)origin_xy[0], (float)origin_xy[1],
      (float)tile_xy[0], (float)tile_xy[1], (float)z_lo, (float)z_hi, (float)z_floor, R->x, R->v);
  GRIDFF_CUDA(ctx, cudaGetLastError());
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return GRIDFF_OK;
}

gridff_status gridff_rmsd_unique(gridff_replicas* R, int32_t tmpl, int32_t n, const float* poses,
                                 const double tile_xy[2], double threshold, int32_t* dup_of, int flags) {
  NvtxRange nvtx_range("gridff_rmsd_unique");
  if (!R || !tile_xy || n < 0 || (n > 0 && (!poses || !dup_of))) return GRIDFF_EINVAL;
  gridff_ctx* ctx = R->ctx;
  if (tmpl < 0 || tmpl >= R->n_tmpl) return set_err(ctx, GRIDFF_EINVAL, "template %d out of range", tmpl);
  if (!(threshold > 0) || !(tile_xy[0] > 0 && tile_xy[1] > 0))
    return set_err(ctx, GRIDFF_EINVAL, "threshold and tile must be positive");
  if (n == 0) return GRIDFF_OK;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const bool dev = flags & GRIDFF_DEVICE_PTRS;
  const size_t pose_bytes = 7 * (size_t)n * sizeof(float), dup_bytes = (size_t)n * sizeof(int32_t);
  char* buf = nullptr;
  const size_t mom_off = 0, pose_off = 256, dup_off = pose_off + ((pose_bytes + 255) & ~(size_t)255);
  GRIDFF_CUDA(ctx, cudaMallocAsync((void**)&buf, dup_off + dup_bytes, s));
  Moments* mom = (Moments*)(buf + mom_off);
  const float* p = dev ? poses : (const float*)(buf + pose_off);
  int* d = dev ? dup_of : (int*)(buf + dup_off);
  gridff_status st = GRIDFF_OK;
  cudaError_t e = cudaSuccess;
  if (!dev) e = cudaMemcpyAsync(buf + pose_off, poses, pose_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    moments_kernel<<<1, 32, 0, s>>>(R->tv, tmpl, mom);
    const int threads = 128;
    dedupe_kernel<<<(unsigned)(((long long)n * 32 + threads - 1) / threads), threads, 0, s>>>(
        mom, p, n, (float)tile_xy[0], (float)tile_xy[1], (float)(threshold * threshold), d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(dup_of, d, dup_bytes, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess && !(dev && (flags & GRIDFF_ASYNC))) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) st = set_err(ctx, GRIDFF_ECUDA, "rmsd_unique: %s", cudaGetErrorString(e));
  return st;
}

}  // extern "C"

extern "C" gridff_status gridff_rmsd_unique_xyz(gridff_ctx* ctx, int32_t na, int32_t n, const float* xyz,
                                                const double tile_xy[2], double threshold, int32_t* dup_of,
                                                int flags) {
  NvtxRange nvtx_range("gridff_rmsd_unique_xyz");
  if (!ctx || !tile_xy || n < 0 || (n > 0 && (!xyz || !dup_of))) return set_err(ctx, GRIDFF_EINVAL, "null argument");
  if (na < 1 || na > GRIDFF_MAX_ATOMS) return set_err(ctx, GRIDFF_EINVAL, "n_atoms %d outside 1..%d", na, GRIDFF_MAX_ATOMS);
  if (!(threshold > 0) || !(tile_xy[0] > 0 && tile_xy[1] > 0))
    return set_err(ctx, GRIDFF_EINVAL, "threshold and tile must be positive");
  if (n == 0) return GRIDFF_OK;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const bool dev = flags & GRIDFF_DEVICE_PTRS;
  const size_t xyz_bytes = (size_t)n * na * 3 * sizeof(float), dup_bytes = (size_t)n * sizeof(int32_t);
  const size_t cen_off = 0, xyz_off = ((size_t)n * sizeof(float2) + 255) & ~(size_t)255;
  const size_t dup_off = xyz_off + ((xyz_bytes + 255) & ~(size_t)255);
  char* buf = nullptr;
  GRIDFF_CUDA(ctx, cudaMallocAsync((void**)&buf, dup_off + dup_bytes, s));
  const float* p = dev ? xyz : (const float*)(buf + xyz_off);
  int* d = dev ? dup_of : (int*)(buf + dup_off);
  float2* cen = (float2*)(buf + cen_off);
  cudaError_t e = cudaSuccess;
  if (!dev) e = cudaMemcpyAsync(buf + xyz_off, xyz, xyz_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    centers_kernel<<<(n + 127) / 128, 128, 0, s>>>(p, na, n, cen);
    dedupe_xyz_kernel<<<(unsigned)(((long long)n * 32 + 127) / 128), 128, 0, s>>>(
        p, cen, na, n, (float)tile_xy[0], (float)tile_xy[1], (float)(threshold * threshold), d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(dup_of, d, dup_bytes, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess && !(dev && (flags & GRIDFF_ASYNC))) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "rmsd_unique_xyz: %s", cudaGetErrorString(e));
  return GRIDFF_OK;
}
