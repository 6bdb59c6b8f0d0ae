// Poses of flexible molecules: the builder (centre of mass, orientation
// quaternion and torsion angles -> atom positions) and its inverse (the
// pose of a relaxed structure, used as a training target of the learned
// pose proposal, Sec. 7 starting configurations).  The rotatable bonds and
// their reference quadruples come from replicas.cu (template_rotors); the
// pose layout is the proposal network's output (GRIDFF_MLP_OUT floats).
#include <math.h>

#include "internal.h"
#include "trace.h"

namespace {

constexpr int kPoseWarps = 4;
constexpr int kPoseLen = GRIDFF_MLP_OUT;   // 3 centre + 4 quaternion + 12 torsions
constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ float3 ldp(const float* s, int i) { return make_float3(s[3 * i], s[3 * i + 1], s[3 * i + 2]); }
__device__ __forceinline__ float3 dif(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dotp(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 crossp(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Dihedral of a-b-c-d: atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3)) with
// b1 = b - a, b2 = c - b, b3 = d - c (IUPAC sign).
__device__ float dihedral_of(float3 a, float3 b, float3 c, float3 d) {
  const float3 b1 = dif(b, a), b2 = dif(c, b), b3 = dif(d, c);
  const float3 n2 = crossp(b2, b3);
  return atan2f(sqrtf(dotp(b2, b2)) * dotp(b1, n2), dotp(crossp(b1, b2), n2));
}

__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
  return v;
}

// Set the rotors' dihedrals of the molecule held in sx (positions [3n],
// shared memory of this warp) to theta[0..] in build order: rotor k turns
// its moving side about the line through b along b -> c by theta_k minus
// the current dihedral (Rodrigues' formula).
__device__ void set_torsions(const TemplateView& tv, int t, int n, float* sx, const float* theta, int lane) {
  const int r0 = tv.rot_off[t], r1 = tv.rot_off[t + 1];
  for (int k = r0; k < r1; ++k) {
    const Rotor R = tv.rot[k];
    __syncwarp();
    const float3 xa = ldp(sx, R.a), xb = ldp(sx, R.b), xc = ldp(sx, R.c), xd = ldp(sx, R.d);
    const float delta = theta[k - r0] - dihedral_of(xa, xb, xc, xd);
    float3 u = dif(xc, xb);
    const float iu = rsqrtf(dotp(u, u));
    u = make_float3(u.x * iu, u.y * iu, u.z * iu);
    float s, c;
    sincosf(delta, &s, &c);
    const float oc = 1.f - c;
    // R = c I + s [u]_x + (1 - c) u u^T
    const float M[9] = {c + oc * u.x * u.x, oc * u.x * u.y - s * u.z, oc * u.x * u.z + s * u.y,
                        oc * u.y * u.x + s * u.z, c + oc * u.y * u.y, oc * u.y * u.z - s * u.x,
                        oc * u.z * u.x - s * u.y, oc * u.z * u.y + s * u.x, c + oc * u.z * u.z};
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      if (!((R.move[i >> 5] >> (i & 31)) & 1u)) continue;
      const float3 p = dif(ldp(sx, i), xb);
      sx[3 * i] = xb.x + M[0] * p.x + M[1] * p.y + M[2] * p.z;
      sx[3 * i + 1] = xb.y + M[3] * p.x + M[4] * p.y + M[5] * p.z;
      sx[3 * i + 2] = xb.z + M[6] * p.x + M[7] * p.y + M[8] * p.z;
    }
  }
  __syncwarp();
}

// Mass-weighted centre of the positions in sx (every lane gets it).
__device__ double3 centre(const TemplateView& tv, int ab, int n, const float* sx, int lane) {
  double m = 0, cx = 0, cy = 0, cz = 0;
  for (int i = lane; i < n; i += 32) {
    const double w = tv.body[ab + i].w;
    m += w;
    cx += w * sx[3 * i];
    cy += w * sx[3 * i + 1];
    cz += w * sx[3 * i + 2];
  }
  m = wsum_d(m);
  return make_double3(wsum_d(cx) / m, wsum_d(cy) / m, wsum_d(cz) / m);
}

__device__ __forceinline__ float fold(float v, float o, float L) { return o + (v - o - L * floorf((v - o) / L)); }

__global__ void __launch_bounds__(32 * kPoseWarps)
build_flex_kernel(TemplateView tv, const int* __restrict__ rep_tmpl, const int* __restrict__ rep_off, int n_rep,
                  const float* __restrict__ poses, int stride, int do_fold, float ox, float oy, float lx, float ly,
                  float* __restrict__ x, float* __restrict__ v) {
  __shared__ float s_x[kPoseWarps][3 * GRIDFF_MAX_ATOMS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sx = s_x[wib];
  for (int r = blockIdx.x * kPoseWarps + wib; r < n_rep; r += gridDim.x * kPoseWarps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    const float* P = poses + (size_t)r * stride;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const float4 b = tv.body[ab + i];
      sx[3 * i] = b.x;
      sx[3 * i + 1] = b.y;
      sx[3 * i + 2] = b.z;
    }
    set_torsions(tv, t, n, sx, P + 7, lane);
    const double3 cm = centre(tv, ab, n, sx, lane);
    float q0 = P[3], q1 = P[4], q2 = P[5], q3 = P[6];
    const float nq = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    if (nq > 1e-12f) {
      q0 /= nq; q1 /= nq; q2 /= nq; q3 /= nq;
    } else {
      q0 = 1.f; q1 = q2 = q3 = 0.f;
    }
    float Rm[9];
    quat_rot(q0, q1, q2, q3, Rm);
    float cx = P[0], cy = P[1];
    if (do_fold) {
      cx = fold(cx, ox, lx);
      cy = fold(cy, oy, ly);
    }
    const float cz = P[2];
    for (int i = lane; i < n; i += 32) {
      const float px = (float)(sx[3 * i] - cm.x), py = (float)(sx[3 * i + 1] - cm.y),
                  pz = (float)(sx[3 * i + 2] - cm.z);
      float* o = x + 3 * ((size_t)off + i);
      o[0] = Rm[0] * px + Rm[1] * py + Rm[2] * pz + cx;
      o[1] = Rm[3] * px + Rm[4] * py + Rm[5] * pz + cy;
      o[2] = Rm[6] * px + Rm[7] * py + Rm[8] * pz + cz;
      float* w = v + 3 * ((size_t)off + i);
      w[0] = w[1] = w[2] = 0.f;
    }
  }
}

__global__ void build_rigid_kernel(int n_rep, const float* __restrict__ poses, int stride, int do_fold, float ox,
                                   float oy, float lx, float ly, float* __restrict__ x, float* __restrict__ v) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rep) return;
  const float* P = poses + (size_t)r * stride;
  float* p = x + 7 * (size_t)r;
  p[0] = do_fold ? fold(P[0], ox, lx) : P[0];
  p[1] = do_fold ? fold(P[1], oy, ly) : P[1];
  p[2] = P[2];
  const float nq = sqrtf(P[3] * P[3] + P[4] * P[4] + P[5] * P[5] + P[6] * P[6]);
  if (nq > 1e-12f) {
    for (int a = 0; a < 4; ++a) p[3 + a] = P[3 + a] / nq;
  } else {
    p[3] = 1.f;
    p[4] = p[5] = p[6] = 0.f;
  }
  for (int a = 0; a < 6; ++a) v[6 * (size_t)r + a] = 0.f;
}

// Eigenvector of the largest eigenvalue of a symmetric 4x4 matrix A (FP64)
// by cyclic Jacobi rotations: each rotation in the plane (p, q) zeroes
// A[p][q] with t = tan(phi) the smaller root of t^2 + 2 theta t - 1 = 0,
// theta = (A[q][q] - A[p][p]) / (2 A[p][q]); V accumulates the rotations.
__device__ void largest_eigvec4(double A[4][4], double out[4]) {
  double V[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  for (int sweep = 0; sweep < 32; ++sweep) {
    double off = 0, diag = 0;
    for (int p = 0; p < 4; ++p) {
      diag += A[p][p] * A[p][p];
      for (int q = p + 1; q < 4; ++q) off += A[p][q] * A[p][q];
    }
    if (off <= 1e-30 * diag || off == 0) break;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 4; ++q) {
        if (A[p][q] == 0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
        const double c = 1 / sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < 4; ++k) {       // columns p, q of A
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 4; ++k) {       // rows p, q of A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 4; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int best = 0;
  for (int p = 1; p < 4; ++p)
    if (A[p][p] > A[best][best]) best = p;
  for (int k = 0; k < 4; ++k) out[k] = V[k][best];
}

__global__ void __launch_bounds__(32 * kPoseWarps)
targets_flex_kernel(TemplateView tv, const int* __restrict__ rep_tmpl, const int* __restrict__ rep_off, int n_rep,
                    const float* __restrict__ x, int do_fold, float ox, float oy, float lx, float ly,
                    float* __restrict__ targets, float* __restrict__ mask) {
  __shared__ float s_y[kPoseWarps][3 * GRIDFF_MAX_ATOMS];
  __shared__ float s_z[kPoseWarps][3 * GRIDFF_MAX_ATOMS];
  __shared__ float s_th[kPoseWarps][GRIDFF_MAX_ROTORS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float *sy = s_y[wib], *sz = s_z[wib], *th = s_th[wib];
  for (int r = blockIdx.x * kPoseWarps + wib; r < n_rep; r += gridDim.x * kPoseWarps) {
    const int t = rep_tmpl[r], n = tv.natoms[t], ab = tv.atom_off[t], off = rep_off[r];
    const int r0 = tv.rot_off[t], nr = tv.rot_off[t + 1] - r0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      for (int a = 0; a < 3; ++a) sy[3 * i + a] = x[3 * ((size_t)off + i) + a];
      const float4 b = tv.body[ab + i];
      sz[3 * i] = b.x;
      sz[3 * i + 1] = b.y;
      sz[3 * i + 2] = b.z;
    }
    __syncwarp();
    if (lane < nr) {
      const Rotor R = tv.rot[r0 + lane];
      th[lane] = dihedral_of(ldp(sy, R.a), ldp(sy, R.b), ldp(sy, R.c), ldp(sy, R.d));
    }
    __syncwarp();
    set_torsions(tv, t, n, sz, th, lane);
    const double3 cy = centre(tv, ab, n, sy, lane), cz = centre(tv, ab, n, sz, lane);
    // mass-weighted cross-covariance S_ab = sum m z_a y_b of the centred sets
    double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = lane; i < n; i += 32) {
      const double w = tv.body[ab + i].w;
      const double z[3] = {sz[3 * i] - cz.x, sz[3 * i + 1] - cz.y, sz[3 * i + 2] - cz.z};
      const double y[3] = {sy[3 * i] - cy.x, sy[3 * i + 1] - cy.y, sy[3 * i + 2] - cy.z};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] += w * z[a] * y[b];
    }
    for (int k = 0; k < 9; ++k) S[k] = wsum_d(S[k]);
    if (lane == 0) {
      const double sxx = S[0], sxy = S[1], sxz = S[2], syx = S[3], syy = S[4], syz = S[5], szx = S[6], szy = S[7],
                   szz = S[8];
      // Horn's matrix: its top eigenvector is the quaternion of the
      // rotation maximising sum m (R z).y
      double N[4][4] = {{sxx + syy + szz, syz - szy, szx - sxz, sxy - syx},
                        {syz - szy, sxx - syy - szz, sxy + syx, szx + sxz},
                        {szx - sxz, sxy + syx, -sxx + syy - szz, syz + szy},
                        {sxy - syx, szx + sxz, syz + szy, -sxx - syy + szz}};
      double q[4];
      largest_eigvec4(N, q);
      const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      const double sg = q[0] < 0 ? -1.0 : 1.0;
      float* T = targets + (size_t)r * kPoseLen;
      T[0] = do_fold ? fold((float)cy.x, ox, lx) : (float)cy.x;
      T[1] = do_fold ? fold((float)cy.y, oy, ly) : (float)cy.y;
      T[2] = (float)cy.z;
      for (int a = 0; a < 4; ++a) T[3 + a] = (float)(sg * q[a] / nq);
      for (int k = 0; k < GRIDFF_MAX_ROTORS; ++k) T[7 + k] = k < nr ? th[k] : 0.f;
      if (mask)
        for (int k = 0; k < GRIDFF_MAX_ROTORS; ++k) mask[(size_t)r * GRIDFF_MAX_ROTORS + k] = k < nr ? 1.f : 0.f;
    }
  }
}

__global__ void targets_rigid_kernel(int n_rep, const float* __restrict__ x, int do_fold, float ox, float oy,
                                     float lx, float ly, float* __restrict__ targets, float* __restrict__ mask) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rep) return;
  const float* p = x + 7 * (size_t)r;
  float* T = targets + (size_t)r * kPoseLen;
  T[0] = do_fold ? fold(p[0], ox, lx) : p[0];
  T[1] = do_fold ? fold(p[1], oy, ly) : p[1];
  T[2] = p[2];
  const float nq = sqrtf(p[3] * p[3] + p[4] * p[4] + p[5] * p[5] + p[6] * p[6]);
  const float sg = p[3] < 0.f ? -1.f : 1.f;
  for (int a = 0; a < 4; ++a) T[3 + a] = nq > 0.f ? sg * p[3 + a] / nq : (a == 0 ? 1.f : 0.f);
  for (int k = 0; k < GRIDFF_MAX_ROTORS; ++k) {
    T[7 + k] = 0.f;
    if (mask) mask[(size_t)r * GRIDFF_MAX_ROTORS + k] = 0.f;
  }
}

bool fold_args(const double* o, const double* L, float f[4]) {
  if (!o || !L) return false;
  f[0] = (float)o[0];
  f[1] = (float)o[1];
  f[2] = (float)L[0];
  f[3] = (float)L[1];
  return true;
}

int pose_blocks(gridff_ctx* ctx, int n_rep) {
  const int need = (n_rep + kPoseWarps - 1) / kPoseWarps;
  const int cap = ctx->n_sm * 8;
  return need < cap ? need : cap;
}

// Lift of a replica set: one warp per replica finds the lowest atom (rigid:
// of R(q) b + c) and, when it lies below z_floor, moves the replica up by
// the difference (rigid: the centre of mass; flexible: every atom).
__global__ void lift_kernel(TemplateView tv, const int* __restrict__ rep_tmpl, const int* __restrict__ rep_off,
                            int n_rep, int rigid, float z_floor, float* __restrict__ x) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_rep) return;
  const int t = rep_tmpl[r];
  const int n = tv.natoms[t], ab = tv.atom_off[t];
  float lowest = INFINITY;
  float* p = rigid ? x + 7 * (size_t)r : x + 3 * (size_t)rep_off[r];
  float Rm[9];
  if (rigid) {
    const float qn = rsqrtf(p[3] * p[3] + p[4] * p[4] + p[5] * p[5] + p[6] * p[6]);
    quat_rot(p[3] * qn, p[4] * qn, p[5] * qn, p[6] * qn, Rm);
  }
  for (int i = lane; i < n; i += 32) {
    if (rigid) {
      const float4 b = tv.body[ab + i];
      lowest = fminf(lowest, p[2] + Rm[6] * b.x + Rm[7] * b.y + Rm[8] * b.z);
    } else {
      lowest = fminf(lowest, p[3 * i + 2]);
    }
  }
  for (int o = 16; o; o >>= 1) lowest = fminf(lowest, __shfl_xor_sync(kAll, lowest, o));
  if (!(lowest < z_floor)) return;   // also leaves replicas with non-finite positions alone
  const float dz = z_floor - lowest;
  if (rigid) {
    if (lane == 0) p[2] += dz;
  } else {
    for (int i = lane; i < n; i += 32) p[3 * i + 2] += dz;
  }
}

}  // namespace

gridff_status enqueue_build_poses(gridff_replicas* R, const float* d_poses, int stride, const double origin_xy[2],
                                  const double tile_xy[2]) {
  gridff_ctx* ctx = R->ctx;
  cudaStream_t s = ctx->stream;
  float f[4] = {0.f, 0.f, 1.f, 1.f};
  const int do_fold = fold_args(origin_xy, tile_xy, f) ? 1 : 0;
  if (do_fold && !(f[2] > 0 && f[3] > 0)) return set_err(ctx, GRIDFF_EINVAL, "tile lengths must be positive");
  if (R->rigid)
    build_rigid_kernel<<<(R->n_rep + 127) / 128, 128, 0, s>>>(R->n_rep, d_poses, stride, do_fold, f[0], f[1], f[2],
                                                              f[3], R->x, R->v);
  else
    build_flex_kernel<<<pose_blocks(ctx, R->n_rep), 32 * kPoseWarps, 0, s>>>(
        R->tv, R->rep_tmpl, R->rep_off, R->n_rep, d_poses, stride, do_fold, f[0], f[1], f[2], f[3], R->x, R->v);
  GRIDFF_CUDA(ctx, cudaGetLastError());
  return GRIDFF_OK;
}

extern "C" {

gridff_status gridff_template_rotors(const gridff_replicas* R, int32_t t, int32_t* n_rot, int32_t* quads) {
  if (!R || !n_rot || t < 0 || t >= R->n_tmpl) return GRIDFF_EINVAL;
  const int r0 = R->h_rot_off[t], r1 = R->h_rot_off[t + 1];
  *n_rot = r1 - r0;
  if (quads)
    for (int k = r0; k < r1; ++k) {
      const Rotor& q = R->h_rot[k];
      quads[4 * (k - r0)] = q.a;
      quads[4 * (k - r0) + 1] = q.b;
      quads[4 * (k - r0) + 2] = q.c;
      quads[4 * (k - r0) + 3] = q.d;
    }
  return GRIDFF_OK;
}

gridff_status gridff_build_poses(gridff_replicas* R, const float* poses, const double origin_xy[2],
                                 const double tile_xy[2], int flags) {
  NvtxRange nvtx_range("gridff_build_poses");
  if (!R || !poses) return set_err(R ? R->ctx : nullptr, GRIDFF_EINVAL, "null argument");
  if ((origin_xy == nullptr) != (tile_xy == nullptr))
    return set_err(R->ctx, GRIDFF_EINVAL, "origin_xy and tile_xy go together");
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const size_t bytes = (size_t)R->n_rep * kPoseLen * sizeof(float);
  const float* d = poses;
  void* tmp = nullptr;
  if (!(flags & GRIDFF_DEVICE_PTRS)) {
    GRIDFF_CUDA(ctx, cudaMallocAsync(&tmp, bytes, s));
    const cudaError_t e = cudaMemcpyAsync(tmp, poses, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaFreeAsync(tmp, s);
      return set_err(ctx, GRIDFF_ECUDA, "pose upload: %s", cudaGetErrorString(e));
    }
    d = (const float*)tmp;
  }
  gridff_status st = enqueue_build_poses(R, d, kPoseLen, origin_xy, tile_xy);
  if (tmp) cudaFreeAsync(tmp, s);
  if (st != GRIDFF_OK) return st;
  if ((flags & GRIDFF_ASYNC) && (flags & GRIDFF_DEVICE_PTRS)) return GRIDFF_OK;
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

gridff_status gridff_lift(gridff_replicas* R, double z_floor, int flags) {
  NvtxRange nvtx_range("gridff_lift");
  if (!R) return GRIDFF_EINVAL;
  gridff_ctx* ctx = R->ctx;
  if (!isfinite(z_floor)) return set_err(ctx, GRIDFF_EINVAL, "z_floor must be finite");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int threads = 128;
  const long long blocks = ((long long)R->n_rep * 32 + threads - 1) / threads;
  lift_kernel<<<(unsigned)blocks, threads, 0, s>>>(R->tv, R->rep_tmpl, R->rep_off, R->n_rep, R->rigid,
                                                   (float)z_floor, R->x);
  GRIDFF_CUDA(ctx, cudaGetLastError());
  if (!(flags & GRIDFF_ASYNC)) GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

gridff_status gridff_pose_targets(const gridff_replicas* R, const double origin_xy[2], const double tile_xy[2],
                                  float* targets, float* tors_mask, int flags) {
  NvtxRange nvtx_range("gridff_pose_targets");
  if (!R || !targets) return set_err(R ? R->ctx : nullptr, GRIDFF_EINVAL, "null argument");
  if ((origin_xy == nullptr) != (tile_xy == nullptr))
    return set_err(R->ctx, GRIDFF_EINVAL, "origin_xy and tile_xy go together");
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  float f[4] = {0.f, 0.f, 1.f, 1.f};
  const int do_fold = fold_args(origin_xy, tile_xy, f) ? 1 : 0;
  if (do_fold && !(f[2] > 0 && f[3] > 0)) return set_err(ctx, GRIDFF_EINVAL, "tile lengths must be positive");
  const bool dev = flags & GRIDFF_DEVICE_PTRS;
  const size_t tb = (size_t)R->n_rep * kPoseLen * sizeof(float), mb = (size_t)R->n_rep * GRIDFF_MAX_ROTORS * 4;
  float *dt = targets, *dm = tors_mask;
  void* tmp = nullptr;
  if (!dev) {
    GRIDFF_CUDA(ctx, cudaMallocAsync(&tmp, tb + mb, s));
    dt = (float*)tmp;
    dm = tors_mask ? (float*)((char*)tmp + tb) : nullptr;
  }
  if (R->rigid)
    targets_rigid_kernel<<<(R->n_rep + 127) / 128, 128, 0, s>>>(R->n_rep, R->x, do_fold, f[0], f[1], f[2], f[3], dt,
                                                                dm);
  else
    targets_flex_kernel<<<pose_blocks(ctx, R->n_rep), 32 * kPoseWarps, 0, s>>>(
        R->tv, R->rep_tmpl, R->rep_off, R->n_rep, R->x, do_fold, f[0], f[1], f[2], f[3], dt, dm);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !dev) {
    e = cudaMemcpyAsync(targets, dt, tb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && tors_mask) e = cudaMemcpyAsync(tors_mask, dm, mb, cudaMemcpyDeviceToHost, s);
  }
  if (tmp) cudaFreeAsync(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "pose targets: %s", cudaGetErrorString(e));
  return GRIDFF_OK;
}

}  // extern "C"
