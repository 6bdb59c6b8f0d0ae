// Learned pose proposal: a small MLP (molecule descriptor + noise in,
// centre of mass + orientation quaternion + torsions out) with bfloat16
// weights and FP32 accumulation on the tensor cores (mma.sync m16n8k16),
// trained on the device with a winner-takes-all pose loss and Adam, and a
// proposal kernel that writes replica poses for gridff_relax.
// Not from the paper: it chooses where GridFF relaxations start.
#include <cuda_bf16.h>
#include <stddef.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace {

constexpr int kOut = 19;      // 3 position + 4 quaternion + 12 torsions
constexpr int kTors = 12;
constexpr int kMaxSplit = 8;  // split-K parts of the weight-gradient GEMM

inline int pad16(int n) { return (n + 15) & ~15; }

// ---------------------------------------------------------------------------
// C[M][N] (FP32) = A[M][K] * B, A row-major bf16 (lda), B given as Bt[N][K]
// row-major bf16 (ldb), i.e. B is K x N column-major.  M % 16 == 0,
// N % 8 == 0, K % 16 == 0, lda and ldb multiples of 8.  Block tile
// 64 x 64, K in slices of 32 staged in shared memory by 16-byte cp.async
// copies (two stages: the next slice loads while the tensor cores work on
// this one; rows and K beyond the matrix are zero-filled); four warps, each
// a 32 x 32 tile of 2 x 4 mma.sync m16n8k16 products per 16 of K, fragments
// read with ldmatrix (rows padded to 40 elements: conflict-free).  Split K:
// block z handles K range [z K, (z + 1) K) and writes its partial product
// to C + z * cstride.
constexpr int kBM = 64, kBN = 64, kBK = 32, kPad = 8, kLds = kBK + kPad;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void ldmatrix_x4(const void* smem, unsigned& r0, unsigned& r1, unsigned& r2,
                                            unsigned& r3) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                        const __nv_bfloat16* __restrict__ Bt, int ldb,
                                                        float* __restrict__ C, int ldc, int M, int N, int K,
                                                        long long cstride) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][kBM][kLds];
  __shared__ __align__(16) __nv_bfloat16 sB[2][kBN][kLds];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;            // warp tile (32 x 32) in the block tile
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  A += (size_t)blockIdx.z * K;
  Bt += (size_t)blockIdx.z * K;
  C += (size_t)blockIdx.z * cstride;
  // a slice is 64 rows x 32 K of A and of Bt: 256 chunks of 8 elements each
  auto load = [&](int stage, int k0) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int chunk = tid + 128 * c, r = chunk >> 2, kc = (chunk & 3) * 8;
      const bool ka = k0 + kc < K;
      const bool va = ka && m0 + r < M, vb = ka && n0 + r < N;
      cp_async16(&sA[stage][r][kc], va ? (const void*)(A + (size_t)(m0 + r) * lda + k0 + kc) : (const void*)A, va);
      cp_async16(&sB[stage][r][kc], vb ? (const void*)(Bt + (size_t)(n0 + r) * ldb + k0 + kc) : (const void*)Bt,
                 vb);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.f;
  const int n_slices = (K + kBK - 1) / kBK;
  load(0, 0);
  for (int sl = 0; sl < n_slices; ++sl) {
    const int stage = sl & 1;
    if (sl + 1 < n_slices) {
      load(stage ^ 1, (sl + 1) * kBK);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    // ldmatrix addresses: lane i serves row (i & 7) of 8 x 8 matrix i >> 3
    const int q = lane >> 3, r8 = lane & 7;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      unsigned a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i)   // A 16 x 16: matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15)
        ldmatrix_x4(&sA[stage][wm * 32 + i * 16 + r8 + (q & 1) * 8][kk + (q >> 1) * 8], a[i][0], a[i][1], a[i][2],
                    a[i][3]);
#pragma unroll
      for (int jp = 0; jp < 2; ++jp)   // two n8 blocks: matrices (n 0-7 | 8-15) x (k 0-7 | 8-15)
        ldmatrix_x4(&sB[stage][wn * 32 + jp * 16 + r8 + (q >> 1) * 8][kk + (q & 1) * 8], b[2 * jp][0],
                    b[2 * jp][1], b[2 * jp + 1][0], b[2 * jp + 1][1]);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    __syncthreads();   // this stage is reloaded two slices later
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = m0 + wm * 32 + i * 16 + g, col = n0 + wn * 32 + j * 8 + 2 * t;
      if (row < M && col < N) {   // M % 16 == 0, N % 8 == 0: a fragment is all in or all out
        float* r0 = C + (size_t)row * ldc + col;
        float* r1 = r0 + (size_t)8 * ldc;
        r0[0] = acc[i][j][0];
        r0[1] = acc[i][j][1];
        r1[0] = acc[i][j][2];
        r1[1] = acc[i][j][3];
      }
    }
}

// C = sum over the S partial products (fixed order: deterministic).
__global__ void splitk_sum_kernel(const float* __restrict__ part, long long cstride, int S, int M, int N, int ldc,
                                  float* __restrict__ C) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const long long off = (idx / N) * ldc + idx % N;
  float v = 0.f;
  for (int k = 0; k < S; ++k) v += part[k * cstride + off];
  C[off] = v;
}

// Input rows (FP32 [rows][n_in]) -> bf16 layer input, row-major [Mp][in_p]
// and transposed [in_p][Mp]; padding zero.
__global__ void input_kernel(const float* __restrict__ X, int rows, int n_in, int Mp, int in_p,
                             __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ HT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Mp * in_p) return;
  const int m = idx / in_p, k = idx % in_p;
  const float v = (m < rows && k < n_in) ? X[(size_t)m * n_in + k] : 0.f;
  const __nv_bfloat16 b = __float2bfloat16(v);
  H[idx] = b;
  HT[(size_t)k * Mp + m] = b;
}

// a = C + bias (pre-activation kept for the ReLU mask); hidden layers emit
// bf16 h = max(a, 0) (row-major and transposed) for the next layer; the last
// layer emits FP32 outputs [rows][n_out].  Padded rows/columns are zero.
__global__ void bias_act_kernel(const float* __restrict__ C, const float* __restrict__ b, int rows, int n_out,
                                int Mp, int out_p, float* __restrict__ Apre, __nv_bfloat16* __restrict__ Hn,
                                __nv_bfloat16* __restrict__ HnT, float* __restrict__ Y) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Mp * out_p) return;
  const int m = idx / out_p, j = idx % out_p;
  const bool live = m < rows && j < n_out;
  const float a = live ? C[idx] + b[j] : 0.f;
  Apre[idx] = a;
  if (Hn) {
    const __nv_bfloat16 h = __float2bfloat16(fmaxf(a, 0.f));
    Hn[idx] = h;
    HnT[(size_t)j * Mp + m] = h;
  } else if (live) {
    Y[(size_t)m * n_out + j] = a;
  }
}

// Winner-takes-all pose loss (see gridff.h): one thread per target; writes
// dL/dY for the winning proposal rows (dY zeroed before) and the target's
// loss share.
__global__ void wta_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                           const float* __restrict__ mask, int n_targets, int K, int out_p, float w_q,
                           float w_t, float tile_x, float tile_y, float* __restrict__ dY,
                           float* __restrict__ loss, int* __restrict__ winner) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_targets) return;
  const float* t = T + (size_t)b * kOut;
  const float* mk = mask ? mask + (size_t)b * kTors : nullptr;
  float best = INFINITY;
  int kb = 0;
  for (int k = 0; k < K; ++k) {
    const float* o = Y + ((size_t)b * K + k) * kOut;
    float dx = o[0] - t[0], dy = o[1] - t[1], dz = o[2] - t[2];
    dx -= tile_x * rintf(dx / tile_x);
    dy -= tile_y * rintf(dy / tile_y);
    float nu = sqrtf(o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6]);
    nu = fmaxf(nu, 1e-12f);
    const float s = (o[3] * t[3] + o[4] * t[4] + o[5] * t[5] + o[6] * t[6]) / nu;
    float d = dx * dx + dy * dy + dz * dz + w_q * (1.f - s * s);
    if (mk)
      for (int j = 0; j < kTors; ++j) d += w_t * mk[j] * (1.f - cosf(o[7 + j] - t[7 + j]));
    if (d < best) {
      best = d;
      kb = k;
    }
  }
  winner[b] = kb;
  loss[b] = best;
  const float* o = Y + ((size_t)b * K + kb) * kOut;
  float* g = dY + ((size_t)b * K + kb) * out_p;
  const float inv_b = 1.f / n_targets;
  float dx = o[0] - t[0], dy = o[1] - t[1], dz = o[2] - t[2];
  dx -= tile_x * rintf(dx / tile_x);
  dy -= tile_y * rintf(dy / tile_y);
  g[0] = 2.f * dx * inv_b;
  g[1] = 2.f * dy * inv_b;
  g[2] = 2.f * dz * inv_b;
  float nu = sqrtf(o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6]);
  nu = fmaxf(nu, 1e-12f);
  float q[4] = {o[3] / nu, o[4] / nu, o[5] / nu, o[6] / nu};
  const float s = q[0] * t[3] + q[1] * t[4] + q[2] * t[5] + q[3] * t[6];
  for (int a = 0; a < 4; ++a) g[3 + a] = -2.f * w_q * s * (t[3 + a] - s * q[a]) / nu * inv_b;
  for (int j = 0; j < kTors; ++j) g[7 + j] = mk ? w_t * mk[j] * sinf(o[7 + j] - t[7 + j]) * inv_b : 0.f;
}

// G (FP32 [Mp][out_p], dL/da of this layer) -> bf16 row-major and transposed.
// If `mask_pre` is given, G is first multiplied by (pre-activation > 0).
__global__ void grad_prep_kernel(float* __restrict__ G, const float* __restrict__ mask_pre, int rows, int n_out,
                                 int Mp, int out_p, __nv_bfloat16* __restrict__ Gb, __nv_bfloat16* __restrict__ GbT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Mp * out_p) return;
  const int m = idx / out_p, j = idx % out_p;
  float v = (m < rows && j < n_out) ? G[idx] : 0.f;
  if (mask_pre && !(mask_pre[idx] > 0.f)) v = 0.f;
  G[idx] = v;
  const __nv_bfloat16 b = __float2bfloat16(v);
  Gb[idx] = b;
  GbT[(size_t)j * Mp + m] = b;
}

// db[j] = sum_m G[m][j] in two passes (deterministic): block (x, y) sums
// rows [y R, (y + 1) R) of 32 columns (8 row groups, coalesced across the
// columns) into part[y][j]; then colsum_final adds the chunks in order.
__global__ void colsum_kernel(const float* __restrict__ G, int Mp, int out_p, int n_out, int rows_per_chunk,
                              float* __restrict__ part) {
  __shared__ float sh[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int m0 = blockIdx.y * rows_per_chunk, m1 = min(Mp, m0 + rows_per_chunk);
  float s = 0.f;
  if (j < n_out)
    for (int m = m0 + threadIdx.y; m < m1; m += 8) s += G[(size_t)m * out_p + j];
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < n_out) {
    float t = 0.f;
    for (int y = 0; y < 8; ++y) t += sh[y][threadIdx.x];
    part[(size_t)blockIdx.y * n_out + j] = t;
  }
}

__global__ void colsum_final_kernel(const float* __restrict__ part, int chunks, int n_out, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_out) return;
  float t = 0.f;
  for (int c = 0; c < chunks; ++c) t += part[(size_t)c * n_out + j];
  db[j] = t;
}

// Adam on FP32 master parameters; c1 = lr / (1 - b1^t), c2 = 1 / (1 - b2^t),
// from the arguments or, when c12 is set, from device memory (the training
// loop's step counters, which a CUDA graph replay advances on the device).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float b1, float b2, float eps, float c1, float c2,
                            const float* __restrict__ c12) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (c12) {
    c1 = c12[0];
    c2 = c12[1];
  }
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= c1 * mi / (sqrtf(vi * c2) + eps);
}

// FP32 master W [out][in] -> bf16 padded copies Wb [out_p][in_p] and
// WbT [in_p][out_p].
__global__ void weights_bf16_kernel(const float* __restrict__ W, int n_out, int n_in, int out_p, int in_p,
                                    __nv_bfloat16* __restrict__ Wb, __nv_bfloat16* __restrict__ WbT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= out_p * in_p) return;
  const int o = idx / in_p, i = idx % in_p;
  const float v = (o < n_out && i < n_in) ? W[(size_t)o * n_in + i] : 0.f;
  const __nv_bfloat16 b = __float2bfloat16(v);
  Wb[idx] = b;
  WbT[(size_t)i * out_p + o] = b;
}

// Counter-based standard normal: splitmix64 of (seed, counter), Box-Muller.
__device__ __forceinline__ float normal01(unsigned long long seed, unsigned long long counter) {
  return normal_of(splitmix64(seed ^ splitmix64(counter)));
}

// Proposal inputs: row r = [descriptor (n_desc), noise (n_noise)].
__global__ void propose_input_kernel(const float* __restrict__ desc, int n_desc, int n_noise, int rows,
                                     unsigned long long seed, int Mp, int in_p, __nv_bfloat16* __restrict__ H,
                                     __nv_bfloat16* __restrict__ HT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Mp * in_p) return;
  const int m = idx / in_p, k = idx % in_p;
  float v = 0.f;
  if (m < rows) {
    if (k < n_desc) v = desc[k];
    else if (k < n_desc + n_noise) v = normal01(seed, (unsigned long long)m * 64 + (k - n_desc));
  }
  const __nv_bfloat16 b = __float2bfloat16(v);
  H[idx] = b;
  HT[(size_t)k * Mp + m] = b;
}

// Network outputs -> rigid poses: centre of mass (x, y folded into the tile
// starting at origin), normalised quaternion (identity if degenerate).
__global__ void pose_kernel(const float* __restrict__ Y, int rows, float ox, float oy, float tile_x, float tile_y,
                            float* __restrict__ pose) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const float* o = Y + (size_t)r * kOut;
  float x = o[0] - ox, y = o[1] - oy;
  x -= tile_x * floorf(x / tile_x);
  y -= tile_y * floorf(y / tile_y);
  float nu = sqrtf(o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6]);
  float* p = pose + 7 * (size_t)r;
  p[0] = x + ox;
  p[1] = y + oy;
  p[2] = o[2];
  if (nu > 1e-12f) {
    p[3] = o[3] / nu; p[4] = o[4] / nu; p[5] = o[5] / nu; p[6] = o[6] / nu;
  } else {
    p[3] = 1.f; p[4] = p[5] = p[6] = 0.f;
  }
}

// Counters of the device-side training loop, advanced once per step on the
// device so that one captured step can be replayed: the random-stream step
// and loss-history index of the current step, the Adam step t and its
// bias-correction factors c12 = {lr / (1 - b1^t), 1 / (1 - b2^t)}.
struct StepCounters {
  long long next_step, step;
  int next_k, k;
  long long t;
  float c12[2];
};

// Start of a step: take the next random-stream step and history slot, and
// (update) advance Adam's t and its bias corrections.
__global__ void step_begin_kernel(StepCounters* c, double lr, double b1, double b2, int update) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->step = c->next_step++;
  c->k = c->next_k++;
  if (update) {
    c->t += 1;
    c->c12[0] = (float)(lr / (1.0 - pow(b1, (double)c->t)));
    c->c12[1] = (float)(1.0 / (1.0 - pow(b2, (double)c->t)));
  }
}

// Training batch drawn on the device: target b of step `step` is row
// splitmix64(seed ^ splitmix64(2^20 step + b)) mod n_all of the training set.
__global__ void sample_targets_kernel(const float* __restrict__ T_all, const float* __restrict__ M_all, int n_all,
                                      int B, unsigned long long seed, const StepCounters* __restrict__ ctr,
                                      float* __restrict__ Ts, float* __restrict__ Ms) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const long long step = ctr->step;
  const unsigned long long h = splitmix64(seed ^ splitmix64(((unsigned long long)step << 20) + b));
  const int row = (int)(h % (unsigned long long)n_all);
  for (int j = 0; j < kOut; ++j) Ts[(size_t)b * kOut + j] = T_all[(size_t)row * kOut + j];
  for (int j = 0; j < kTors; ++j) Ms[(size_t)b * kTors + j] = M_all ? M_all[(size_t)row * kTors + j] : 0.f;
}

// Training inputs: row m = [descriptor, N(0,1) noise], noise j of row m of
// step `step` from the counter 64 (2^20 step + m) + j.
__global__ void train_inputs_kernel(const float* __restrict__ desc, int n_desc, int n_noise, int rows,
                                    unsigned long long seed, const StepCounters* __restrict__ ctr, int Mp, int in_p,
                                    __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ HT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Mp * in_p) return;
  const long long step = ctr->step;
  const int m = idx / in_p, k = idx % in_p;
  float v = 0.f;
  if (m < rows) {
    if (k < n_desc) {
      v = desc[k];
    } else if (k < n_desc + n_noise) {
      const unsigned long long c = ((((unsigned long long)step << 20) + m) << 6) + (k - n_desc);
      v = normal_of(splitmix64(seed ^ splitmix64(c)));
    }
  }
  const __nv_bfloat16 b = __float2bfloat16(v);
  H[idx] = b;
  HT[(size_t)k * Mp + m] = b;
}

// hist[k] = mean of loss[0..n) for the step's history slot k (one block).
__global__ void loss_mean_kernel(const float* __restrict__ loss, int n, float* __restrict__ hist,
                                 const StepCounters* __restrict__ ctr) {
  float* out = hist + ctr->k;
  __shared__ float part[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += loss[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = part[0] / n;
}

inline unsigned grid1(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct gridff_mlp {
  gridff_ctx* ctx = nullptr;
  int device = 0;
  int L = 0;                       // layers
  std::vector<int> sizes, pads;    // widths and padded widths (L + 1)
  std::vector<size_t> woff, boff;  // offsets of W_l, b_l in the flat parameter array
  size_t n_params = 0;
  float* P = nullptr;              // FP32 master parameters [n_params]
  float* Gr = nullptr;             // gradients
  float* Am = nullptr;             // Adam first moments
  float* Av = nullptr;             // Adam second moments
  std::vector<__nv_bfloat16*> Wb, WbT;
  long long t = 0;                 // Adam step counter
  // batch workspace
  int cap = 0;                     // padded rows
  std::vector<__nv_bfloat16*> H, HT;   // layer inputs (L)
  std::vector<float*> Apre;             // pre-activations (L)
  float* C = nullptr;              // GEMM output scratch [cap][max_pad]
  float* Cpart = nullptr;          // split-K partial products [8][max_pad][max_pad]
  float* G = nullptr;              // gradient scratch [cap][max_pad]
  float* G2 = nullptr;
  __nv_bfloat16* Gb = nullptr;
  __nv_bfloat16* GbT = nullptr;
  float* Y = nullptr;              // outputs [cap][kOut]
  float* Xs = nullptr;             // staged host inputs [cap][n_in]
  float* Ts = nullptr;             // staged targets
  float* Ms = nullptr;             // staged torsion masks
  float* loss = nullptr;           // [cap]
  int* winner = nullptr;           // [cap]
  float* desc = nullptr;           // [n_in]
  std::vector<void*> owned;
  // device-resident training set and loss history (gridff_mlp_train)
  float* T_all = nullptr;
  float* M_all = nullptr;
  int n_all = 0;
  float* loss_hist = nullptr;
  int loss_cap = 0;
  long long rng_step = 0;
  StepCounters* ctr = nullptr;     // device step counters of the training loop
};

namespace {

template <class T>
cudaError_t dalloc(gridff_mlp* m, T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e == cudaSuccess) m->owned.push_back(*p);
  return e;
}

gridff_status ensure_batch(gridff_mlp* m, int rows) {
  const int Mp = pad16(rows);
  if (Mp <= m->cap) return GRIDFF_OK;
  gridff_ctx* ctx = m->ctx;
  // release the old workspace (parameters stay)
  std::vector<void*> keep;
  auto is_ws = [&](void* p) {
    for (auto* h : m->H) if (p == h) return true;
    for (auto* h : m->HT) if (p == h) return true;
    for (auto* a : m->Apre) if (p == a) return true;
    return p == m->C || p == m->Cpart || p == m->G || p == m->G2 || p == m->Gb || p == m->GbT || p == m->Y || p == m->Xs ||
           p == m->Ts || p == m->Ms || p == m->loss || p == m->winner;
  };
  cudaStreamSynchronize(ctx->stream);
  for (void* p : m->owned) {
    if (is_ws(p)) cudaFree(p);
    else keep.push_back(p);
  }
  m->owned = keep;
  int maxp = *std::max_element(m->pads.begin(), m->pads.end());
  m->H.assign(m->L, nullptr);
  m->HT.assign(m->L, nullptr);
  m->Apre.assign(m->L, nullptr);
  bool ok = true;
  for (int l = 0; l < m->L; ++l) {
    ok &= dalloc(m, &m->H[l], (size_t)Mp * m->pads[l]) == cudaSuccess;
    ok &= dalloc(m, &m->HT[l], (size_t)Mp * m->pads[l]) == cudaSuccess;
    ok &= dalloc(m, &m->Apre[l], (size_t)Mp * m->pads[l + 1]) == cudaSuccess;
  }
  // C also holds a weight gradient [out_p][in_p], which can exceed Mp rows
  ok &= dalloc(m, &m->C, (size_t)std::max(Mp, maxp) * maxp) == cudaSuccess;
  ok &= dalloc(m, &m->Cpart, (size_t)kMaxSplit * maxp * maxp) == cudaSuccess;
  ok &= dalloc(m, &m->G, (size_t)Mp * maxp) == cudaSuccess;
  ok &= dalloc(m, &m->G2, (size_t)Mp * maxp) == cudaSuccess;
  ok &= dalloc(m, &m->Gb, (size_t)Mp * maxp) == cudaSuccess;
  ok &= dalloc(m, &m->GbT, (size_t)Mp * maxp) == cudaSuccess;
  ok &= dalloc(m, &m->Y, (size_t)Mp * kOut) == cudaSuccess;
  ok &= dalloc(m, &m->Xs, (size_t)Mp * m->sizes[0]) == cudaSuccess;
  ok &= dalloc(m, &m->Ts, (size_t)Mp * kOut) == cudaSuccess;
  ok &= dalloc(m, &m->Ms, (size_t)Mp * kTors) == cudaSuccess;
  ok &= dalloc(m, &m->loss, (size_t)Mp) == cudaSuccess;
  ok &= dalloc(m, &m->winner, (size_t)Mp) == cudaSuccess;
  if (!ok) return set_err(ctx, GRIDFF_ENOMEM, "MLP workspace for %d rows", rows);
  m->cap = Mp;
  return GRIDFF_OK;
}

// C = A B^T-layout product; with `part` (scratch of kMaxSplit * M * ldc
// floats) a long-K product with few output tiles is split over K.
void gemm(cudaStream_t s, const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bt, int ldb, float* C, int ldc,
          int M, int N, int K, float* part = nullptr) {
  const long long warps = (long long)(M / 16) * (N / 8);
  int S = 1;
  if (part && warps < 2048)
    for (int cand = kMaxSplit; cand > 1; cand >>= 1)
      if ((K / 16) % cand == 0 && K / cand >= 128) {
        S = cand;
        break;
      }
  const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, S);
  if (S == 1) {
    gemm_bf16_kernel<<<grid, 128, 0, s>>>(A, lda, Bt, ldb, C, ldc, M, N, K, 0);
    return;
  }
  const long long cstride = (long long)M * ldc;
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(A, lda, Bt, ldb, part, ldc, M, N, K / S, cstride);
  splitk_sum_kernel<<<grid1((long long)M * N), 256, 0, s>>>(part, cstride, S, M, N, ldc, C);
}

void refresh_bf16(gridff_mlp* m) {
  for (int l = 0; l < m->L; ++l) {
    const int in = m->sizes[l], out = m->sizes[l + 1], ip = m->pads[l], op = m->pads[l + 1];
    weights_bf16_kernel<<<grid1((long long)op * ip), 256, 0, m->ctx->stream>>>(m->P + m->woff[l], out, in, op,
                                                                                ip, m->Wb[l], m->WbT[l]);
  }
}

// Forward of `rows` rows whose layer-0 input is already in H[0]/HT[0].
void forward_rows(gridff_mlp* m, int rows) {
  cudaStream_t s = m->ctx->stream;
  const int Mp = pad16(rows);
  for (int l = 0; l < m->L; ++l) {
    const int ip = m->pads[l], op = m->pads[l + 1];
    gemm(s, m->H[l], ip, m->Wb[l], ip, m->C, op, Mp, op, ip);
    const bool last = l == m->L - 1;
    bias_act_kernel<<<grid1((long long)Mp * op), 256, 0, s>>>(
        m->C, m->P + m->boff[l], rows, m->sizes[l + 1], Mp, op, m->Apre[l], last ? nullptr : m->H[l + 1],
        last ? nullptr : m->HT[l + 1], m->Y);
  }
}

// One training step on inputs already in H[0]/HT[0] and targets in Ts/Ms:
// forward, winner-takes-all loss, backward, Adam (unless NO_UPDATE).
// Enqueued on the context stream, no synchronisation.
gridff_status enqueue_train(gridff_mlp* m, int n_targets, int K, bool mask_on, const gridff_train_params* tp,
                            int flags, const StepCounters* ctr = nullptr) {
  gridff_ctx* ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int rows = n_targets * K;
  const int Mp = pad16(rows), L = m->L;
  forward_rows(m, rows);
  // loss and dL/dY (written into G with the last layer's padded stride)
  const int op_last = m->pads[L];
  GRIDFF_CUDA(ctx, cudaMemsetAsync(m->G, 0, (size_t)Mp * op_last * sizeof(float), s));
  wta_kernel<<<grid1(n_targets, 128), 128, 0, s>>>(m->Y, m->Ts, mask_on ? m->Ms : nullptr, n_targets, K, op_last,
                                                  tp->w_q, tp->w_t, (float)tp->tile[0], (float)tp->tile[1], m->G,
                                                  m->loss, m->winner);
  // backward
  float* Gcur = m->G;
  float* Gnext = m->G2;
  for (int l = L - 1; l >= 0; --l) {
    const int ip = m->pads[l], op = m->pads[l + 1];
    grad_prep_kernel<<<grid1((long long)Mp * op), 256, 0, s>>>(Gcur, l == L - 1 ? nullptr : m->Apre[l], rows,
                                                               m->sizes[l + 1], Mp, op, m->Gb, m->GbT);
    {
      const int n_out = m->sizes[l + 1];
      const int rpc = std::max(256, (Mp + 63) / 64);
      const int chunks = (Mp + rpc - 1) / rpc;
      colsum_kernel<<<dim3((n_out + 31) / 32, chunks), dim3(32, 8), 0, s>>>(Gcur, Mp, op, n_out, rpc, m->Cpart);
      colsum_final_kernel<<<grid1(n_out, 128), 128, 0, s>>>(m->Cpart, chunks, n_out, m->Gr + m->boff[l]);
    }
    // dW [out][in] = G^T X: A = GbT [op][Mp], Bt = HT [ip][Mp]
    gemm(s, m->GbT, Mp, m->HT[l], Mp, m->C, ip, op, ip, Mp, m->Cpart);
    // copy the live block of C into the flat gradient array
    GRIDFF_CUDA(ctx, cudaMemcpy2DAsync(m->Gr + m->woff[l], m->sizes[l] * sizeof(float), m->C, ip * sizeof(float),
                                       m->sizes[l] * sizeof(float), m->sizes[l + 1], cudaMemcpyDeviceToDevice, s));
    if (l > 0) {
      // dL/d(input) = G W: A = Gb [Mp][op], Bt = WbT [ip][op]
      gemm(s, m->Gb, op, m->WbT[l], op, Gnext, ip, Mp, ip, op);
      std::swap(Gcur, Gnext);
    }
  }
  GRIDFF_CUDA(ctx, cudaGetLastError());
  if (!(flags & GRIDFF_MLP_NO_UPDATE)) {
    float c1 = 0.f, c2 = 0.f;
    if (!ctr) {   // else the step's counters on the device hold t and the factors
      m->t += 1;
      const double b1 = tp->beta1, b2 = tp->beta2;
      c1 = (float)(tp->lr / (1.0 - pow(b1, (double)m->t)));
      c2 = (float)(1.0 / (1.0 - pow(b2, (double)m->t)));
    }
    adam_kernel<<<grid1((long long)m->n_params), 256, 0, s>>>(m->P, m->Gr, m->Am, m->Av, (int)m->n_params,
                                                              tp->beta1, tp->beta2, tp->eps, c1, c2,
                                                              ctr ? reinterpret_cast<const float*>(
                                                                        reinterpret_cast<const char*>(ctr) +
                                                                        offsetof(StepCounters, c12))
                                                                  : nullptr);
    refresh_bf16(m);
  }
  return GRIDFF_OK;
}

}  // namespace

extern "C" {

gridff_status gridff_mlp_create(gridff_ctx* ctx, int32_t n_layers, const int32_t* sizes, gridff_mlp** out) {
  if (!ctx || !sizes || !out || n_layers < 1 || n_layers > 16) return set_err(ctx, GRIDFF_EINVAL, "bad MLP shape");
  *out = nullptr;
  if (sizes[n_layers] != kOut) return set_err(ctx, GRIDFF_EINVAL, "the output width must be %d", kOut);
  for (int l = 0; l <= n_layers; ++l)
    if (sizes[l] < 1 || sizes[l] > 4096) return set_err(ctx, GRIDFF_EINVAL, "layer width %d", sizes[l]);
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  gridff_mlp* m = new gridff_mlp();
  m->ctx = ctx;
  m->device = ctx->device;
  m->L = n_layers;
  for (int l = 0; l <= n_layers; ++l) {
    m->sizes.push_back(sizes[l]);
    m->pads.push_back(pad16(sizes[l]));
  }
  size_t off = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->woff.push_back(off);
    off += (size_t)sizes[l] * sizes[l + 1];
    m->boff.push_back(off);
    off += sizes[l + 1];
  }
  m->n_params = off;
  bool ok = dalloc(m, &m->P, off) == cudaSuccess && dalloc(m, &m->Gr, off) == cudaSuccess &&
            dalloc(m, &m->Am, off) == cudaSuccess && dalloc(m, &m->Av, off) == cudaSuccess &&
            dalloc(m, &m->desc, (size_t)sizes[0]) == cudaSuccess;
  m->Wb.assign(n_layers, nullptr);
  m->WbT.assign(n_layers, nullptr);
  for (int l = 0; l < n_layers && ok; ++l) {
    ok &= dalloc(m, &m->Wb[l], (size_t)m->pads[l] * m->pads[l + 1]) == cudaSuccess;
    ok &= dalloc(m, &m->WbT[l], (size_t)m->pads[l] * m->pads[l + 1]) == cudaSuccess;
  }
  if (!ok) {
    gridff_mlp_destroy(m);
    return set_err(ctx, GRIDFF_ENOMEM, "MLP parameters");
  }
  cudaMemsetAsync(m->P, 0, off * sizeof(float), ctx->stream);
  cudaMemsetAsync(m->Am, 0, off * sizeof(float), ctx->stream);
  cudaMemsetAsync(m->Av, 0, off * sizeof(float), ctx->stream);
  refresh_bf16(m);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    gridff_mlp_destroy(m);
    return set_err(ctx, GRIDFF_ECUDA, "MLP init");
  }
  *out = m;
  return GRIDFF_OK;
}

void gridff_mlp_destroy(gridff_mlp* m) {
  if (!m) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(m->device);
  for (void* p : m->owned) cudaFree(p);
  cudaSetDevice(prev);
  cudaGetLastError();
  delete m;
}

int64_t gridff_mlp_num_params(const gridff_mlp* m) { return m ? (int64_t)m->n_params : 0; }

gridff_status gridff_mlp_set_params(gridff_mlp* m, const float* params) {
  if (!m || !params) return GRIDFF_EINVAL;
  gridff_ctx* ctx = m->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->P, params, m->n_params * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  GRIDFF_CUDA(ctx, cudaMemsetAsync(m->Am, 0, m->n_params * sizeof(float), ctx->stream));
  GRIDFF_CUDA(ctx, cudaMemsetAsync(m->Av, 0, m->n_params * sizeof(float), ctx->stream));
  m->t = 0;
  refresh_bf16(m);
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return GRIDFF_OK;
}

gridff_status gridff_mlp_get_params(gridff_mlp* m, float* params, float* grads) {
  if (!m) return GRIDFF_EINVAL;
  gridff_ctx* ctx = m->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  if (params)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(params, m->P, m->n_params * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (grads)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(grads, m->Gr, m->n_params * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return GRIDFF_OK;
}

gridff_status gridff_mlp_forward(gridff_mlp* m, int32_t rows, const float* x, float* y) {
  NvtxRange nvtx_range("gridff_mlp_forward");
  if (!m || !x || !y || rows < 1) return set_err(m ? m->ctx : nullptr, GRIDFF_EINVAL, "bad argument");
  gridff_ctx* ctx = m->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  gridff_status st = ensure_batch(m, rows);
  if (st != GRIDFF_OK) return st;
  cudaStream_t s = ctx->stream;
  const int Mp = pad16(rows), n_in = m->sizes[0];
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->Xs, x, (size_t)rows * n_in * sizeof(float), cudaMemcpyHostToDevice, s));
  input_kernel<<<grid1((long long)Mp * m->pads[0]), 256, 0, s>>>(m->Xs, rows, n_in, Mp, m->pads[0], m->H[0],
                                                                  m->HT[0]);
  forward_rows(m, rows);
  GRIDFF_CUDA(ctx, cudaGetLastError());
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(y, m->Y, (size_t)rows * kOut * sizeof(float), cudaMemcpyDeviceToHost, s));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

gridff_status gridff_mlp_train_step(gridff_mlp* m, int32_t n_targets, int32_t K, const float* x,
                                    const float* targets, const float* tors_mask,
                                    const gridff_train_params* tp, float* loss_out, int flags) {
  NvtxRange nvtx_range("gridff_mlp_train_step");
  if (!m || !x || !targets || !tp || n_targets < 1 || K < 1)
    return set_err(m ? m->ctx : nullptr, GRIDFF_EINVAL, "bad argument");
  gridff_ctx* ctx = m->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const int rows = n_targets * K;
  gridff_status st = ensure_batch(m, std::max(rows, n_targets));
  if (st != GRIDFF_OK) return st;
  cudaStream_t s = ctx->stream;
  const int Mp = pad16(rows), n_in = m->sizes[0];
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->Xs, x, (size_t)rows * n_in * sizeof(float), cudaMemcpyHostToDevice, s));
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->Ts, targets, (size_t)n_targets * kOut * sizeof(float), cudaMemcpyHostToDevice, s));
  if (tors_mask)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->Ms, tors_mask, (size_t)n_targets * kTors * sizeof(float),
                                     cudaMemcpyHostToDevice, s));
  input_kernel<<<grid1((long long)Mp * m->pads[0]), 256, 0, s>>>(m->Xs, rows, n_in, Mp, m->pads[0], m->H[0], m->HT[0]);
  if ((st = enqueue_train(m, n_targets, K, tors_mask != nullptr, tp, flags)) != GRIDFF_OK) return st;
  if (loss_out) {
    std::vector<float> l(n_targets);
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(l.data(), m->loss, n_targets * sizeof(float), cudaMemcpyDeviceToHost, s));
    GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
    double sum = 0;
    for (float v : l) sum += v;
    *loss_out = (float)(sum / n_targets);
  } else {
    GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  }
  GRIDFF_CUDA(ctx, cudaGetLastError());
  return GRIDFF_OK;
}

gridff_status gridff_mlp_set_targets(gridff_mlp* m, int32_t n, const float* targets, const float* tors_mask) {
  if (!m || n < 1 || !targets) return set_err(m ? m->ctx : nullptr, GRIDFF_EINVAL, "bad argument");
  gridff_ctx* ctx = m->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (void* p : {(void*)m->T_all, (void*)m->M_all}) {
    if (!p) continue;
    cudaFree(p);
    m->owned.erase(std::remove(m->owned.begin(), m->owned.end(), p), m->owned.end());
  }
  m->T_all = m->M_all = nullptr;
  m->n_all = 0;
  if (dalloc(m, &m->T_all, (size_t)n * kOut) != cudaSuccess ||
      (tors_mask && dalloc(m, &m->M_all, (size_t)n * kTors) != cudaSuccess))
    return set_err(ctx, GRIDFF_ENOMEM, "training set of %d rows", n);
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->T_all, targets, (size_t)n * kOut * sizeof(float), cudaMemcpyHostToDevice,
                                   ctx->stream));
  if (tors_mask)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->M_all, tors_mask, (size_t)n * kTors * sizeof(float), cudaMemcpyHostToDevice,
                                     ctx->stream));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  m->n_all = n;
  return GRIDFF_OK;
}

gridff_status gridff_mlp_train(gridff_mlp* m, int32_t steps, int32_t n_targets, int32_t K, const float* descriptor,
                               int32_t n_desc, uint64_t seed, const gridff_train_params* tp, float* losses) {
  NvtxRange nvtx_range("gridff_mlp_train");
  if (!m || !tp || steps < 0 || n_targets < 1 || K < 1 || n_desc < 0 || (n_desc > 0 && !descriptor))
    return set_err(m ? m->ctx : nullptr, GRIDFF_EINVAL, "bad argument");
  gridff_ctx* ctx = m->ctx;
  if (m->n_all < 1) return set_err(ctx, GRIDFF_EINVAL, "no training set (gridff_mlp_set_targets)");
  if (n_desc > m->sizes[0] || m->sizes[0] - n_desc > 64)
    return set_err(ctx, GRIDFF_EINVAL, "descriptor of %d floats for %d inputs", n_desc, m->sizes[0]);
  if ((long long)n_targets * K >= (1 << 20)) return set_err(ctx, GRIDFF_EINVAL, "batch rows must be below 2^20");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const int rows = n_targets * K;
  gridff_status st = ensure_batch(m, rows);
  if (st != GRIDFF_OK) return st;
  if (steps > m->loss_cap) {
    if (m->loss_hist) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(m->loss_hist);
      m->owned.erase(std::remove(m->owned.begin(), m->owned.end(), (void*)m->loss_hist), m->owned.end());
      m->loss_hist = nullptr;
    }
    if (dalloc(m, &m->loss_hist, (size_t)steps) != cudaSuccess) return set_err(ctx, GRIDFF_ENOMEM, "loss history");
    m->loss_cap = steps;
  }
  if (!m->ctr && dalloc(m, &m->ctr, 1) != cudaSuccess) return set_err(ctx, GRIDFF_ENOMEM, "step counters");
  cudaStream_t s = ctx->stream;
  const int Mp = pad16(rows);
  if (n_desc > 0)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->desc, descriptor, n_desc * sizeof(float), cudaMemcpyHostToDevice, s));
  // The loop is launch-bound (about 45 small launches per step), so one step
  // is captured in a CUDA graph and replayed `steps` times; everything that
  // changes between steps (random-stream step, history slot, Adam t and its
  // factors) lives in device counters advanced by the graph's first node.
  StepCounters c0{};
  c0.next_step = m->rng_step;
  c0.t = m->t;
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->ctr, &c0, sizeof(c0), cudaMemcpyHostToDevice, s));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));   // c0 is a host temporary
  if (steps > 0) {
    GRIDFF_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    step_begin_kernel<<<1, 32, 0, s>>>(m->ctr, tp->lr, tp->beta1, tp->beta2, 1);
    sample_targets_kernel<<<grid1(n_targets, 128), 128, 0, s>>>(m->T_all, m->M_all, m->n_all, n_targets,
                                                                (unsigned long long)seed, m->ctr, m->Ts, m->Ms);
    train_inputs_kernel<<<grid1((long long)Mp * m->pads[0]), 256, 0, s>>>(
        m->desc, n_desc, m->sizes[0] - n_desc, rows, (unsigned long long)seed, m->ctr, Mp, m->pads[0], m->H[0],
        m->HT[0]);
    st = enqueue_train(m, n_targets, K, m->M_all != nullptr, tp, 0, m->ctr);
    loss_mean_kernel<<<1, 256, 0, s>>>(m->loss, n_targets, m->loss_hist, m->ctr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != GRIDFF_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "training graph: %s", cudaGetErrorString(e));
    m->rng_step += steps;
    m->t += steps;
  }
  GRIDFF_CUDA(ctx, cudaGetLastError());
  if (losses && steps > 0)
    GRIDFF_CUDA(ctx, cudaMemcpyAsync(losses, m->loss_hist, steps * sizeof(float), cudaMemcpyDeviceToHost, s));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

gridff_status gridff_mlp_propose(gridff_mlp* m, gridff_replicas* R, const float* descriptor, int32_t n_desc,
                                 uint64_t seed, const double origin_xy[2], const double tile_xy[2]) {
  NvtxRange nvtx_range("gridff_mlp_propose");
  if (!m || !R || !descriptor || !origin_xy || !tile_xy) return set_err(m ? m->ctx : nullptr, GRIDFF_EINVAL, "null argument");
  gridff_ctx* ctx = m->ctx;
  if (n_desc < 0 || n_desc > m->sizes[0]) return set_err(ctx, GRIDFF_EINVAL, "descriptor longer than the input");
  if (m->sizes[0] - n_desc > 64) return set_err(ctx, GRIDFF_EINVAL, "at most 64 noise inputs per row");
  if (!(tile_xy[0] > 0 && tile_xy[1] > 0)) return set_err(ctx, GRIDFF_EINVAL, "tile lengths must be positive");
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const int rows = R->n_rep;
  gridff_status st = ensure_batch(m, rows);
  if (st != GRIDFF_OK) return st;
  cudaStream_t s = ctx->stream;
  const int Mp = pad16(rows);
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(m->desc, descriptor, n_desc * sizeof(float), cudaMemcpyHostToDevice, s));
  propose_input_kernel<<<grid1((long long)Mp * m->pads[0]), 256, 0, s>>>(m->desc, n_desc, m->sizes[0] - n_desc, rows,
                                                                         (unsigned long long)seed, Mp, m->pads[0],
                                                                         m->H[0], m->HT[0]);
  forward_rows(m, rows);
  if (R->rigid) {
    pose_kernel<<<grid1(rows, 128), 128, 0, s>>>(m->Y, rows, (float)origin_xy[0], (float)origin_xy[1],
                                                 (float)tile_xy[0], (float)tile_xy[1], R->x);
    GRIDFF_CUDA(ctx, cudaMemsetAsync(R->v, 0, 6 * (size_t)rows * sizeof(float), s));
  } else if ((st = enqueue_build_poses(R, m->Y, kOut, origin_xy, tile_xy)) != GRIDFF_OK) {
    return st;
  }
  GRIDFF_CUDA(ctx, cudaGetLastError());
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  return GRIDFF_OK;
}

// Descriptor of a molecule template (host computation, 64 floats): atom
// count, composition by mass class, charge moments, principal moments of
// inertia, size and the number of torsion terms; zero padding.
gridff_status gridff_molecule_descriptor(const gridff_molecule* mol, float* out) {
  if (!mol || !out || mol->n_atoms < 1 || !mol->xyz || !mol->mass || !mol->q) return GRIDFF_EINVAL;
  const int n = mol->n_atoms;
  for (int i = 0; i < 64; ++i) out[i] = 0.f;
  double M = 0, c[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    M += mol->mass[i];
    for (int a = 0; a < 3; ++a) c[a] += mol->mass[i] * mol->xyz[3 * i + a];
  }
  for (int a = 0; a < 3; ++a) c[a] /= M;
  int cls[5] = {0, 0, 0, 0, 0};   // <4 amu, 10-13, 13-15, 15-17, other
  double Q = 0, dip[3] = {0, 0, 0}, I[3][3] = {{0}}, rg = 0, rmax = 0;
  for (int i = 0; i < n; ++i) {
    const double m = mol->mass[i];
    cls[m < 4 ? 0 : m < 13 ? 1 : m < 15 ? 2 : m < 17 ? 3 : 4]++;
    double r[3] = {mol->xyz[3 * i] - c[0], mol->xyz[3 * i + 1] - c[1], mol->xyz[3 * i + 2] - c[2]};
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    Q += mol->q[i];
    for (int a = 0; a < 3; ++a) dip[a] += mol->q[i] * r[a];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) I[a][b] += m * ((a == b ? r2 : 0.0) - r[a] * r[b]);
    rg += m * r2;
    rmax = std::max(rmax, sqrt(r2));
  }
  // eigenvalues of the symmetric 3x3 inertia tensor (trigonometric method)
  double p1 = I[0][1] * I[0][1] + I[0][2] * I[0][2] + I[1][2] * I[1][2];
  double ev[3];
  double tr = I[0][0] + I[1][1] + I[2][2];
  if (p1 < 1e-18) {
    ev[0] = I[0][0]; ev[1] = I[1][1]; ev[2] = I[2][2];
  } else {
    double qm = tr / 3;
    double p2 = (I[0][0] - qm) * (I[0][0] - qm) + (I[1][1] - qm) * (I[1][1] - qm) + (I[2][2] - qm) * (I[2][2] - qm) + 2 * p1;
    double p = sqrt(p2 / 6);
    double Bm[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Bm[a][b] = (I[a][b] - (a == b ? qm : 0.0)) / p;
    double detB = Bm[0][0] * (Bm[1][1] * Bm[2][2] - Bm[1][2] * Bm[2][1]) -
                  Bm[0][1] * (Bm[1][0] * Bm[2][2] - Bm[1][2] * Bm[2][0]) +
                  Bm[0][2] * (Bm[1][0] * Bm[2][1] - Bm[1][1] * Bm[2][0]);
    double r = std::min(1.0, std::max(-1.0, detB / 2));
    double phi = acos(r) / 3;
    ev[0] = qm + 2 * p * cos(phi);
    ev[2] = qm + 2 * p * cos(phi + 2.0943951023931953);
    ev[1] = 3 * qm - ev[0] - ev[2];
  }
  std::sort(ev, ev + 3);
  int k = 0;
  out[k++] = n / 128.f;
  for (int j = 0; j < 5; ++j) out[k++] = (float)cls[j] / n;
  out[k++] = (float)Q;
  out[k++] = (float)sqrt(dip[0] * dip[0] + dip[1] * dip[1] + dip[2] * dip[2]) / 10.f;
  for (int j = 0; j < 3; ++j) out[k++] = (float)sqrt(ev[j] / M) / 5.f;
  out[k++] = (float)sqrt(rg / M) / 5.f;
  out[k++] = (float)rmax / 10.f;
  out[k++] = mol->n_torsions / 12.f;
  return GRIDFF_OK;
}

}  // extern "C"
