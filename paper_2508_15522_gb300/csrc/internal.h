// Internal declarations of libgridff (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "gridff.h"

#define GRIDFF_MAX_ATOMS 128          // atoms per molecule template
#define GRIDFF_ATOMS_PER_LANE 4       // GRIDFF_MAX_ATOMS / 32
#define GRIDFF_KE 14.399645f          // eV*A/e^2
#define GRIDFF_ACC 9.648533e-3f       // A/fs^2 per eV/(A*amu)

#ifdef __CUDACC__
// SplitMix64 (Steele, Lea and Flood, 2014): the output for state x
// (advance by the golden gamma, then the variant-13 mix).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
// Uniform [0, 1) from the top 24 bits of a 64-bit draw.
__device__ __forceinline__ float uniform_of(unsigned long long s) {
  return (float)(s >> 40) * (1.0f / 16777216.0f);
}
// Standard normal from one 64-bit draw by Box-Muller:
// u1 = ((s >> 40) + 1) / 2^24 in (0, 1], u2 = ((s >> 16) mod 2^24) / 2^24.
__device__ __forceinline__ float normal_of(unsigned long long s) {
  const float u1 = (float)((s >> 40) + 1) * (1.0f / 16777216.0f);
  const float u2 = (float)((s >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// Rotation matrix (row-major) of a unit quaternion (w, x, y, z).
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
#endif

struct gridff_ctx {
  int device = 0;
  int n_sm = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  volatile int* ctrl_host = nullptr;  // host-mapped: [0] abort flag
  int* ctrl_dev = nullptr;            // device alias of ctrl_host
  int* result_dev = nullptr;          // device word: OR of per-replica stop bits
  size_t l2_prev_limit = 0;           // persisting-L2 limit before the first L2-window launch
  int l2_limit_set = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0.0;
  std::string err;
};

// Record kinds: 4 slots {C, P, L, 0}, or 2 slots {P, L} for grids without
// the Coulomb channel; FP32, or FP16 / BF16 holding coefficient / scale
// with a power-of-two scale per channel.
enum RecKind { REC_F32x4 = 0, REC_F32x2 = 1, REC_F16x4 = 2, REC_F16x2 = 3, REC_BF16x4 = 4, REC_BF16x2 = 5 };
inline int rec_bytes_of(int kind) {
  return kind == REC_F32x4 ? 16 : (kind == REC_F32x2 || kind == REC_F16x4 || kind == REC_BF16x4) ? 8 : 4;
}

// Coefficient grid as the kernels see it (passed by value).
// The record array is padded so that every 4x4x4 stencil is a set of 16
// contiguous runs of 4 records:
//   padded x index p <-> logical (p - 1) mod nx, p in [0, nx + 3)
//   padded y index    likewise
//   padded z index p <-> logical clamp(p - 1, 0, nz - 1), p in [0, nz + 2)
struct GridView {
  const void* rec;
  int kind;              // RecKind
  float sC, sP, sL;      // channel scales (1 for FP32)
  int nx, ny, nz;
  int nyp, nzp;
  long long sx;          // record stride between x planes = nyp * nzp
  float x0, y0, z0;
  float inv_dx, inv_dy, inv_dz;
  float Lx, Ly, inv_Lx, inv_Ly;
  float uzf;             // floor in z spacings above the first node (ghost planes)
};

struct gridff_grid {
  gridff_ctx* ctx = nullptr;
  int device = 0;                 // kept here so that destroy never reads ctx
  int dims[3] = {0, 0, 0};
  double origin[3] = {0, 0, 0};
  double spacing[3] = {0, 0, 0};
  int channels = 0;
  int storage = 0;
  int kind = REC_F32x4;
  float scale[3] = {1.f, 1.f, 1.f};   // C, P, L
  void* rec = nullptr;
  size_t rec_bytes = 0;
  int nxp = 0, nyp = 0, nzp = 0;
  double* f64_values = nullptr;   // [C][nx][ny][nz] if kept
  double* f64_coefs = nullptr;
  int n_ch = 0;                   // channels present, in order C, P, L
  int ghost = 0;                  // node planes below the floor
  double floor_z = 0.0;           // floor = origin[2] + ghost * spacing[2]
  GridView view() const;
};

// Per-atom bonded term records (template-local atom indices).
struct BondRec { int j; int own; float k; float r0; };   // own: count the energy here
struct AngleRec { int a, b, c, role; float k, cos0, pad0, pad1; };
struct TorsionRec { int a, b, c, d; int role; int n; float V, cn0; };

// Unique bond (each bond once).
struct BondTerm { int i, j; float k, r0; };

// Rotatable bond of a flexible template: reference quadruple (a, b, c, d)
// whose dihedral is the torsion coordinate, and the atoms on c's side of
// the bond (b, c) (bit i & 31 of move[i >> 5]).  Kept in build order.
struct Rotor {
  int a, b, c, d;
  uint32_t move[4];
};

// Molecule templates as the kernels see them (all device pointers).
struct TemplateView {
  const int* natoms;        // [T]
  const int* atom_off;      // [T+1] offsets into the per-atom arrays
  const float4* body;       // [A] {x, y, z, mass}
  const float4* par;        // [A] {Q, P, L, 0}   (grid factors, Eqs. E_Coulomb, V_Morse)
  const float4* nb;         // [A] {q, R, eps, 0} (intramolecular nonbonded)
  const uint32_t* excl;     // [A*4] bit j set: pair (i, j) excluded
  const int* bond_off;      // [A+1]
  const BondRec* bonds;
  const int* angle_off;     // [A+1]
  const AngleRec* angles;
  const int* tors_off;      // [A+1]
  const TorsionRec* tors;
  const int* ub_off;        // [T+1] unique bonds
  const BondTerm* ub;
  const int* ua_off;        // [T+1] unique angles (AngleRec, role unused)
  const AngleRec* ua;
  const int* ut_off;        // [T+1] unique torsions (TorsionRec, role unused)
  const TorsionRec* ut;
  const int* rot_off;       // [T+1] rotatable bonds
  const Rotor* rot;
  const float4* rigid;      // [T] {M, I1, I2, I3}
  const float* rmax;        // [T]
  float alpha;
};

// Accumulated results of one relax/run launch (device memory of the context).
struct DevResult {
  unsigned long long atom_evals;
  int stop_bits;      // OR of GRIDFF_REP_ABORTED / GRIDFF_REP_STEPLIMIT over replicas
  int n_converged;
  int max_steps;
  int next;           // work-queue position (replicas handed out so far)
  int handoff_timeouts;   // split relaxations whose first part did not arrive in time
  int pad;
};

// Launch configuration of a relaxation (mirrors gridff_launch_config).
struct LaunchCfg {
  int kernel = -1;   // GRIDFF_KERNEL_*; -1 = not chosen (heuristic default)
  int W = 32;        // rigid sub-warp: lanes per replica
  int wpb = 4;       // warps per block
  int S = 0;         // stencil-cache slots per replica (0 = no staging)
  int queue = 0;     // work queue in decreasing cost order
  int l2win = 0;     // grid in an L2 persisting access-policy window
  int blocks = 0;    // block cap (0 = every block resident at once)
  int gcache = 0;    // flexible unique-term kernel: stencil cache in global memory
};

struct gridff_replicas {
  gridff_ctx* ctx = nullptr;
  int device = 0;              // kept here so that destroy never reads ctx
  int n_rep = 0;
  int n_atoms = 0;          // total atoms over replicas
  int n_tmpl = 0;
  int rigid = 0;
  float alpha = 1.5f;
  int max_natoms = 0;
  // device
  void* tmpl_blob = nullptr;   // one allocation holding every template array
  TemplateView tv{};
  int* rep_tmpl = nullptr;     // [n_rep]
  int* rep_off = nullptr;      // [n_rep+1]
  int* order = nullptr;        // [n_rep] replicas by decreasing estimated cost (work-queue order)
  float* x = nullptr;          // flexible [3N]; rigid [7 n_rep]
  float* v = nullptr;          // flexible [3N]; rigid [6 n_rep]
  float* fire_dt = nullptr;
  float* fire_alpha = nullptr;
  int* fire_nplus = nullptr;
  int* status = nullptr;
  int* steps = nullptr;
  double* energy = nullptr;
  int* handoff = nullptr;      // [n_rep] sub-warp schedule: first part of a split warp task written
  float4* handoff_p = nullptr; // [n_rep] rigid NVE: quaternion momentum at the end of a head part
  float* last_x = nullptr;     // final evaluation of the last relaxation: rigid [7 n_rep] poses,
  float* last_f = nullptr;     //   [6 n_rep] total force + body torque; flexible [3N] positions, [3N] forces
  float4* gval = nullptr;      // flexible: global stencil cache [16 N] (atom i of replica r: 16 rep_off[r] + ...)
  int* gkey = nullptr;         //   [N] cell of each cached stencil (-1 = empty)
  // host copy of offsets
  int* h_rep_off = nullptr;
  int* h_rot_off = nullptr;    // [n_tmpl+1] rotatable bonds (host copy)
  Rotor* h_rot = nullptr;
  LaunchCfg cfg;               // set by gridff_tune / gridff_set_launch_config
};

// error helpers -------------------------------------------------------------
gridff_status set_err(gridff_ctx* ctx, gridff_status st, const char* fmt, ...);

// Relaxation launch shared by gridff_relax, the autotuner and graph capture
// (dynamics.cu).  prepare_relax validates cfg for R and sets kernel
// attributes (not capturable); enqueue_relax puts the FIRE reset (unless
// CONTINUE), the result reset and the relaxation kernel on the context
// stream (capturable; no synchronisation).
LaunchCfg default_launch_cfg(const gridff_replicas* R, bool use_grid);
gridff_status prepare_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, const LaunchCfg& c,
                            int flags, int* blocks_out);
// Pose builder on the context stream (poses.cu): d_poses on the device,
// row r at d_poses + r * stride (GRIDFF_MLP_OUT floats used); centres
// folded into the tile when origin_xy and tile_xy are given.
gridff_status enqueue_build_poses(gridff_replicas* R, const float* d_poses, int stride, const double origin_xy[2],
                                  const double tile_xy[2]);
gridff_status enqueue_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R, const LaunchCfg& c,
                            int blocks, int nsteps, const gridff_fire_params& P, int flags);
gridff_status check_fire_params(gridff_ctx* ctx, const gridff_fire_params& P);
// Binned point evaluation (points.cu): device arrays, enqueued on the
// context stream (gridff_eval_points with GRIDFF_POINTS_BINNED).
gridff_status enqueue_eval_points_binned(gridff_ctx* ctx, const gridff_grid* grid, int64_t n, const float* xyz,
                                         const float* qpl, float* E, float* F, int32_t* status);
#define GRIDFF_CUDA(ctx, call)                                                     \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return set_err((ctx), GRIDFF_ECUDA, "%s failed: %s (%s:%d)", #call,          \
                     cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

