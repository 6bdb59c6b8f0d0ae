/*
 * gridff.h - C ABI of libgridff, a GB300 (sm_103a) implementation of the hot
 * path of GridFF: molecule-substrate interaction by tricubic B-spline
 * interpolation of precomputed substrate grids, fused with an intramolecular
 * force field and FIRE relaxation / NVE dynamics over many independent
 * replicas of a molecule (arXiv 2508.15522).
 *
 * Paper passages that define the operations (section / equation):
 *   E = sum_i E_i(r_i, t_i, Q_i)                               Sec. 3, Eq. E
 *   E_i^C = Q_i V^C(r_i)                                       Sec. 3, Eq. E_Coulomb
 *   E_i^M = P_i V^P(r_i) + L_i V^L(r_i),
 *     P_i = eps_i e^{2 alpha R_i}, L_i = -2 eps_i e^{alpha R_i},
 *     V^P = sum_j eps_j e^{-2 alpha (|r - r_j| - R_j)},
 *     V^L = sum_j eps_j e^{-alpha (|r - r_j| - R_j)}           Sec. 3, Eqs. E_Morse, V_Morse
 *   periodic substrate, vacuum padding, monopole/dipole
 *     correction; molecule folded into the surface cell       Sec. 4
 *   cubic B-spline basis, 4x4x4 stencil, z fastest in memory,
 *     forces = analytic gradient of the interpolant,
 *     coefficients fitted to reproduce the node values       Sec. 5, Eqs. Bspline1D, Bspline
 *   FIRE relaxation, force threshold                          Sec. 6, Sec. 7
 *   replicas run entirely on the GPU                          Sec. 7
 *
 * Units: Angstrom, eV, elementary charge e, fs, amu.  V^C is stored in volts
 * (the Coulomb constant k_e = 14.399645 eV A / e^2 is folded into it).
 *
 * Conventions
 *  - Every function returns a gridff_status; GRIDFF_OK is 0.  On failure
 *    gridff_last_error(ctx) returns a message (valid until the next call on
 *    that context).  Problems of single replicas (an atom below the grid, a
 *    non-finite force) never fail a call: they are reported in the
 *    per-replica status word (GRIDFF_REP_* bits).
 *  - The caller owns every array it passes.  Handles (context, grid,
 *    replicas) own the device memory they allocate; *_destroy frees it.
 *    Grids and replica sets must not be used after their context is
 *    destroyed; destroying them afterwards is allowed (it needs only the
 *    device id they recorded).
 *  - Array arguments are host pointers unless GRIDFF_DEVICE_PTRS is set in
 *    `flags`, in which case they are device pointers (e.g. torch CUDA
 *    tensors) and are used in place without copies.
 *  - All work is ordered on the context's CUDA stream.  Calls synchronise
 *    that stream before returning unless GRIDFF_ASYNC is set (device
 *    pointers only).
 *  - Layouts: "replica-major CSR": the atoms of replica r occupy rows
 *    atom_offset[r] .. atom_offset[r+1]-1 of every per-atom array; a 3-vector
 *    per atom is stored as 3 consecutive floats (x, y, z).
 *  - Not thread-safe per context; different contexts are independent.
 */
#ifndef GRIDFF_H
#define GRIDFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GRIDFF_OK = 0,
  GRIDFF_EINVAL = 1,      /* invalid argument (message says which) */
  GRIDFF_ENOMEM = 2,      /* device or host allocation failed */
  GRIDFF_ECUDA = 3,       /* CUDA runtime error (message has cudaGetErrorString) */
  GRIDFF_EABORTED = 4,    /* the host abort flag stopped a relax/run call */
  GRIDFF_ESTEPLIMIT = 5,  /* the clock budget of a relax/run call ran out */
  GRIDFF_ENOTSUP = 6,     /* combination the library does not support */
  GRIDFF_ETIMEOUT = 7     /* a bounded wait inside a kernel ran out (a relaxation split across
                             two warps did not receive its first part in time); the replicas
                             concerned keep the state of that first part */
} gridff_status;

/* per-replica status bits (status_out arrays, gridff_get_fire_state).  A
 * call ORs in what it meets over all its steps; gridff_relax starts from
 * zero unless GRIDFF_CONTINUE, the MD calls may carry BELOW and NONFINITE
 * over from earlier calls */
#define GRIDFF_REP_CONVERGED 1   /* FIRE force norm fell below f_conv */
#define GRIDFF_REP_BELOW 2       /* an atom was below the grid's floor at some evaluation
                                    (evaluated on its ghost planes, or clamped to the
                                    lowest node plane below them) */
#define GRIDFF_REP_NONFINITE 4   /* a force or position was NaN/Inf: replica frozen */
#define GRIDFF_REP_ABORTED 8     /* stopped by the abort flag before finishing */
#define GRIDFF_REP_STEPLIMIT 16  /* stopped by the clock budget before finishing */

/* flags */
#define GRIDFF_DEVICE_PTRS 1     /* array arguments are device pointers */
#define GRIDFF_ASYNC 2           /* do not synchronise before returning */
#define GRIDFF_CONTINUE 4        /* relax: keep FIRE scalars and status from the last call */
#define GRIDFF_NO_GRID 8         /* eval/relax/run: skip the grid term */
#define GRIDFF_NO_INTRA 16       /* eval/relax/run: skip the intramolecular terms */
#define GRIDFF_POINTS_BINNED 32  /* eval_points: put the points in cell order on the device first */
#define GRIDFF_TEST_NO_HANDOFF 256  /* relax (rigid sub-warp layout), test hook of the bounded wait:
                                       the first parts of split relaxations publish no hand-off,
                                       so their second parts give up after about a second and the
                                       call returns GRIDFF_ETIMEOUT; the context stays usable */

/* grid channels */
#define GRIDFF_CH_C 1            /* Coulomb V^C (volts) */
#define GRIDFF_CH_P 2            /* Pauli V^P */
#define GRIDFF_CH_L 4            /* London V^L */

/* coefficient storage (precision tiers).  A grid with the Coulomb channel
 * stores 4 slots {C, P, L, 0} per node, a grid without it 2 slots {P, L}.
 * FP16 / BF16 hold coefficient / s_ch, s_ch = 2^(e - 15) with
 * max |coefficient of the channel| < 2^e (so |value| < 2^15), rounded to
 * the nearest FP16 / BF16 number (ties to even) from the FP64 coefficient;
 * the kernels multiply by s_ch in FP32.  Interpolation, forces and the
 * channel combination stay FP32 for every tier. */
#define GRIDFF_STORE_F32 0       /* float32: 16 (4 slots) or 8 (2 slots) bytes per node */
#define GRIDFF_STORE_F16 1       /* IEEE half: 8 or 4 bytes per node, per-channel scale */
#define GRIDFF_STORE_BF16 2      /* bfloat16: 8 or 4 bytes per node, per-channel scale */

typedef struct gridff_ctx gridff_ctx;
typedef struct gridff_grid gridff_grid;
typedef struct gridff_replicas gridff_replicas;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to order all work on, or NULL to let the context create and
 * own one.  Allocates a small host-mapped control block (abort flag).
 * Errors: EINVAL (bad device), ECUDA. */
gridff_status gridff_create(int device, void* cuda_stream, gridff_ctx** out);
void gridff_destroy(gridff_ctx* ctx);
/* Message of the last failing call on ctx ("" if none); never NULL. */
const char* gridff_last_error(const gridff_ctx* ctx);
/* The stream the context orders work on (a cudaStream_t). */
void* gridff_stream(const gridff_ctx* ctx);
/* Raise (1) or clear (0) the abort flag read by running relax/run kernels
 * (host-mapped memory; may be called from another host thread). */
void gridff_set_abort(gridff_ctx* ctx, int value);

/* ------------------------------------------------------------------- grid */

/* Rigid substrate: n atoms of one periodic supercell (Sec. 3, Sec. 4). */
typedef struct {
  int32_t n_atoms;
  const double* xyz;   /* [n*3] positions (A) */
  const double* q;     /* [n] charges (e) */
  const double* R;     /* [n] Morse radii R_j (A); pair distance R_i + R_j */
  const double* eps;   /* [n] Morse eps_j (sqrt eV); pair depth eps_i eps_j */
  double cell[9];      /* rows A1, A2 (in-plane, z = 0) and A3 = (0, 0, Lz):
                          the 3D-periodic Ewald cell with vacuum padding */
} gridff_substrate;

typedef struct {
  double origin[3];    /* lower corner of the grid box (A) */
  double length[3];    /* box lengths; x and y must be a lattice period of the
                          substrate (the grid is periodic in x, y) */
  double spacing;      /* target spacing h: n = ceil(L/h - 1e-9), dx = L/n */
  double alpha;        /* Morse alpha (1/A), default 1.5 (Sec. 6) */
  double rcut;         /* hard cutoff of the Morse sums (A), default 17 (Sec. 6) */
  double ewald_tol;    /* real/reciprocal tail tolerance, default 1e-10 */
  double ewald_rcut;   /* Ewald real-space cutoff (A), default 12 */
  int32_t channels;    /* GRIDFF_CH_* mask; default C|P|L; C is skipped when
                          all substrate charges are zero */
  int32_t storage;     /* GRIDFF_STORE_*, default F32 */
  int32_t keep_f64;    /* keep the FP64 node values and coefficients for
                          gridff_grid_download_f64 */
  int32_t ghost_below; /* node planes below the box (0..64, default 0): the
                          node values are also computed at z0 - k dz,
                          k = 1..ghost_below, and fitted with the rest, so
                          that the clamped end of the fit lies that far below
                          the floor z0; the floor stays z0 (points below it
                          are flagged GRIDFF_REP_BELOW).  The grid's nodes
                          (gridff_grid_info) then start at z0 - ghost_below dz,
                          which must lie more than 0.1 A above every substrate
                          atom (else EINVAL) */
} gridff_grid_opts;

/* Fill opts with the defaults above (origin/length/spacing zeroed). */
void gridff_grid_opts_default(gridff_grid_opts* opts);

/* Build the coefficient grid of a substrate on the GPU (Sec. 3-5):
 * node values V^C (3D Ewald sum with the slab dipole correction, FP64),
 * V^P, V^L (direct sums over atoms and in-plane images within rcut, FP64),
 * then the exact B-spline coefficients (separable line solves, FP64:
 * periodic in x, y; clamped end coefficients in z, at the lowest ghost
 * plane when opts->ghost_below > 0), stored as `storage`.
 * Substrate arrays are host pointers.  Errors: EINVAL (sizes, cell, box),
 * ENOMEM, ECUDA. */
gridff_status gridff_build_grid(gridff_ctx* ctx, const gridff_substrate* sub,
                                const gridff_grid_opts* opts, gridff_grid** out);

/* Make a grid from given coefficients (host array, FP64, layout
 * [channel][ix][iy][iz], channels in the order C, P, L of `channels`).
 * Grid nodes are origin + k*spacing; x, y periodic with period dims*spacing. */
gridff_status gridff_grid_from_coefs(gridff_ctx* ctx, const double origin[3],
                                     const double spacing[3], const int32_t dims[3],
                                     int32_t channels, const double* coefs,
                                     int32_t storage, gridff_grid** out);

/* Allocation-free B-spline coefficient fit.  Some callers cannot allocate
 * device memory at the point where they fit: the device memory is already
 * reserved by another allocator (a framework's caching pool) so cudaMalloc
 * would fail, or the caller runs a latency-bound loop in which cudaFree's
 * implicit device synchronisation is not acceptable.  This entry point does
 * the fit step of gridff_build_grid without any allocation.  The paper has
 * no counterpart.  It solves the same separable collocation system
 * (periodic x, y; clamped z) for n_channels channels of FP64 node values,
 * layout [channel][ix][iy][iz]:
 *   values  device pointer to the node values (read; may equal coefs)
 *   coefs   device pointer receiving the coefficients (same layout)
 *   dims    nx, ny, nz, each in 4..4096
 * Work is ordered on the context stream; without GRIDFF_ASYNC the call
 * synchronises it.  The line-solve tables live in one fixed device array
 * of about 288 KB inside the library (every GPU that loads the library
 * holds it until the process exits); no call allocates or frees memory.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make the first call on each device before any
 * stream capture.  All calls share the array and it keeps the last call's
 * tables (each call rewrites them before use): calls that overlap on the
 * GPU (different streams or contexts on one device) race.
 * Errors: EINVAL (null pointer, n_channels < 1, a dimension outside
 * 4..4096, a pointer that is not memory of the context's device, or values
 * and coefs that overlap without being equal; the message names it), ECUDA. */
gridff_status gridff_fit_coefs_noalloc(gridff_ctx* ctx, const double* values, double* coefs,
                                       const int32_t dims[3], int32_t n_channels, int flags);

/* The floor of the grid (A): the lowest z of its domain; evaluations
 * below it are flagged GRIDFF_REP_BELOW.  The box origin z0 of
 * gridff_build_grid (its nodes start ghost_below planes lower), the first
 * node plane of gridff_grid_from_coefs. */
gridff_status gridff_grid_floor(const gridff_grid* grid, double* z_floor);

/* Grid metadata; any output pointer may be NULL.  dims and origin describe
 * the node lattice, ghost planes included. */
gridff_status gridff_grid_info(const gridff_grid* grid, int32_t dims[3], double origin[3],
                               double spacing[3], int32_t* channels, size_t* device_bytes);

/* Storage tier of the grid and its channel scales s_C, s_P, s_L (1 for
 * FP32 and for absent channels). */
gridff_status gridff_grid_storage(const gridff_grid* grid, int32_t* storage, float scales[3]);

/* Copy FP64 node values (what = 0) or coefficients (what = 1), layout
 * [channel][ix][iy][iz], to a host array.  Needs keep_f64 at build time.
 * Errors: EINVAL if not kept. */
gridff_status gridff_grid_download_f64(const gridff_grid* grid, int what, double* host_out);
void gridff_grid_destroy(gridff_grid* grid);

/* Grid files (a substrate's grid is built once and reused in many
 * simulations, Sec. 5).  gridff_grid_save writes the grid to `path`: an 8-byte magic
 * "GRIDFF\1\0", the header size (int32) and header (node counts, padded
 * extents, channels, storage, record kind, ghost planes, origin, spacing,
 * floor, channel scales, record bytes), the padded record array the
 * kernels read, and, when the grid kept them, its FP64 node values and
 * coefficients; little-endian as the host writes it.  gridff_grid_load
 * reads such a file into a new grid on ctx's device (identical records:
 * evaluations are bit for bit those of the saved grid).
 * Errors: EINVAL (null argument, unreadable file, another format or an
 * inconsistent header, a short file), ENOMEM, ECUDA. */
gridff_status gridff_grid_save(const gridff_grid* grid, const char* path);
gridff_status gridff_grid_load(gridff_ctx* ctx, const char* path, gridff_grid** out);

/* --------------------------------------------------------------- replicas */

/* One molecule template (host arrays).  Per-atom parameters of Sec. 3:
 * charge Q_i, Morse R_i and eps_i (the library forms P_i and L_i).
 * Intramolecular terms (reduced UFF-like form; Sec. 6 and Sec. 8 name UFF
 * without its terms):
 *   bond     k (r - r0)^2
 *   angle    k (cos(theta) - cos0)^2
 *   torsion  V/2 (1 - cos(n phi0) cos(n phi))
 *   nonbonded Morse (eps_i eps_j, R_i + R_j, alpha) + k_e q_i q_j / r on every
 *            pair more than two bonds apart (derived from the bonds).
 * Rigid molecules ignore the terms; their `xyz` must be the body frame:
 * principal axes, centred at the centre of mass. */
typedef struct {
  int32_t n_atoms;            /* 1..128 */
  const float* xyz;           /* [n*3] reference/body coordinates */
  const float* q;             /* [n] */
  const float* R;             /* [n] */
  const float* eps;           /* [n] */
  const float* mass;          /* [n] amu, > 0 */
  int32_t n_bonds;
  const int32_t* bonds;       /* [n_bonds*2] */
  const float* bond_k;
  const float* bond_r0;
  int32_t n_angles;
  const int32_t* angles;      /* [n_angles*3], vertex in the middle */
  const float* angle_k;
  const float* angle_cos0;
  int32_t n_torsions;
  const int32_t* torsions;    /* [n_torsions*4] */
  const float* torsion_V;
  const int32_t* torsion_n;
  const float* torsion_cos_nphi0;
} gridff_molecule;

/* Create a replica set: n_rep replicas, replica r is a copy of template
 * template_of[r].  rigid != 0: every replica is a rigid body (state =
 * pose); else flexible (state = atom positions).  Positions and velocities
 * start at zero; set them with gridff_set_state.  Errors: EINVAL, ENOMEM. */
gridff_status gridff_replicas_create(gridff_ctx* ctx, int32_t n_templates,
                                     const gridff_molecule* templates, int32_t n_rep,
                                     const int32_t* template_of, int32_t rigid,
                                     double alpha, gridff_replicas** out);
void gridff_replicas_destroy(gridff_replicas* reps);

/* Sizes: number of replicas and total atoms; atom_offset[n_rep+1] (host
 * array, may be NULL) receives the replica-major CSR offsets. */
gridff_status gridff_replicas_info(const gridff_replicas* reps, int32_t* n_rep,
                                   int32_t* n_atoms_total, int32_t* atom_offset);

/* State.  Flexible: x, v are [n_atoms_total*3] (A, A/fs).
 * Rigid: x is [n_rep*7] = centre of mass (3) + orientation quaternion
 * (w, x, y, z), v is [n_rep*6] = COM velocity (A/fs) + body-frame angular
 * velocity (rad/fs).  v may be NULL (set: zero; get: skipped). */
gridff_status gridff_set_state(gridff_replicas* reps, const float* x, const float* v, int flags);
gridff_status gridff_get_state(gridff_replicas* reps, float* x, float* v, int flags);

/* Atom positions of every replica ([n_atoms_total*3]; for rigid replicas
 * r_i = R(q) b_i + com). */
gridff_status gridff_get_positions(gridff_replicas* reps, float* x, int flags);

/* FIRE scalars and status of every replica; any pointer may be NULL. */
gridff_status gridff_get_fire_state(gridff_replicas* reps, float* dt, float* alpha,
                                    int32_t* nplus, int32_t* status, int32_t* steps,
                                    double* energy, int flags);

/* Final evaluation of each replica in the last gridff_relax call: the state
 * at which the relaxation last evaluated the forces without moving on
 * afterwards (its last iteration, convergence, or a non-finite value), and
 * the forces there, i.e. the forces that produced gridff_get_fire_state's
 * energy (Sec. 6: FIRE reads these forces; Sec. 7: force threshold).
 * Rigid: x [n_rep*7] pose (centre, quaternion), f [n_rep*6] total force
 * (lab frame, eV/A) and torque about the centre of mass (body frame,
 * eV).  Flexible: x [n_atoms_total*3] positions, f [n_atoms_total*3] forces
 * (grid + intramolecular).  Entries of replicas that the last call stopped
 * by the abort flag or the clock budget, or that it did not evaluate, keep
 * their earlier record; never-recorded entries are NaN.  Written once per
 * replica and call (not per step).  Either pointer may be NULL; host arrays
 * unless GRIDFF_DEVICE_PTRS.  Errors: EINVAL, ECUDA. */
gridff_status gridff_get_last_eval(gridff_replicas* reps, float* x, float* f, int flags);

/* ------------------------------------------------------------- evaluation */

/* Energies and forces at the current state (Sec. 3, Sec. 5):
 * E_out[n_rep]      total energy per replica (grid + intramolecular), FP64
 * F_out[n_atoms*3]  force per atom (eV/A)
 * Eatom_out[n_atoms] grid energy per atom (may be NULL)
 * status_out[n_rep] GRIDFF_REP_* bits (may be NULL)
 * grid may be NULL with GRIDFF_NO_GRID.  Errors: EINVAL, ECUDA. */
gridff_status gridff_eval(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* reps,
                          int flags, double* E_out, float* F_out, float* Eatom_out,
                          int32_t* status_out);

typedef struct {
  float dt_start;      /* fs, default 0.5 */
  float dt_max;        /* fs, default 2.0 */
  int32_t n_min;       /* default 5 */
  float f_inc;         /* default 1.1 */
  float f_dec;         /* default 0.5 */
  float alpha_start;   /* default 0.1 */
  float f_alpha;       /* default 0.99 */
  float d_max;         /* per-atom displacement cap (A), default 0.1 */
  float f_conv;        /* convergence on the force 2-norm (eV/A), default 1e-3;
                          0 runs exactly nsteps */
  double clock_budget_s;  /* stop after this many seconds of kernel time
                             (0 = none): status ESTEPLIMIT */
} gridff_fire_params;

void gridff_fire_params_default(gridff_fire_params* p);

typedef struct {
  int64_t atom_evals;      /* sum over replicas of atoms x evaluations done */
  int32_t n_converged;     /* replicas with GRIDFF_REP_CONVERGED */
  int32_t max_steps;       /* most evaluations done by one replica */
} gridff_relax_result;

/* The substrate field alone at n independent points (the grid-interpolation
 * steps of the path: fold into the tile, cell and fractional coordinates,
 * cubic B-spline weights, gather of the 4x4x4 coefficient stencil,
 * contraction, channel combination; Sec. 5 and Eqs. E, E_Coulomb, V_Morse).
 * Point i at xyz[3i..3i+2] (A) with grid factors qpl[3i..3i+2] = (Q, P, L)
 * (charge and the Morse factors of gridff_template_factors) gets
 * E[i] = Q V^C + P V^P + L V^L (eV) and F[3i..3i+2] = -grad E (eV/A);
 * status[i] (may be NULL): GRIDFF_REP_BELOW below the grid (clamped to its
 * bottom cell), GRIDFF_REP_NONFINITE for a non-finite position (E = F = 0
 * then) or result; above the grid E = F = 0.  One
 * evaluation per point, no reuse between points.  Default layout: a quad of
 * lanes per point, points in input order.  GRIDFF_POINTS_BINNED: the points
 * are first put in the order of their grid cell by a counting sort on the
 * device (bins of 1 x 1 x 4 cells, z fastest, as the coefficient records lie
 * in memory), then evaluated one lane per point in that order, so that
 * neighbouring lanes gather from the same cache lines; the results go to
 * the points' own indices and agree with the default layout up to FP32
 * summation order.  It takes stream-ordered scratch of about 12 B per point
 * and 8 B per bin (n < 2^31; ENOTSUP beyond 2^30 bins).
 * flags: GRIDFF_DEVICE_PTRS, GRIDFF_ASYNC, GRIDFF_POINTS_BINNED.  The kernel
 * time (every launch of the call) is kept for gridff_last_kernel_ms
 * (synchronous calls).  Errors: EINVAL, ENOTSUP, ECUDA. */
gridff_status gridff_eval_points(gridff_ctx* ctx, const gridff_grid* grid, int64_t n, const float* xyz,
                                 const float* qpl, float* E, float* F, int32_t* status, int flags);

/* Grid factors (Q, P, L) of the atoms of template t (Eqs. E_Coulomb,
 * V_Morse: Q = q, P = eps e^{2 alpha R}, L = -2 eps e^{alpha R}), as the
 * kernels use them: qpl[3 n_atoms(t)].  Errors: EINVAL, ECUDA. */
gridff_status gridff_template_factors(const gridff_replicas* reps, int32_t t, float* qpl);

/* FIRE relaxation of every replica for up to nsteps iterations in one
 * persistent launch (layout per gridff_launch_config; state kept in
 * registers or shared memory).  FIRE as the paper's relaxations use it
 * (Sec. 6: relaxed scans and the timing runs; Sec. 7: relaxation of every
 * replica on the GPU with a force-norm threshold).
 * Iteration: forces; convergence test |F|_2 < f_conv (rigid: |F_tot|^2 +
 * |tau|^2); P = F.v; P > 0: mix v towards F, grow dt after n_min steps;
 * else v = 0, dt *= f_dec; semi-implicit Euler with per-atom cap d_max.
 * Rigid replicas apply the rule to (COM velocity, total force) and (body
 * angular velocity, body torque).  Without GRIDFF_CONTINUE the FIRE
 * scalars and status are reset first.  result may be NULL.  The result
 * does not depend on the layout or schedule beyond FP32 summation order
 * (rigid layouts: bit for bit).
 * Errors: EINVAL, ECUDA, EABORTED, ESTEPLIMIT (state is consistent),
 * ETIMEOUT (rigid sub-warp layout: a split relaxation's second part gave up
 * waiting for its first; the replicas concerned keep the first part's
 * state). */
gridff_status gridff_relax(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* reps,
                           int32_t nsteps, const gridff_fire_params* params, int flags,
                           gridff_relax_result* result);

/* ------------------------------------------- launch configuration, tuning */

/* How gridff_relax lays a relaxation out on the GPU.  The paper runs one
 * work-group per replica (Sec. 7); these are the GB300 layouts this
 * library offers for the same computation (every layout gives the same
 * result up to FP32 summation order). */
#define GRIDFF_KERNEL_RIGID_SUBWARP 0  /* rigid: lanes_per_replica lanes per replica, lane per atom,
                                          every atom's stencil cached (cache_slots >= atoms) */
#define GRIDFF_KERNEL_RIGID_QUAD 1     /* rigid: warp per replica, 4 lanes per atom */
#define GRIDFF_KERNEL_FLEX_QUAD 2      /* flexible: warp per replica, 4 lanes per atom for the grid
                                          and for that atom's intramolecular terms */
#define GRIDFF_KERNEL_FLEX_TERMS 3     /* flexible: warp per replica, grid by 4 lanes per atom, then
                                          each intramolecular term once (lane per term) with
                                          shared-memory force scatter */

typedef struct {
  int32_t kernel;             /* GRIDFF_KERNEL_* */
  int32_t lanes_per_replica;  /* RIGID_SUBWARP: 8, 16 or 32 */
  int32_t warps_per_block;    /* SUBWARP, QUAD kernels: 4; FLEX_TERMS: 2, 4 or 8 */
  int32_t cache_slots;        /* stencil staging: shared-memory stencil-cache slots per replica
                                 (the first cache_slots atoms keep their 4x4x4 stencil between
                                 steps); 0 = no staging, every gather from L2/HBM */
  int32_t queue;              /* FLEX_TERMS: 1 = replicas handed out by an atomic work queue in
                                 decreasing cost order (uneven sizes), 0 = static round robin.
                                 RIGID_SUBWARP: 1 = warp tasks handed out by an atomic queue,
                                 2 = the (task, iteration) grid cut into equal ranges per warp (a
                                 task may be split between two warps), 0 = per call: the queue
                                 when f_conv > 0 (replicas may stop early), else the ranges */
  int32_t l2_window;          /* 1 = the grid is put in an L2 persisting access-policy window
                                 (reserves persisting L2 for the context until gridff_destroy);
                                 no window when the call skips the grid term (GRIDFF_NO_GRID) */
  int32_t blocks;             /* 0 = as many blocks as are resident on the GPU at once; > 0 = at
                                 most this many (the kernels are persistent and loop over work);
                                 also caps gridff_run's sub-warp kernel for rigid replicas */
  int32_t cache_global;       /* FLEX_TERMS with cache_slots = 0: 1 = every atom keeps its 4x4x4
                                 channel-combined stencil (256 B) between steps in a device buffer
                                 of 260 B per atom of the set, allocated at the first use; a step
                                 whose atom stays in its cell reads 256 contiguous bytes instead of
                                 gathering 16 runs of the grid.  0 = no such buffer */
} gridff_launch_config;

/* Fix the launch configuration of relaxations of `reps` (NULL: back to the
 * library's heuristic).  Errors: EINVAL when the configuration does not
 * apply to the replica set (checked here and at launch). */
gridff_status gridff_set_launch_config(gridff_replicas* reps, const gridff_launch_config* cfg);
/* The configuration gridff_relax would use now (heuristic if none set);
 * use_grid = 0 for relaxations with GRIDFF_NO_GRID. */
gridff_status gridff_get_launch_config(const gridff_replicas* reps, int use_grid, gridff_launch_config* cfg);

typedef struct {
  gridff_launch_config cfg;
  double atom_evals_per_s;    /* measured rate of the trial (0 = did not fit) */
  double ms;                  /* kernel time of the trial */
} gridff_tune_trial;

/* Autotuner: times short relaxations (trial_steps FIRE iterations from the
 * current state, FIRE scalars reset, force threshold as in params) of
 * candidate configurations by coordinate descent over the kernel (and warps
 * per block), the stencil staging (cache slots, or the unique-term kernel's
 * global stencil cache), the work queue and the L2
 * window, picks the fastest in atom evaluations per second and makes it the
 * replica set's configuration.  The state (positions, velocities, FIRE
 * scalars, status, counters, energies) is restored afterwards.  Allocates
 * scratch for one copy of the state.  trials (may be NULL) receives up to
 * max_trials records; n_trials the number run.
 * Errors: EINVAL, ENOMEM, ECUDA. */
gridff_status gridff_tune(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* reps,
                          const gridff_fire_params* params, int32_t trial_steps, int flags,
                          gridff_launch_config* best, gridff_tune_trial* trials,
                          int32_t max_trials, int32_t* n_trials);

/* One relaxation captured in a CUDA graph: FIRE reset (unless
 * GRIDFF_CONTINUE), result reset and the persistent relaxation kernel of
 * the replica set's configuration at the time of capture, all on the
 * context stream.  Each gridff_graph_launch replays it (one graph launch);
 * the replica set, grid, nsteps and params are fixed at capture.
 * Capture needs a context stream that is not the legacy default stream.
 * Errors: EINVAL, ECUDA. */
typedef struct gridff_graph gridff_graph;
gridff_status gridff_relax_graph_create(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* reps,
                                        int32_t nsteps, const gridff_fire_params* params, int flags,
                                        gridff_graph** out);
/* Replay.  result != NULL: wait for it and fill result (as gridff_relax,
 * including EABORTED/ESTEPLIMIT); result == NULL: return after enqueueing. */
gridff_status gridff_graph_launch(gridff_graph* graph, gridff_relax_result* result);
void gridff_graph_destroy(gridff_graph* graph);

typedef struct {
  float dt;               /* fs */
  int32_t record_every;   /* energy trace cadence in steps (0 = no trace) */
  double clock_budget_s;  /* as in gridff_fire_params */
} gridff_md_params;

/* NVE dynamics for nsteps (Sec. 7: the molecular-dynamics loop of all
 * replicas runs on the GPU): velocity Verlet (flexible) or the NO_SQUISH
 * symplectic rigid-body splitting (rigid; the sub-warp kernel with the
 * time-sliced schedule of gridff_relax, the block cap of the replica set's
 * launch configuration honoured).  energy_trace (may be NULL)
 * receives [(nsteps/record_every + 1) * n_rep] total energies (FP64, eV),
 * record k of replica r at [k*n_rep + r]; record 0 is the start.
 * Errors: EINVAL, ECUDA, EABORTED, ESTEPLIMIT, ETIMEOUT (as gridff_relax). */
gridff_status gridff_run(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* reps,
                         int32_t nsteps, const gridff_md_params* params, int flags,
                         double* energy_trace);

/* ------------------------------------------------------------------ poses */

/* Poses of flexible molecules.  A pose is GRIDFF_MLP_OUT = 19 floats:
 * centre of mass (3, A), orientation quaternion (w, x, y, z; normalised on
 * use, zero = no rotation), torsion angles (GRIDFF_MAX_ROTORS = 12, rad).
 * The torsions act on the template's rotatable bonds, defined from its
 * bonds and torsion terms: root = the lowest-index atom with one bond
 * (atom 0 if none); a breadth-first search from it (neighbours in
 * increasing index order) gives parents and depths; the candidates are the
 * distinct central bonds of the torsion terms in the order of their first
 * term; a candidate is rotatable when it is a search-tree edge (b = parent
 * end, c = child end) not in a ring, b has a parent and c another
 * neighbour; the first 12 are kept and ordered by the depth of b (stable).
 * Rotor k's coordinate is the dihedral of (parent(b), b, c, d), d the
 * lowest-index neighbour of c other than b (IUPAC sign: positive for a
 * right-handed turn about b -> c); its moving side is the set of atoms
 * reached from c without crossing (b, c).  Rigid templates have none. */
#define GRIDFF_MAX_ROTORS 12

/* Rotatable bonds of template t: *n_rot, and quads[4k..4k+3] = (a, b, c, d)
 * of rotor k in build order (quads may be NULL).  Errors: EINVAL. */
gridff_status gridff_template_rotors(const gridff_replicas* reps, int32_t t, int32_t* n_rot, int32_t* quads);

/* Set the state of every replica from poses[19 r .. 19 r + 18]: flexible
 * replicas get the positions of the pose builder (from the template's
 * reference geometry, set each rotor's dihedral to its torsion by rotating
 * the moving side about the bond, in build order; then rotate about the
 * centre of mass by the normalised quaternion and put the centre at the
 * pose's), rigid replicas the pose (centre, normalised quaternion;
 * torsions ignored); velocities are zeroed.  origin_xy, tile_xy (both or
 * neither may be NULL): the centre is first folded into [origin, origin +
 * tile) in x and y.  flags: GRIDFF_DEVICE_PTRS (poses on the device),
 * GRIDFF_ASYNC.  Computed in FP32 on the device.  Errors: EINVAL, ECUDA. */
gridff_status gridff_build_poses(gridff_replicas* reps, const float* poses, const double origin_xy[2],
                                 const double tile_xy[2], int flags);

/* Lift every replica whose lowest atom lies below z_floor (A) by the
 * difference, so that its lowest atom is at z_floor (rigid: the centre of
 * mass moves; flexible: every atom moves by the same amount); replicas at or
 * above it, or with non-finite positions, are left as they are.  The rule of
 * gridff_random_poses' z_floor, applied to starting structures from other
 * sources (learned proposals, built poses; Sec. 7 starts molecules from
 * placements above the surface).  flags: GRIDFF_ASYNC.
 * Errors: EINVAL, ECUDA. */
gridff_status gridff_lift(gridff_replicas* reps, double z_floor, int flags);

/* Poses of the replicas' current state (the inverse of the builder, for
 * training targets): torsions = the rotors' dihedrals, centre = the centre
 * of mass (folded into the tile when origin_xy, tile_xy are given),
 * orientation = the unit quaternion (w >= 0) of the rotation that best maps
 * the built geometry with those torsions onto the state, mass-weighted
 * (Horn's quaternion method, FP64 on the device).  Rigid replicas: their
 * pose with w >= 0.  targets[19 n_rep]; tors_mask[12 n_rep] (may be NULL):
 * 1 for the template's rotors, 0 past them.  flags: GRIDFF_DEVICE_PTRS.
 * Errors: EINVAL, ECUDA. */
gridff_status gridff_pose_targets(const gridff_replicas* reps, const double origin_xy[2], const double tile_xy[2],
                                  float* targets, float* tors_mask, int flags);

/* --------------------------------------------------------------- sampling */

/* Random starting poses of a rigid replica set (Sec. 7: molecules start
 * from random placements over the surface).  Replica r draws six uniforms
 * u_j = (splitmix64(seed XOR splitmix64(64 r + j)) >> 40) / 2^24, j = 0..5
 * (the generator of gridff_mlp_propose): orientation by Shoemake's method,
 *   a = sqrt(1 - u0), b = sqrt(u0),
 *   q = (w, x, y, z) = (b cos 2pi u2, a sin 2pi u1, a cos 2pi u1, b sin 2pi u2),
 * centre of mass (origin_x + u3 Lx, origin_y + u4 Ly, z_lo + u5 (z_hi - z_lo)),
 * then raised, if needed, until the lowest atom is at z_floor.  Velocities
 * are zeroed.  Errors: EINVAL, ENOTSUP (flexible replicas), ECUDA. */
gridff_status gridff_random_poses(gridff_replicas* reps, uint64_t seed, const double origin_xy[2],
                                  const double tile_xy[2], double z_lo, double z_hi,
                                  double z_floor);

/* RMSD uniqueness filter of relaxed rigid poses (Sec. 7).  poses [n][7]
 * (centre of mass, quaternion; normalised here) are poses of template
 * `tmpl` of reps, ordered by the caller (e.g. by energy).  RMSD between
 * two poses = sqrt(mean over atoms |r_i - r'_i|^2), the centres compared
 * by the minimum image on the tile in x and y.  dup_of[i] receives the
 * smallest j < i whose RMSD to pose i is below `threshold`, else -1; a
 * pose with dup_of = -1 is a new structure.  Host arrays unless
 * GRIDFF_DEVICE_PTRS.  Errors: EINVAL, ECUDA. */
gridff_status gridff_rmsd_unique(gridff_replicas* reps, int32_t tmpl, int32_t n, const float* poses,
                                 const double tile_xy[2], double threshold, int32_t* dup_of,
                                 int flags);

/* --------------------------------------------------------- pose proposal */

/* Learned proposal of starting poses for relaxations.  The paper has no
 * counterpart: its sampling starts from random poses and Langevin heating
 * (Sec. 7); this network learns where relaxed minima lie and proposes
 * starting poses near them.
 *
 * Network: sizes[0] inputs (molecule descriptor followed by N(0,1) noise),
 * n_layers fully connected layers a_l = h_{l-1} W_l^T + b_l, ReLU on the
 * hidden layers, linear output of GRIDFF_MLP_OUT = 19 values:
 * centre of mass (3, A), orientation (4, normalised on use), torsions (12,
 * rad).  W_l is [sizes[l+1]][sizes[l]] row-major.  Parameters are held in
 * FP32 (master copy, Adam moments); every GEMM runs with bfloat16 operands
 * (round to nearest even) and FP32 accumulation on the tensor cores.
 * The flat parameter order is W_0, b_0, W_1, b_1, ...  */
#define GRIDFF_MLP_OUT 19
#define GRIDFF_MLP_NO_UPDATE 1   /* train_step: gradients only, no Adam step */

typedef struct gridff_mlp gridff_mlp;

typedef struct {
  float lr;          /* Adam learning rate */
  float beta1;       /* default 0.9 */
  float beta2;       /* default 0.999 */
  float eps;         /* default 1e-8 */
  float w_q;         /* weight of the orientation term, default 1 */
  float w_t;         /* weight of the torsion terms, default 0.25 */
  double tile[2];    /* periodic tile (Lx, Ly) of the substrate, A */
} gridff_train_params;

/* Create a network with n_layers layers of widths sizes[0..n_layers]
 * (sizes[n_layers] must be 19, widths 1..4096).  Parameters start at zero;
 * set them with gridff_mlp_set_params.  Errors: EINVAL, ENOMEM, ECUDA. */
gridff_status gridff_mlp_create(gridff_ctx* ctx, int32_t n_layers, const int32_t* sizes,
                                gridff_mlp** out);
void gridff_mlp_destroy(gridff_mlp* mlp);
int64_t gridff_mlp_num_params(const gridff_mlp* mlp);

/* Copy FP32 parameters in (host array, flat order above); resets the Adam
 * moments and step counter.  get_params copies parameters and/or the
 * gradients of the last train step out (either pointer may be NULL). */
gridff_status gridff_mlp_set_params(gridff_mlp* mlp, const float* params);
gridff_status gridff_mlp_get_params(gridff_mlp* mlp, float* params, float* grads);

/* Forward pass: x [rows][sizes[0]] (host, FP32) -> y [rows][19] (host). */
gridff_status gridff_mlp_forward(gridff_mlp* mlp, int32_t rows, const float* x, float* y);

/* One training step with the winner-takes-all pose loss.  x holds
 * n_targets*K input rows (row b*K + k is proposal k of target b);
 * targets [n_targets][19] are relaxed poses (unit quaternion);
 * tors_mask [n_targets][12] (may be NULL = no torsions) selects the live
 * torsions.  Distance of an output o to a target t:
 *   |c - t_c|^2 (x, y by minimum image on the tile)
 *   + w_q (1 - (q . t_q)^2), q = o_q / |o_q|
 *   + w_t sum_j mask_j (1 - cos(o_j - t_j));
 * loss = mean over targets of the minimum over its K proposals; only the
 * winning proposal back-propagates.  Then one Adam step (unless
 * GRIDFF_MLP_NO_UPDATE).  loss_out (may be NULL) receives the loss.
 * Errors: EINVAL, ENOMEM, ECUDA. */
gridff_status gridff_mlp_train_step(gridff_mlp* mlp, int32_t n_targets, int32_t K, const float* x,
                                    const float* targets, const float* tors_mask,
                                    const gridff_train_params* params, float* loss_out, int flags);

/* Upload a training set of n target poses ([n][19], unit quaternions) and
 * optional torsion masks ([n][12], NULL = no torsions) into device memory
 * owned by the network (replaces the previous set).
 * Errors: EINVAL, ENOMEM, ECUDA. */
gridff_status gridff_mlp_set_targets(gridff_mlp* mlp, int32_t n, const float* targets,
                                     const float* tors_mask);

/* `steps` training steps on the device with no host round trip between
 * them.  Step s (a counter kept by the network across calls) draws its
 * n_targets targets from the training set, target b being row
 * splitmix64(seed XOR splitmix64(2^20 s + b)) mod n, and K input rows per
 * target: the descriptor (n_desc floats, host) followed by
 * sizes[0] - n_desc <= 64 normal draws, draw j of row m from the counter
 * 64 (2^20 s + m) + j (the generator of gridff_mlp_propose); then the
 * winner-takes-all loss, backward pass and Adam step of
 * gridff_mlp_train_step.  losses (host, may be NULL) receives the mean loss
 * of every step.  n_targets K < 2^20.  One step is captured in a CUDA graph
 * on the context's stream and replayed `steps` times (the stream must not
 * be under capture by the caller); synchronises before returning.
 * Errors: EINVAL (no training set), ENOMEM, ECUDA. */
gridff_status gridff_mlp_train(gridff_mlp* mlp, int32_t steps, int32_t n_targets, int32_t K,
                               const float* descriptor, int32_t n_desc, uint64_t seed,
                               const gridff_train_params* params, float* losses);

/* Propose one pose per replica (rigid or flexible; flexible replicas are
 * placed by the pose builder of gridff_build_poses): inputs are the
 * descriptor (n_desc <= sizes[0] floats, host) followed by
 * sizes[0] - n_desc <= 64 standard normal draws from a counter-based
 * generator: for row r (= replica) and noise index j,
 *   s = splitmix64(seed XOR splitmix64(64 r + j))   (splitmix64(x): the
 *       output of Steele-Lea-Flood SplitMix64 from state x),
 *   u1 = ((s >> 40) + 1) / 2^24,  u2 = ((s >> 16) mod 2^24) / 2^24,
 *   z = sqrt(-2 ln u1) cos(2 pi u2)   (Box-Muller, FP32).  The output's
 * centre of mass is folded into the tile [origin, origin + tile) in x and
 * y; the quaternion is normalised (identity if zero).  Writes the replica
 * state (rigid: poses; flexible: built positions) and zero velocities.
 * Errors: EINVAL, ENOMEM, ECUDA. */
gridff_status gridff_mlp_propose(gridff_mlp* mlp, gridff_replicas* reps, const float* descriptor,
                                 int32_t n_desc, uint64_t seed, const double origin_xy[2],
                                 const double tile_xy[2]);

/* 64-float descriptor of a molecule template (host computation): atom
 * count / 128; fractions of atoms by mass class (< 4, 4-13, 13-15, 15-17,
 * >= 17 amu); net charge; dipole about the centre of mass / 10; square
 * roots of the principal moments of inertia per mass / 5 (ascending);
 * radius of gyration / 5; largest distance from the centre of mass / 10;
 * torsion count / 12; zero padding.  Errors: EINVAL. */
gridff_status gridff_molecule_descriptor(const gridff_molecule* mol, float* out);

/* ----------------------------------------------------------------- Langevin */

typedef struct {
  float dt;               /* fs */
  float temperature;      /* K */
  float gamma;            /* friction (1/fs) */
  uint64_t seed;          /* noise stream */
  int64_t step0;          /* global index of the first step of this call (noise counter) */
  double clock_budget_s;  /* as in gridff_fire_params */
} gridff_langevin_params;

/* Langevin dynamics of flexible replicas for nsteps (the thermalisation
 * step of the paper's minima hopping, Sec. 7), BAOAB splitting with
 * c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2):
 *   v += dt/2 a;  x += dt/2 v;  v = c1 v + c2 sqrt(kB T / m) xi;
 *   x += dt/2 v;  forces;  v += dt/2 a      (kB = 8.617333262e-5 eV/K).
 * xi of replica r, global step s = step0 + k, component m = 3 i + a is
 *   z(splitmix64(splitmix64(seed XOR splitmix64(r)) XOR (512 s + m)))
 * with z(.) the Box-Muller normal of gridff_mlp_propose's generator.
 * The replicas' energies receive the energy of the final state; status
 * bits ABORTED / STEPLIMIT / NONFINITE as for gridff_run.  Uses the
 * replica set's unique-term launch configuration if one is set.
 * Errors: EINVAL, ENOTSUP (rigid replicas), ECUDA, EABORTED, ESTEPLIMIT. */
gridff_status gridff_langevin(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* reps,
                              int32_t nsteps, const gridff_langevin_params* params, int flags);

/* RMSD uniqueness filter for flexible structures (Sec. 7): xyz holds n
 * structures of one molecule of n_atoms atoms ([n][n_atoms][3], ordered by
 * the caller, e.g. by energy).  RMSD of structures A, B = sqrt(mean over
 * atoms |a_i - b_i - t|^2) where t shifts B by whole tile periods in x, y
 * so that the atoms' mean positions are closest (minimum image); no
 * alignment (adsorption site and orientation count).  dup_of[i] = smallest
 * j < i within `threshold`, else -1.  Host arrays unless GRIDFF_DEVICE_PTRS.
 * Errors: EINVAL (n_atoms outside 1..128), ECUDA. */
gridff_status gridff_rmsd_unique_xyz(gridff_ctx* ctx, int32_t n_atoms, int32_t n, const float* xyz,
                                     const double tile_xy[2], double threshold, int32_t* dup_of, int flags);

/* ------------------------------------------------------------ measurement */

/* Read `bytes` of a device buffer `iters` times with a streaming kernel and
 * return the achieved read bandwidth (GB/s, best of a few launch shapes)
 * measured with CUDA events on the context stream.  `device_buf` must hold at least `bytes` (16-byte aligned,
 * multiple of 16 bytes).  Used as the L2 roofline denominator when the
 * buffer fits in L2. */
gridff_status gridff_probe_read_bandwidth(gridff_ctx* ctx, const void* device_buf,
                                          size_t bytes, int32_t iters, double* gbs_out);

/* Milliseconds of the last relax/run kernel, measured with CUDA events
 * around the launch on the context stream (0 if none yet). */
double gridff_last_kernel_ms(const gridff_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRIDFF_H */
