// Launch configuration of relaxations: explicit setting, the autotuner
// (timed trials by coordinate descent) and CUDA-graph capture of one
// relaxation.  The computation is the same for every configuration; only
// its layout on the GPU changes.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace {

LaunchCfg from_public(const gridff_launch_config& p) {
  LaunchCfg c;
  c.kernel = p.kernel;
  c.W = p.lanes_per_replica;
  c.wpb = p.warps_per_block;
  c.S = p.cache_slots;
  c.queue = p.queue;
  c.l2win = p.l2_window;
  c.blocks = p.blocks;
  c.gcache = p.cache_global;
  return c;
}

gridff_launch_config to_public(const LaunchCfg& c) {
  gridff_launch_config p;
  p.kernel = c.kernel;
  p.lanes_per_replica = c.W;
  p.warps_per_block = c.wpb;
  p.cache_slots = c.S;
  p.queue = c.queue;
  p.l2_window = c.l2win;
  p.blocks = c.blocks;
  p.cache_global = c.gcache;
  return p;
}

bool same(const LaunchCfg& a, const LaunchCfg& b) {
  return a.kernel == b.kernel && a.W == b.W && a.wpb == b.wpb && a.S == b.S && a.queue == b.queue &&
         a.l2win == b.l2win && a.blocks == b.blocks && a.gcache == b.gcache;
}

// One copy of a replica set's mutable state (tuning trials restore it).
struct Snapshot {
  void* buf = nullptr;
  size_t nx = 0, nv = 0, n = 0;
  ~Snapshot() {
    if (buf) cudaFree(buf);
  }
  size_t bytes() const { return (nx + nv) * 4 + n * (4 * 5 + 8); }
  char* at(size_t k) const {
    const size_t offs[8] = {0,
                            nx * 4,
                            (nx + nv) * 4,
                            (nx + nv) * 4 + n * 4,
                            (nx + nv) * 4 + n * 8,
                            (nx + nv) * 4 + n * 12,
                            (nx + nv) * 4 + n * 16,
                            (nx + nv) * 4 + n * 20};
    return (char*)buf + offs[k];
  }
};

cudaError_t snap(const gridff_replicas* R, Snapshot& S, bool save, cudaStream_t s) {
  void* dev[8] = {R->x, R->v, R->fire_dt, R->fire_alpha, R->fire_nplus, R->status, R->steps, R->energy};
  const size_t sz[8] = {S.nx * 4, S.nv * 4, S.n * 4, S.n * 4, S.n * 4, S.n * 4, S.n * 4, S.n * 8};
  for (int k = 0; k < 8; ++k) {
    cudaError_t e = save ? cudaMemcpyAsync(S.at(k), dev[k], sz[k], cudaMemcpyDeviceToDevice, s)
                         : cudaMemcpyAsync(dev[k], S.at(k), sz[k], cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

struct gridff_graph {
  gridff_ctx* ctx = nullptr;
  int device = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

gridff_status gridff_set_launch_config(gridff_replicas* R, const gridff_launch_config* cfg) {
  if (!R) return GRIDFF_EINVAL;
  if (!cfg) {
    R->cfg = LaunchCfg();
    return GRIDFF_OK;
  }
  gridff_ctx* ctx = R->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  const LaunchCfg c = from_public(*cfg);
  LaunchCfg shape = c;       // the L2 window is checked at launch, where the grid is known
  shape.l2win = 0;
  int blocks = 0;
  gridff_status st = prepare_relax(ctx, nullptr, R, shape, 0, &blocks);
  if (st != GRIDFF_OK) return st;
  R->cfg = c;
  return GRIDFF_OK;
}

gridff_status gridff_get_launch_config(const gridff_replicas* R, int use_grid, gridff_launch_config* cfg) {
  if (!R || !cfg) return GRIDFF_EINVAL;
  *cfg = to_public(R->cfg.kernel >= 0 ? R->cfg : default_launch_cfg(R, use_grid != 0));
  return GRIDFF_OK;
}

gridff_status gridff_tune(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R,
                          const gridff_fire_params* prm, int32_t trial_steps, int flags,
                          gridff_launch_config* best_out, gridff_tune_trial* trials, int32_t max_trials,
                          int32_t* n_trials) {
  NvtxRange nvtx_range("gridff_tune");
  if (!ctx || !R || R->ctx != ctx) return set_err(ctx, GRIDFF_EINVAL, "bad context or replicas");
  if (!(flags & GRIDFF_NO_GRID) && !grid) return set_err(ctx, GRIDFF_EINVAL, "grid is NULL");
  if (trial_steps < 1) return set_err(ctx, GRIDFF_EINVAL, "trial_steps < 1");
  gridff_fire_params def;
  gridff_fire_params_default(&def);
  const gridff_fire_params& P = prm ? *prm : def;
  gridff_status st = check_fire_params(ctx, P);
  if (st != GRIDFF_OK) return st;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  flags &= ~(GRIDFF_CONTINUE | GRIDFF_ASYNC | GRIDFF_DEVICE_PTRS);
  const bool use_grid = !(flags & GRIDFF_NO_GRID);

  Snapshot snapshot;
  snapshot.n = R->n_rep;
  snapshot.nx = R->rigid ? 7 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  snapshot.nv = R->rigid ? 6 * (size_t)R->n_rep : 3 * (size_t)R->n_atoms;
  if (cudaMalloc(&snapshot.buf, snapshot.bytes()) != cudaSuccess)
    return set_err(ctx, GRIDFF_ENOMEM, "tuning snapshot");
  GRIDFF_CUDA(ctx, snap(R, snapshot, true, s));

  // candidate values per dimension
  std::vector<std::pair<int, int>> kernels;   // (kernel, W or wpb)
  std::vector<int> slots;
  if (R->rigid) {
    if (use_grid)
      for (int W : {8, 16, 32}) kernels.push_back({GRIDFF_KERNEL_RIGID_SUBWARP, W});
    kernels.push_back({GRIDFF_KERNEL_RIGID_QUAD, 4});
  } else {
    kernels.push_back({GRIDFF_KERNEL_FLEX_QUAD, 4});
    for (int w : {2, 4, 8}) kernels.push_back({GRIDFF_KERNEL_FLEX_TERMS, w});
  }
  for (int S : {0, 16, 32, 48, 64, 96, 128})
    if (S <= R->max_natoms) slots.push_back(S);
  if (std::find(slots.begin(), slots.end(), R->max_natoms) == slots.end()) slots.push_back(R->max_natoms);
  int max_persist = 0;
  cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device);
  const bool try_l2 = use_grid && grid && max_persist > 0;

  std::vector<std::pair<LaunchCfg, double>> seen;
  int32_t count = 0;
  auto trial = [&](LaunchCfg c, double& rate) -> gridff_status {
    // normalise the fields that do not apply to the kernel
    if (c.kernel == GRIDFF_KERNEL_RIGID_SUBWARP) {
      c.wpb = 4;
      c.S = R->max_natoms;
      c.queue = 0;
    } else {
      c.W = 32;
    }
    if (c.kernel != GRIDFF_KERNEL_FLEX_TERMS) c.queue = c.gcache = 0;
    if (c.gcache) c.S = 0;
    if (c.kernel == GRIDFF_KERNEL_RIGID_QUAD || c.kernel == GRIDFF_KERNEL_FLEX_QUAD) c.wpb = 4;
    for (auto& kv : seen)
      if (same(kv.first, c)) {
        rate = kv.second;
        return GRIDFF_OK;
      }
    rate = 0;
    double ms = 0;
    int blocks = 0;
    gridff_status ps = prepare_relax(ctx, grid, R, c, flags, &blocks);
    if (ps == GRIDFF_OK) {
      GRIDFF_CUDA(ctx, snap(R, snapshot, false, s));
      GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
      gridff_status es = enqueue_relax(ctx, grid, R, c, blocks, trial_steps, P, flags);
      if (es != GRIDFF_OK) return es;
      GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev1, s));
      DevResult h{};
      GRIDFF_CUDA(ctx, cudaMemcpyAsync(&h, ctx->result_dev, sizeof(DevResult), cudaMemcpyDeviceToHost, s));
      GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
      float fms = 0;
      GRIDFF_CUDA(ctx, cudaEventElapsedTime(&fms, ctx->ev0, ctx->ev1));
      ms = fms;
      rate = fms > 0 ? (double)h.atom_evals / (fms * 1e-3) : 0;
    } else if (ps == GRIDFF_ECUDA) {
      return ps;
    }
    seen.push_back({c, rate});
    if (trials && count < max_trials) {
      trials[count].cfg = to_public(c);
      trials[count].atom_evals_per_s = rate;
      trials[count].ms = ms;
    }
    ++count;
    return GRIDFF_OK;
  };

  LaunchCfg best = default_launch_cfg(R, use_grid);
  double best_rate = 0;
  st = trial(best, best_rate);
  for (int pass = 0; pass < 2 && st == GRIDFF_OK; ++pass) {
    // kernel / block shape
    for (auto& kw : kernels) {
      LaunchCfg c = best;
      c.kernel = kw.first;
      if (kw.first == GRIDFF_KERNEL_RIGID_SUBWARP) c.W = kw.second;
      else c.wpb = kw.second;
      if (kw.first == GRIDFF_KERNEL_FLEX_TERMS && best.kernel != GRIDFF_KERNEL_FLEX_TERMS) c.queue = 1;
      double r = 0;
      if ((st = trial(c, r)) != GRIDFF_OK) break;
      if (r > best_rate) {
        best_rate = r;
        best = c;
      }
    }
    // stencil staging: shared-memory slots, or (unique-term kernel) every
    // atom's stencil in global memory
    if (best.kernel != GRIDFF_KERNEL_RIGID_SUBWARP)
      for (int S : slots) {
        if (st != GRIDFF_OK) break;
        LaunchCfg c = best;
        c.S = S;
        c.gcache = 0;
        double r = 0;
        if ((st = trial(c, r)) != GRIDFF_OK) break;
        if (r > best_rate) {
          best_rate = r;
          best = c;
        }
      }
    if (best.kernel == GRIDFF_KERNEL_FLEX_TERMS && use_grid && st == GRIDFF_OK) {
      LaunchCfg c = best;
      c.S = 0;
      c.gcache = 1;
      double r = 0;
      if ((st = trial(c, r)) == GRIDFF_OK && r > best_rate) {
        best_rate = r;
        best = c;
      }
    }
    // work queue, L2 window
    for (int dim = 0; dim < 2 && st == GRIDFF_OK; ++dim) {
      if (dim == 0 && best.kernel != GRIDFF_KERNEL_FLEX_TERMS) continue;
      if (dim == 1 && !try_l2) continue;
      LaunchCfg c = best;
      if (dim == 0) c.queue = !c.queue;
      else c.l2win = !c.l2win;
      double r = 0;
      if ((st = trial(c, r)) != GRIDFF_OK) break;
      if (r > best_rate) {
        best_rate = r;
        best = c;
      }
    }
  }
  cudaError_t e = snap(R, snapshot, false, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st != GRIDFF_OK) return st;
  if (e != cudaSuccess) return set_err(ctx, GRIDFF_ECUDA, "restoring the state: %s", cudaGetErrorString(e));
  if (best_rate <= 0) return set_err(ctx, GRIDFF_EINVAL, "no configuration ran");
  // normalise as the trial did
  for (auto& kv : seen)
    if (kv.second == best_rate) best = kv.first;
  R->cfg = best;
  if (best_out) *best_out = to_public(best);
  if (n_trials) *n_trials = count;
  return GRIDFF_OK;
}

gridff_status gridff_relax_graph_create(gridff_ctx* ctx, const gridff_grid* grid, gridff_replicas* R,
                                        int32_t nsteps, const gridff_fire_params* prm, int flags,
                                        gridff_graph** out) {
  NvtxRange nvtx_range("gridff_relax_graph_create");
  if (!ctx || !R || !out || R->ctx != ctx) return set_err(ctx, GRIDFF_EINVAL, "null argument");
  *out = nullptr;
  if (!(flags & GRIDFF_NO_GRID) && !grid) return set_err(ctx, GRIDFF_EINVAL, "grid is NULL");
  if (grid && grid->ctx != ctx) return set_err(ctx, GRIDFF_EINVAL, "grid belongs to another context");
  if (nsteps < 0) return set_err(ctx, GRIDFF_EINVAL, "nsteps < 0");
  gridff_fire_params def;
  gridff_fire_params_default(&def);
  const gridff_fire_params& P = prm ? *prm : def;
  gridff_status st = check_fire_params(ctx, P);
  if (st != GRIDFF_OK) return st;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  if (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy)
    return set_err(ctx, GRIDFF_EINVAL, "graph capture needs a non-default context stream");
  flags &= ~(GRIDFF_ASYNC | GRIDFF_DEVICE_PTRS);
  const LaunchCfg c = R->cfg.kernel >= 0 ? R->cfg : default_launch_cfg(R, !(flags & GRIDFF_NO_GRID));
  int blocks = 0;
  if ((st = prepare_relax(ctx, grid, R, c, flags, &blocks)) != GRIDFF_OK) return st;
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  gridff_graph* G = new gridff_graph();
  G->ctx = ctx;
  G->device = ctx->device;
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    delete G;
    return set_err(ctx, GRIDFF_ECUDA, "begin capture: %s", cudaGetErrorString(e));
  }
  st = enqueue_relax(ctx, grid, R, c, blocks, nsteps, P, flags);
  e = cudaStreamEndCapture(ctx->stream, &G->graph);
  if (st == GRIDFF_OK && e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  if (st != GRIDFF_OK || e != cudaSuccess) {
    gridff_graph_destroy(G);
    cudaGetLastError();
    return st != GRIDFF_OK ? st : set_err(ctx, GRIDFF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  *out = G;
  return GRIDFF_OK;
}

gridff_status gridff_graph_launch(gridff_graph* G, gridff_relax_result* result) {
  NvtxRange nvtx_range("gridff_graph_launch");
  if (!G) return GRIDFF_EINVAL;
  gridff_ctx* ctx = G->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
  GRIDFF_CUDA(ctx, cudaGraphLaunch(G->exec, s));
  GRIDFF_CUDA(ctx, cudaEventRecord(ctx->ev1, s));
  if (!result) return GRIDFF_OK;
  DevResult h{};
  GRIDFF_CUDA(ctx, cudaMemcpyAsync(&h, ctx->result_dev, sizeof(DevResult), cudaMemcpyDeviceToHost, s));
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(s));
  float ms = 0.f;
  GRIDFF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  ctx->last_ms = ms;
  result->atom_evals = (int64_t)h.atom_evals;
  result->n_converged = h.n_converged;
  result->max_steps = h.max_steps;
  if (h.stop_bits & GRIDFF_REP_ABORTED) return set_err(ctx, GRIDFF_EABORTED, "aborted by the host flag");
  if (h.stop_bits & GRIDFF_REP_STEPLIMIT) return set_err(ctx, GRIDFF_ESTEPLIMIT, "clock budget exhausted");
  return GRIDFF_OK;
}

void gridff_graph_destroy(gridff_graph* G) {
  if (!G) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(G->device);
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  cudaSetDevice(prev);
  cudaGetLastError();
  delete G;
}

}  // extern "C"
