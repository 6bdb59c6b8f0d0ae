// Grid files: a built coefficient grid written to disk and read back, so
// that a substrate's grid is built once and reused in many simulations
// (Sec. 5).  The file holds exactly what the kernels
// read (the padded record array) plus the metadata that interprets it, and,
// when the grid kept them, the FP64 node values and coefficients.
//
// Layout (little-endian, as written by the host):
//   char[8]  magic "GRIDFF\x01\x00"
//   int32    header bytes (of the header struct below)
//   header   dims[3], nxp, nyp, nzp, channels, storage, kind, n_ch, ghost,
//            has_f64 (int32); origin[3], spacing[3], floor_z (double);
//            scale[3] (float); rec_bytes (uint64)
//   bytes    records [rec_bytes]
//   double   values [n_ch][nx][ny][nz], coefs [n_ch][nx][ny][nz] (has_f64)
#include <stdio.h>
#include <string.h>

#include <vector>

#include "internal.h"
#include "trace.h"

namespace {

constexpr char kMagic[8] = {'G', 'R', 'I', 'D', 'F', 'F', 1, 0};

struct FileHeader {
  int32_t dims[3];
  int32_t nxp, nyp, nzp;
  int32_t channels, storage, kind, n_ch, ghost, has_f64;
  double origin[3], spacing[3], floor_z;
  float scale[3];
  uint64_t rec_bytes;
};

struct File {
  FILE* f = nullptr;
  explicit File(FILE* p) : f(p) {}
  ~File() {
    if (f) fclose(f);
  }
};

bool put(FILE* f, const void* p, size_t n) { return fwrite(p, 1, n, f) == n; }
bool get(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n; }

}  // namespace

extern "C" {

gridff_status gridff_grid_save(const gridff_grid* g, const char* path) {
  NvtxRange nvtx_range("gridff_grid_save");
  if (!g || !path) return GRIDFF_EINVAL;
  gridff_ctx* ctx = g->ctx;
  GRIDFF_CUDA(ctx, cudaSetDevice(g->device));
  FileHeader h{};
  for (int a = 0; a < 3; ++a) {
    h.dims[a] = g->dims[a];
    h.origin[a] = g->origin[a];
    h.spacing[a] = g->spacing[a];
    h.scale[a] = g->scale[a];
  }
  h.nxp = g->nxp;
  h.nyp = g->nyp;
  h.nzp = g->nzp;
  h.channels = g->channels;
  h.storage = g->storage;
  h.kind = g->kind;
  h.n_ch = g->n_ch;
  h.ghost = g->ghost;
  h.has_f64 = g->f64_values && g->f64_coefs;
  h.floor_z = g->floor_z;
  h.rec_bytes = g->rec_bytes;
  GRIDFF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // the grid's build or upload has finished
  std::vector<unsigned char> rec(g->rec_bytes);
  GRIDFF_CUDA(ctx, cudaMemcpy(rec.data(), g->rec, g->rec_bytes, cudaMemcpyDeviceToHost));
  const size_t n64 = (size_t)g->dims[0] * g->dims[1] * g->dims[2] * g->n_ch;
  std::vector<double> v, c;
  if (h.has_f64) {
    v.resize(n64);
    c.resize(n64);
    GRIDFF_CUDA(ctx, cudaMemcpy(v.data(), g->f64_values, n64 * sizeof(double), cudaMemcpyDeviceToHost));
    GRIDFF_CUDA(ctx, cudaMemcpy(c.data(), g->f64_coefs, n64 * sizeof(double), cudaMemcpyDeviceToHost));
  }
  File file(fopen(path, "wb"));
  if (!file.f) return set_err(ctx, GRIDFF_EINVAL, "cannot open %s for writing", path);
  const int32_t hb = (int32_t)sizeof(FileHeader);
  bool ok = put(file.f, kMagic, sizeof(kMagic)) && put(file.f, &hb, sizeof(hb)) && put(file.f, &h, sizeof(h)) &&
            put(file.f, rec.data(), rec.size());
  if (ok && h.has_f64) ok = put(file.f, v.data(), n64 * sizeof(double)) && put(file.f, c.data(), n64 * sizeof(double));
  if (!ok) return set_err(ctx, GRIDFF_EINVAL, "write to %s failed", path);
  return GRIDFF_OK;
}

gridff_status gridff_grid_load(gridff_ctx* ctx, const char* path, gridff_grid** out) {
  NvtxRange nvtx_range("gridff_grid_load");
  if (!ctx || !path || !out) return set_err(ctx, GRIDFF_EINVAL, "null argument");
  *out = nullptr;
  File file(fopen(path, "rb"));
  if (!file.f) return set_err(ctx, GRIDFF_EINVAL, "cannot open %s", path);
  char magic[8];
  int32_t hb = 0;
  FileHeader h{};
  if (!get(file.f, magic, sizeof(magic)) || memcmp(magic, kMagic, sizeof(kMagic)) != 0)
    return set_err(ctx, GRIDFF_EINVAL, "%s is not a grid file", path);
  if (!get(file.f, &hb, sizeof(hb)) || hb != (int32_t)sizeof(FileHeader) || !get(file.f, &h, sizeof(h)))
    return set_err(ctx, GRIDFF_EINVAL, "%s: header of another layout", path);
  // the header must describe the record array it announces
  const bool dims_ok = h.dims[0] >= 4 && h.dims[1] >= 4 && h.dims[2] >= 4 && h.dims[0] <= (1 << 16) &&
                       h.dims[1] <= (1 << 16) && h.dims[2] <= (1 << 16) && h.nxp == h.dims[0] + 3 &&
                       h.nyp == h.dims[1] + 3 && h.nzp == h.dims[2] + 2;
  const bool kind_ok = h.kind >= REC_F32x4 && h.kind <= REC_BF16x2 && h.n_ch >= 1 && h.n_ch <= 3 &&
                       h.storage >= GRIDFF_STORE_F32 && h.storage <= GRIDFF_STORE_BF16 &&
                       __builtin_popcount((unsigned)h.channels & 7u) == h.n_ch;
  if (!dims_ok || !kind_ok ||
      h.rec_bytes != (uint64_t)h.nxp * h.nyp * h.nzp * (uint64_t)rec_bytes_of(h.kind) || h.ghost < 0 ||
      h.ghost >= h.dims[2])
    return set_err(ctx, GRIDFF_EINVAL, "%s: inconsistent header", path);
  std::vector<unsigned char> rec(h.rec_bytes);
  if (!get(file.f, rec.data(), rec.size())) return set_err(ctx, GRIDFF_EINVAL, "%s: truncated records", path);
  const size_t n64 = (size_t)h.dims[0] * h.dims[1] * h.dims[2] * h.n_ch;
  std::vector<double> v, c;
  if (h.has_f64) {
    v.resize(n64);
    c.resize(n64);
    if (!get(file.f, v.data(), n64 * sizeof(double)) || !get(file.f, c.data(), n64 * sizeof(double)))
      return set_err(ctx, GRIDFF_EINVAL, "%s: truncated FP64 arrays", path);
  }
  GRIDFF_CUDA(ctx, cudaSetDevice(ctx->device));
  gridff_grid* g = new gridff_grid();
  g->ctx = ctx;
  g->device = ctx->device;
  for (int a = 0; a < 3; ++a) {
    g->dims[a] = h.dims[a];
    g->origin[a] = h.origin[a];
    g->spacing[a] = h.spacing[a];
    g->scale[a] = h.scale[a];
  }
  g->nxp = h.nxp;
  g->nyp = h.nyp;
  g->nzp = h.nzp;
  g->channels = h.channels;
  g->storage = h.storage;
  g->kind = h.kind;
  g->n_ch = h.n_ch;
  g->ghost = h.ghost;
  g->floor_z = h.floor_z;
  g->rec_bytes = h.rec_bytes;
  if (cudaMalloc(&g->rec, g->rec_bytes) != cudaSuccess ||
      (h.has_f64 && (cudaMalloc(&g->f64_values, n64 * sizeof(double)) != cudaSuccess ||
                     cudaMalloc(&g->f64_coefs, n64 * sizeof(double)) != cudaSuccess))) {
    cudaGetLastError();
    gridff_grid_destroy(g);
    return set_err(ctx, GRIDFF_ENOMEM, "grid of %zu bytes", (size_t)h.rec_bytes);
  }
  cudaError_t e = cudaMemcpy(g->rec, rec.data(), g->rec_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && h.has_f64) {
    e = cudaMemcpy(g->f64_values, v.data(), n64 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->f64_coefs, c.data(), n64 * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    gridff_grid_destroy(g);
    return set_err(ctx, GRIDFF_ECUDA, "grid upload: %s", cudaGetErrorString(e));
  }
  *out = g;
  return GRIDFF_OK;
}

}  // extern "C"
