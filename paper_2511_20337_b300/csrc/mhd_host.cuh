// Host-side helpers shared by the single-grid and the batched entry points:
// configuration checks, the padded grid descriptor, and state copies between
// the boundary layout of include/mhd.h and the padded device fields.
#pragma once
#include <climits>
#include <cstring>

#include "mhd.h"
#include "mhd_kernels.cuh"

namespace mhd {

inline int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return MHD_OK;
  if (e == cudaErrorMemoryAllocation) return MHD_ERR_OOM;
  return MHD_ERR_CUDA;
}
#define CK(x)                         \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return cuda_err(e_); \
  } while (0)

inline int blocks_for(long long work, int threads, int cap = 148 * 32) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

inline int validate(const mhd_config* c) {
  if (!c) return MHD_ERR_ARG;
  if (c->ndim != 2 && c->ndim != 3) return MHD_ERR_ARG;
  if (c->nx < 1 || c->ny < 1 || (c->ndim == 3 && c->nz < 1)) return MHD_ERR_ARG;
  for (int d = 0; d < c->ndim; d++)
    if (!(c->x1[d] > c->x0[d])) return MHD_ERR_ARG;
  if (!(c->gamma > 1.0)) return MHD_ERR_ARG;
  if (c->recon < MHD_RECON_PLM || c->recon > MHD_RECON_PPM) return MHD_ERR_ARG;
  if (c->riemann != MHD_RIEMANN_HLL && c->riemann != MHD_RIEMANN_HLLD) return MHD_ERR_ARG;
  if (c->rk != 2 && c->rk != 3) return MHD_ERR_ARG;
  if (!(c->cfl > 0.0)) return MHD_ERR_ARG;
  if (!(c->p_floor >= 0.0)) return MHD_ERR_ARG;
  if (c->divb != MHD_DIVB_CT && c->divb != MHD_DIVB_GLM) return MHD_ERR_ARG;
  if (c->divb == MHD_DIVB_GLM && (!(c->glm_alpha >= 0.0) || c->p_floor != 0.0)) return MHD_ERR_ARG;
  if (c->emf != MHD_EMF_UCT_HLL && c->emf != MHD_EMF_UCT_HLLD) return MHD_ERR_ARG;
  if (c->emf == MHD_EMF_UCT_HLLD && (c->riemann != MHD_RIEMANN_HLLD || c->divb != MHD_DIVB_CT)) return MHD_ERR_ARG;
  for (int d = 0; d < c->ndim; d++) {
    for (int s = 0; s < 2; s++)
      if (c->bc[2 * d + s] != MHD_BC_PERIODIC && c->bc[2 * d + s] != MHD_BC_OUTFLOW) return MHD_ERR_ARG;
    if ((c->bc[2 * d] == MHD_BC_PERIODIC) != (c->bc[2 * d + 1] == MHD_BC_PERIODIC)) return MHD_ERR_ARG;
  }
  return MHD_OK;
}

inline Grid make_grid(const mhd_config* c) {
  Grid g{};
  g.ndim = c->ndim;
  g.n[0] = c->nx;
  g.n[1] = c->ny;
  g.n[2] = c->ndim == 3 ? c->nz : 1;
  g.G = c->recon == MHD_RECON_PLM ? 2 : 3;
  g.ext[0] = g.n[0] + 2 * g.G + 1;
  g.ext[1] = g.n[1] + 2 * g.G + 1;
  g.ext[2] = c->ndim == 3 ? g.n[2] + 2 * g.G + 1 : 1;
  g.sy = g.ext[0];
  g.sz = g.ext[0] * g.ext[1];
  int Gz = c->ndim == 3 ? g.G : 0;
  g.origin = Gz * g.sz + g.G * g.sy + g.G;
  for (int d = 0; d < 3; d++) {
    double x0 = d < c->ndim ? c->x0[d] : 0.0, x1 = d < c->ndim ? c->x1[d] : 1.0;
    g.dx[d] = (x1 - x0) / g.n[d];
    g.idx[d] = 1.0 / g.dx[d];
    g.periodic[d] = d < c->ndim ? (c->bc[2 * d] == MHD_BC_PERIODIC) : 1;
  }
  g.gamma = c->gamma;
  g.gm1 = c->gamma - 1.0;
  g.igm1 = 1.0 / (c->gamma - 1.0);
  g.cfl = c->cfl;
  g.p_floor = c->p_floor;
  g.glm = c->divb == MHD_DIVB_GLM;
  return g;
}

inline void reset_scalars_host(DevScalars* h) {
  memset(h, 0, sizeof(*h));
  h->bad_cell = LLONG_MAX;
}

// guard words (mhd_guard.cu): kGuardWords before a pool's first field and at
// least that many after every field, each holding the canary, a signalling NaN
// that no arithmetic produces and no memset writes
constexpr int kGuardWords = 32;
constexpr unsigned long long kGuardCanary = 0x7ff0dead5afe5afeull;
long long guard_stride(long long used);              // field stride with room for the guard after it
long long guard_block_words(int nfields, long long stride);  // a block's words, leading guard included
int guard_fill(cudaStream_t s, double* base, int nfields, long long stride, long long used);
// Scan nblocks blocks (sync): MHD_OK, or MHD_ERR_GUARD with the first damaged
// word (block, field, word: < 0 before field 0, >= 0 past the field's end).
int guard_check_blocks(cudaStream_t s, int nblocks, const double* const* bases, const int* nfields,
                       const long long* strides, const long long* used, int* block, int* field, long long* word);

// A small host<->device copy in a stream's order, waited for.  Unlike
// cudaMemcpy it does not go through the legacy default stream, so it never
// waits for the work of other contexts.
inline cudaError_t copy_sync(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, s);
  return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

// The reset values in host memory that lives as long as the library, so that
// a context can copy them to the device without waiting for the copy.
inline const DevScalars* reset_scalars_source() {
  static const DevScalars h = [] {
    DevScalars s;
    reset_scalars_host(&s);
    return s;
  }();
  return &h;
}

// cudaMemcpy3D between the caller's dense array (extents e[3]) and the
// interior of a padded device field.
inline int copy_field(const Grid& g, cudaStream_t stream, double* field, const double* ext_ptr, double* ext_out,
                      const int e[3], bool to_device) {
  cudaMemcpy3DParms p{};
  cudaPitchedPtr dense = make_cudaPitchedPtr(to_device ? (void*)ext_ptr : (void*)ext_out, (size_t)e[0] * 8, e[0], e[1]);
  cudaPitchedPtr padded = make_cudaPitchedPtr((void*)field, (size_t)g.ext[0] * 8, g.ext[0], g.ext[1]);
  int Gz = g.ndim == 3 ? g.G : 0;
  if (to_device) {
    p.srcPtr = dense;
    p.dstPtr = padded;
    p.dstPos = make_cudaPos((size_t)g.G * 8, g.G, Gz);
  } else {
    p.srcPtr = padded;
    p.srcPos = make_cudaPos((size_t)g.G * 8, g.G, Gz);
    p.dstPtr = dense;
  }
  p.extent = make_cudaExtent((size_t)e[0] * 8, e[1], e[2]);
  p.kind = cudaMemcpyDefault;
  CK(cudaMemcpy3DAsync(&p, stream));
  return MHD_OK;
}

// Extents of state slot q in the boundary layout: cells, or the staggered
// face fields of the CT scheme (slots 5..7; cell arrays with GLM).
__host__ __device__ inline void slot_extents(const Grid& g, int slot, int e[3]) {
  e[0] = g.n[0];
  e[1] = g.n[1];
  e[2] = g.n[2];
  if (!g.glm && slot >= 5 && slot < 8 && slot - 5 < g.ndim) e[slot - 5] += 1;
}


}  // namespace mhd
