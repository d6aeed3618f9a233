// Batched ensemble entry points of libmhd (declared in include/mhd.h): many
// independent grids of one scheme, each with its own size, domain, gamma, CFL
// number and dt, advanced together -- every kernel of a stage is one launch
// over all runs, and a step is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mhd.h"
#include "mhd_host.cuh"
#include "mhd_kernels.cuh"
#include "mhd_probe.h"

using namespace mhd;

namespace {

// kernel classes that need a block table (block -> run)
enum { T_GHOST_X = 0, T_GHOST_Y, T_GHOST_Z, T_ROWS_X, T_ROWS_Y, T_ROWS_Z, T_PRIM, T_SWEEP_X, T_SWEEP_Y, T_SWEEP_Z,
       T_EDGE, T_N };
constexpr int kBlockBig = 256, kBlockSweep = 128;
constexpr int kSmallCells = 128 * 128;  // runs with at most this many cells form the "small" size class

}  // namespace

struct mhd_batch {
  int nruns = 0;
  mhd_config cfg0{};  // scheme options shared by all runs
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<RunDev> runs;  // host copy of the device descriptors
  RunDev* runs_d = nullptr;
  double* pool = nullptr;
  DevScalars* sc = nullptr;  // one per run
  std::vector<int> blk;      // T_N tables of nruns+1 entries
  int* blk_d = nullptr;
  std::vector<char> has_state;
  int seglen_small = 16, seglen_large = 16;
  long long launches = 0;
  int launches_per_step = 0;
  cudaGraphExec_t graph{};
  bool graph_ready = false;
  // the ghost shell of U^n matches its interior (set by a read-out's ghost
  // fill, cleared by anything that changes U^n)
  bool u0_ghosts_fresh = false;
  // packed state I/O: run r's slots start at pack_off[r] (nruns+1 entries)
  std::vector<long long> pack_off;
  long long* pack_off_d = nullptr;
  double* pack_stage = nullptr;  // device staging of host packed arrays (first use)
  // profiling: an event after every launch, tagged with its kernel class
  bool prof_on = false;
  int prof_n = 0;
  cudaEvent_t prof_ev[128];
  int prof_cls[128];
  // guard words: run r's fields form one guarded block at guard_base[r]
  int guard_fields = 0;
  std::vector<const double*> guard_base;
  std::vector<long long> guard_stride_w, guard_used;
};

namespace {

void prof_mark(mhd_batch* b, int cls) {
  if (!b->prof_on || b->prof_n >= 128) return;
  cudaEventRecord(b->prof_ev[b->prof_n], b->stream);
  b->prof_cls[b->prof_n] = cls;
  b->prof_n++;
}

const int* table(const mhd_batch* b, int t) { return b->blk_d + (size_t)t * (b->nruns + 1); }
int table_blocks(const mhd_batch* b, int t) { return b->blk[(size_t)t * (b->nruns + 1) + b->nruns]; }

// Threads of a batched (direct-load) sweep along d: pencils x segments.
long long sweep_rows_direct(const Grid& g, int d, int nd, int seglen) {
  long long rows = 1;
  for (int t = 0; t < nd; t++)
    if (t != d) rows *= g.n[t] + 2;
  return rows * ((g.n[d] + 1 + seglen - 1) / seglen);
}

// Block tables of every kernel class from each run's work and block size.
int build_tables(mhd_batch* b) {
  const int R = b->nruns, nd = b->cfg0.ndim;
  b->blk.assign((size_t)T_N * (R + 1), 0);
  for (int t = 0; t < T_N; t++) {
    long long acc = 0;
    for (int r = 0; r < R; r++) {
      const RunDev& run = b->runs[r];
      const Grid& g = run.g;
      long long work = 0;
      int bs = kBlockBig;
      switch (t) {
        case T_GHOST_X: case T_GHOST_Y: case T_GHOST_Z: work = ghost_layers_work(g, t - T_GHOST_X); break;
        case T_ROWS_X: case T_ROWS_Y: case T_ROWS_Z: work = ghost_rows_work(g, t - T_ROWS_X); break;
        case T_PRIM: work = nd == 2 ? prim_work<2>(g) : prim_work<3>(g); break;
        case T_SWEEP_X:
          work = sweep_rows_direct(g, 0, nd, run.seglen);
          bs = kBlockSweep;
          break;
        case T_SWEEP_Y:
          work = sweep_rows_direct(g, 1, nd, run.seglen);
          bs = kBlockSweep;
          break;
        case T_SWEEP_Z:
          work = nd == 3 ? sweep_rows_direct(g, 2, nd, run.seglen) : 0;
          bs = kBlockSweep;
          break;
        case T_EDGE: work = nd == 2 ? edge_work<2>(g) : edge_work<3>(g); break;
      }
      b->blk[(size_t)t * (R + 1) + r] = (int)acc;
      acc += (work + bs - 1) / bs;
      if (acc > INT_MAX) return MHD_ERR_ARG;
    }
    b->blk[(size_t)t * (R + 1) + R] = (int)acc;
  }
  if (!b->blk_d) CK(cudaMalloc(&b->blk_d, sizeof(int) * b->blk.size()));
  CK(cudaMemcpyAsync(b->blk_d, b->blk.data(), sizeof(int) * b->blk.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->runs_d, b->runs.data(), sizeof(RunDev) * b->runs.size(), cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return MHD_OK;
}

void set_seglens(mhd_batch* b) {
  for (auto& r : b->runs) r.seglen = (long long)r.g.n[0] * r.g.n[1] * r.g.n[2] <= kSmallCells ? b->seglen_small
                                                                                                : b->seglen_large;
}

template <int NDIM, int RECON, int RS>
void batch_sweeps(mhd_batch* b, int reg) {
  const int R = b->nruns;
  batch_sweep_kernel<0, NDIM, RECON, RS><<<table_blocks(b, T_SWEEP_X), kBlockSweep, 0, b->stream>>>(
      b->runs_d, table(b, T_SWEEP_X), R, reg, 0);
  prof_mark(b, MHD_KCLASS_SWEEP_X);
  batch_sweep_kernel<1, NDIM, RECON, RS><<<table_blocks(b, T_SWEEP_Y), kBlockSweep, 0, b->stream>>>(
      b->runs_d, table(b, T_SWEEP_Y), R, reg, 1);
  prof_mark(b, MHD_KCLASS_SWEEP_Y);
  b->launches += 2;
  if constexpr (NDIM == 3) {
    batch_sweep_kernel<2, NDIM, RECON, RS><<<table_blocks(b, T_SWEEP_Z), kBlockSweep, 0, b->stream>>>(
        b->runs_d, table(b, T_SWEEP_Z), R, reg, 1);
    prof_mark(b, MHD_KCLASS_SWEEP_Z);
    b->launches++;
  }
}
template <int NDIM, int RECON>
void batch_sweeps_r(mhd_batch* b, int reg) {
  if (b->cfg0.riemann != MHD_RIEMANN_HLLD) batch_sweeps<NDIM, RECON, RS_HLL>(b, reg);
  else if (b->cfg0.emf == MHD_EMF_UCT_HLLD) batch_sweeps<NDIM, RECON, RS_HLLD_UCT>(b, reg);
  else batch_sweeps<NDIM, RECON, RS_HLLD>(b, reg);
}
template <int NDIM>
void batch_sweeps_n(mhd_batch* b, int reg) {
  const int r = b->cfg0.recon;
  if (r == MHD_RECON_PLM) batch_sweeps_r<NDIM, RECON_PLM>(b, reg);
  else if (r == MHD_RECON_WENOZ) batch_sweeps_r<NDIM, RECON_WENOZ>(b, reg);
  else batch_sweeps_r<NDIM, RECON_PPM>(b, reg);
}

// One RK stage s of every run (the CFL dt of each run in the first stage).
void batch_stage(mhd_batch* b, int s) {
  const int rk = b->cfg0.rk, nd = b->cfg0.ndim, R = b->nruns;
  const int reg = s == 0 ? 0 : (s == 1 ? 1 : 2);
  const int out = s == 0 ? 1 : ((rk == 2 || s == 2) ? 0 : 2);
  const int mode = s == 0 ? COMB_FIRST : (rk == 2 ? COMB_RK2_FINAL : (s == 1 ? COMB_RK3_SECOND : COMB_RK3_FINAL));
  const Grid& g0 = b->runs[0].g;  // boundary kinds are shared by all runs
  for (int pass = 0; pass < 2; pass++)
    for (int d = 0; d < nd; d++) {
      if ((pass == 0) != (g0.periodic[d] != 0)) continue;
      if (g0.periodic[d]) {
        batch_ghost_periodic_kernel<<<table_blocks(b, T_GHOST_X + d), kBlockBig, 0, b->stream>>>(
            b->runs_d, table(b, T_GHOST_X + d), R, d, reg);
        prof_mark(b, MHD_KCLASS_GHOST);
        b->launches++;
      } else {
        batch_ghost_outflow_copy_kernel<<<table_blocks(b, T_GHOST_X + d), kBlockBig, 0, b->stream>>>(
            b->runs_d, table(b, T_GHOST_X + d), R, d, reg);
        prof_mark(b, MHD_KCLASS_GHOST);
        batch_ghost_outflow_normal_kernel<<<table_blocks(b, T_ROWS_X + d), kBlockBig, 0, b->stream>>>(
            b->runs_d, table(b, T_ROWS_X + d), R, d, reg);
        prof_mark(b, MHD_KCLASS_GHOST);
        b->launches += 2;
      }
    }
  const int np = table_blocks(b, T_PRIM);
  if (nd == 2) {
    if (s == 0) batch_prim_kernel<2, true><<<np, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_PRIM), R, reg);
    else batch_prim_kernel<2, false><<<np, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_PRIM), R, reg);
  } else {
    if (s == 0) batch_prim_kernel<3, true><<<np, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_PRIM), R, reg);
    else batch_prim_kernel<3, false><<<np, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_PRIM), R, reg);
  }
  prof_mark(b, MHD_KCLASS_PRIM);
  b->launches++;
  if (nd == 2) batch_sweeps_n<2>(b, reg);
  else batch_sweeps_n<3>(b, reg);
  const int ne = table_blocks(b, T_EDGE);
  const bool hlld = b->cfg0.emf == MHD_EMF_UCT_HLLD;
  if (nd == 2) {
    if (hlld) batch_emf_kernel<2, true><<<ne, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_EDGE), R, reg);
    else batch_emf_kernel<2, false><<<ne, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_EDGE), R, reg);
  } else {
    if (hlld) batch_emf_kernel<3, true><<<ne, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_EDGE), R, reg);
    else batch_emf_kernel<3, false><<<ne, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_EDGE), R, reg);
  }
  prof_mark(b, MHD_KCLASS_EMF);
  if (nd == 2) batch_ct_rk_kernel<2><<<ne, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_EDGE), R, reg, out, mode);
  else batch_ct_rk_kernel<3><<<ne, kBlockBig, 0, b->stream>>>(b->runs_d, table(b, T_EDGE), R, reg, out, mode);
  prof_mark(b, MHD_KCLASS_CT_RK);
  b->launches += 2;
}

void batch_run_step(mhd_batch* b) {
  b->u0_ghosts_fresh = false;
  for (int s = 0; s < b->cfg0.rk; s++) batch_stage(b, s);
}

void drop_graph(mhd_batch* b) {
  if (b->graph_ready) cudaGraphExecDestroy(b->graph);
  b->graph_ready = false;
}

// ghost fill of U[0] of every run (before reading the state out)
void batch_ghost_u0(mhd_batch* b) {
  const int nd = b->cfg0.ndim, R = b->nruns;
  const Grid& g0 = b->runs[0].g;
  for (int pass = 0; pass < 2; pass++)
    for (int d = 0; d < nd; d++) {
      if ((pass == 0) != (g0.periodic[d] != 0)) continue;
      if (g0.periodic[d]) {
        batch_ghost_periodic_kernel<<<table_blocks(b, T_GHOST_X + d), kBlockBig, 0, b->stream>>>(
            b->runs_d, table(b, T_GHOST_X + d), R, d, 0);
      } else {
        batch_ghost_outflow_copy_kernel<<<table_blocks(b, T_GHOST_X + d), kBlockBig, 0, b->stream>>>(
            b->runs_d, table(b, T_GHOST_X + d), R, d, 0);
        batch_ghost_outflow_normal_kernel<<<table_blocks(b, T_ROWS_X + d), kBlockBig, 0, b->stream>>>(
            b->runs_d, table(b, T_ROWS_X + d), R, d, 0);
      }
    }
}

// Packed state I/O: one thread per element of the packed array; its run by
// binary search over the run offsets, then its slot and dense index, then
// the padded cell (the mapping of copy_field).
__device__ __forceinline__ int pack_run(const long long* __restrict__ off, int nruns, long long id) {
  int lo = 0, hi = nruns;  // off[lo] <= id < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= id) lo = mid;
    else hi = mid;
  }
  return lo;
}
template <bool TO_FIELDS>
__global__ void batch_pack_kernel(const RunDev* __restrict__ runs, const long long* __restrict__ off, int nruns,
                                  double* pack) {
  const long long total = off[nruns];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int r = pack_run(off, nruns, id);
    const RunDev& R = runs[r];
    long long l = id - off[r];
    int q = 0, e[3];
    for (; q < 8; q++) {
      slot_extents(R.g, q, e);
      const long long nq = (long long)e[0] * e[1] * e[2];
      if (l < nq) break;
      l -= nq;
    }
    const int li = (int)l;  // a slot of one run holds fewer than 2^31 elements
    const int t = li / e[0];
    const int c = R.g.at(li - t * e[0], t % e[1], t / e[1]);
    if (TO_FIELDS) R.U[0].q[q][c] = pack[id];
    else pack[id] = R.U[0].q[q][c];
  }
}
// Reset every run's device scalars (bad_cell starts at the largest index).
__global__ void batch_reset_scalars_kernel(DevScalars* sc, int nruns) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  DevScalars z{};
  z.bad_cell = LLONG_MAX;
  sc[r] = z;
}

bool same_scheme(const mhd_config& a, const mhd_config& c) {
  if (a.ndim != c.ndim || a.recon != c.recon || a.riemann != c.riemann || a.rk != c.rk || a.emf != c.emf)
    return false;
  for (int s = 0; s < 2 * a.ndim; s++)
    if (a.bc[s] != c.bc[s]) return false;
  return true;
}

}  // namespace

extern "C" {

int mhd_batch_create(int nruns, const mhd_config* cfgs, mhd_batch** out) {
  if (!out || !cfgs || nruns < 1) return MHD_ERR_ARG;
  *out = nullptr;
  for (int r = 0; r < nruns; r++) {
    int rc = validate(&cfgs[r]);
    if (!rc && cfgs[r].divb != MHD_DIVB_CT) rc = MHD_ERR_ARG;  // the batched kernels are CT-only
    if (rc) return rc;
    if (!same_scheme(cfgs[0], cfgs[r])) return MHD_ERR_ARG;
  }
  mhd_batch* b = new (std::nothrow) mhd_batch();
  if (!b) return MHD_ERR_OOM;
  b->nruns = nruns;
  b->cfg0 = cfgs[0];
  if (cfgs[0].stream) {
    b->stream = (cudaStream_t)cfgs[0].stream;
  } else {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) { delete b; return MHD_ERR_CUDA; }
    b->own_stream = true;
  }
  const int ningr = cfgs[0].emf == MHD_EMF_UCT_HLLD ? 6 : 5;  // face ingredients per direction
  const int nfields = 3 * 8 + 8 + 6 + 3 * ningr + 3;
  std::vector<size_t> field(nruns);
  size_t total = 0;
  b->runs.resize(nruns);
  for (int r = 0; r < nruns; r++) {
    b->runs[r].g = make_grid(&cfgs[r]);
    const Grid& g = b->runs[r].g;
    long long elems = (long long)g.ext[0] * g.ext[1] * g.ext[2];
    if (elems > (long long)INT_MAX - 1) { mhd_batch_destroy(b); return MHD_ERR_ARG; }
    field[r] = (size_t)guard_stride(elems);
    total += (size_t)guard_block_words(nfields, (long long)field[r]);
    b->guard_used.push_back(elems);
    b->guard_stride_w.push_back((long long)field[r]);
  }
  b->guard_fields = nfields;
  if (cudaMalloc(&b->pool, total * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->sc, sizeof(DevScalars) * nruns) != cudaSuccess ||
      cudaMalloc(&b->runs_d, sizeof(RunDev) * nruns) != cudaSuccess) {
    cudaGetLastError();
    mhd_batch_destroy(b);
    return MHD_ERR_OOM;
  }
  cudaMemsetAsync(b->pool, 0, total * sizeof(double), b->stream);
  double* p = b->pool;
  for (int r = 0; r < nruns; r++) {
    RunDev& run = b->runs[r];
    guard_fill(b->stream, p, nfields, (long long)field[r], b->guard_used[r]);
    b->guard_base.push_back(p);
    p += kGuardWords;
    auto next = [&]() { double* q = p; p += field[r]; return q; };
    for (int k = 0; k < 3; k++)
      for (int q = 0; q < 8; q++) run.U[k].q[q] = next();
    for (int q = 0; q < 8; q++) run.P.q[q] = next();
    for (int q = 0; q < 6; q++) run.L.q[q] = next();
    for (int d = 0; d < 3; d++)
      for (int q = 0; q < ningr; q++) run.ING.a[d][q] = next();
    for (int d = 0; d < 3; d++) run.E.e[d] = next();
    run.sc = b->sc + r;
  }
  std::vector<DevScalars> hs(nruns);
  for (auto& h : hs) reset_scalars_host(&h);
  cudaMemcpyAsync(b->sc, hs.data(), sizeof(DevScalars) * nruns, cudaMemcpyHostToDevice, b->stream);
  set_seglens(b);
  int rc = build_tables(b);  // synchronises the stream (hs lives on this frame)
  if (rc) { mhd_batch_destroy(b); return rc; }
  b->has_state.assign(nruns, 0);
  // packed I/O offsets: run r's 8 slots in the layout of mhd_batch_set_conserved
  b->pack_off.assign(nruns + 1, 0);
  for (int r = 0; r < nruns; r++) {
    long long n = 0;
    for (int q = 0; q < 8; q++) {
      int e[3];
      slot_extents(b->runs[r].g, q, e);
      n += (long long)e[0] * e[1] * e[2];
    }
    b->pack_off[r + 1] = b->pack_off[r] + n;
  }
  if (cudaMalloc(&b->pack_off_d, sizeof(long long) * (nruns + 1)) != cudaSuccess ||
      cudaMemcpy(b->pack_off_d, b->pack_off.data(), sizeof(long long) * (nruns + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaGetLastError();
    mhd_batch_destroy(b);
    return MHD_ERR_OOM;
  }
  *out = b;
  return MHD_OK;
}

long long mhd_batch_packed_size(const mhd_batch* b) { return b ? b->pack_off[b->nruns] : -1; }

namespace {
// The device array a packed transfer reads or writes: the caller's device
// array, or the staging buffer for a host one (allocated on first use).
int pack_target(mhd_batch* b, int mem, const double* user, double** dev) {
  if (mem == MHD_MEM_DEVICE) {
    *dev = const_cast<double*>(user);
    return MHD_OK;
  }
  if (!b->pack_stage && cudaMalloc(&b->pack_stage, sizeof(double) * b->pack_off[b->nruns]) != cudaSuccess) {
    cudaGetLastError();
    b->pack_stage = nullptr;
    return MHD_ERR_OOM;
  }
  *dev = b->pack_stage;
  return MHD_OK;
}
int pack_blocks(const mhd_batch* b) {
  const long long n = b->pack_off[b->nruns];
  const long long nb = (n + 255) / 256;
  return (int)(nb < 65535LL * 64 ? nb : 65535LL * 64);
}
}  // namespace

int mhd_batch_set_conserved_packed(mhd_batch* b, int mem, const double* packed) {
  if (!b || !packed || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  double* src = nullptr;
  int rc = pack_target(b, mem, packed, &src);
  if (rc) return rc;
  if (mem == MHD_MEM_HOST)
    CK(cudaMemcpyAsync(src, packed, sizeof(double) * b->pack_off[b->nruns], cudaMemcpyHostToDevice, b->stream));
  batch_pack_kernel<true><<<pack_blocks(b), 256, 0, b->stream>>>(b->runs_d, b->pack_off_d, b->nruns, src);
  batch_reset_scalars_kernel<<<(b->nruns + 255) / 256, 256, 0, b->stream>>>(b->sc, b->nruns);
  CK(cudaGetLastError());
  b->has_state.assign(b->nruns, 1);
  b->u0_ghosts_fresh = false;
  return MHD_OK;
}

int mhd_batch_get_conserved_packed(mhd_batch* b, int mem, double* packed) {
  if (!b || !packed || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  for (int r = 0; r < b->nruns; r++)
    if (!b->has_state[r]) return MHD_ERR_STATE;
  double* dst = nullptr;
  int rc = pack_target(b, mem, packed, &dst);
  if (rc) return rc;
  if (!b->u0_ghosts_fresh) {
    batch_ghost_u0(b);
    b->u0_ghosts_fresh = true;
  }
  batch_pack_kernel<false><<<pack_blocks(b), 256, 0, b->stream>>>(b->runs_d, b->pack_off_d, b->nruns, dst);
  CK(cudaGetLastError());
  if (mem == MHD_MEM_HOST)
    CK(cudaMemcpyAsync(packed, dst, sizeof(double) * b->pack_off[b->nruns], cudaMemcpyDeviceToHost, b->stream));
  return MHD_OK;
}

int mhd_batch_destroy(mhd_batch* b) {
  if (!b) return MHD_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  cudaFree(b->pack_off_d);
  cudaFree(b->pack_stage);
  cudaFree(b->pool);
  cudaFree(b->sc);
  cudaFree(b->runs_d);
  cudaFree(b->blk_d);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return MHD_OK;
}

int mhd_batch_set_conserved(mhd_batch* b, int run, int mem, const double* const* U, const double* const* B) {
  if (!b || run < 0 || run >= b->nruns || !U || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE))
    return MHD_ERR_ARG;
  for (int q = 0; q < 5; q++)
    if (!U[q]) return MHD_ERR_ARG;
  for (int q = 0; q < 3; q++)
    if (!B[q]) return MHD_ERR_ARG;
  const RunDev& R = b->runs[run];
  for (int q = 0; q < 8; q++) {
    int e[3];
    slot_extents(R.g, q, e);
    int rc = copy_field(R.g, b->stream, R.U[0].q[q], q < 5 ? U[q] : B[q - 5], nullptr, e, true);
    if (rc) return rc;
  }
  CK(cudaMemcpyAsync(R.sc, reset_scalars_source(), sizeof(DevScalars), cudaMemcpyHostToDevice, b->stream));
  b->has_state[run] = 1;
  b->u0_ghosts_fresh = false;
  return MHD_OK;
}

int mhd_batch_get_conserved(mhd_batch* b, int run, int mem, double* const* U, double* const* B) {
  const int rc = mhd_batch_get_conserved_async(b, run, mem, U, B);
  if (rc) return rc;
  CK(cudaStreamSynchronize(b->stream));
  return MHD_OK;
}

int mhd_batch_synchronize(mhd_batch* b) {
  if (!b) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream));
  return MHD_OK;
}

int mhd_batch_get_conserved_async(mhd_batch* b, int run, int mem, double* const* U, double* const* B) {
  if (!b || run < 0 || run >= b->nruns || !U || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE))
    return MHD_ERR_ARG;
  if (!b->has_state[run]) return MHD_ERR_STATE;
  if (!b->u0_ghosts_fresh) {  // once per state: the read-outs of all runs share it
    batch_ghost_u0(b);
    b->u0_ghosts_fresh = true;
  }
  const RunDev& R = b->runs[run];
  for (int q = 0; q < 8; q++) {
    double* dst = q < 5 ? U[q] : B[q - 5];
    if (!dst) return MHD_ERR_ARG;
    int e[3];
    slot_extents(R.g, q, e);
    int rc = copy_field(R.g, b->stream, R.U[0].q[q], nullptr, dst, e, false);
    if (rc) return rc;
  }
  CK(cudaGetLastError());
  return MHD_OK;
}

int mhd_batch_step(mhd_batch* b, int nsteps) {
  if (!b || nsteps < 0) return MHD_ERR_ARG;
  for (int r = 0; r < b->nruns; r++)
    if (!b->has_state[r]) return MHD_ERR_STATE;
  if (nsteps == 0) return MHD_OK;
  if (!b->graph_ready) {
    long long before = b->launches;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    batch_run_step(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return cuda_err(e);
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_err(e);
    b->graph_ready = true;
    b->launches_per_step = (int)(b->launches - before);
    b->launches = before;
  }
  for (int s = 0; s < nsteps; s++) {
    CK(cudaGraphLaunch(b->graph, b->stream));
    b->u0_ghosts_fresh = false;
    b->launches += b->launches_per_step;
  }
  return MHD_OK;
}

int mhd_batch_autotune(mhd_batch* b, int* seglen_small, int* seglen_large) {
  if (!b) return MHD_ERR_ARG;
  for (int r = 0; r < b->nruns; r++)
    if (!b->has_state[r]) return MHD_ERR_STATE;
  // the trials advance the state: keep U[0] of every run and the device scalars
  std::vector<size_t> fsz(b->nruns);
  size_t total = 0;
  for (int r = 0; r < b->nruns; r++) {
    fsz[r] = (size_t)(b->runs[r].U[0].q[1] - b->runs[r].U[0].q[0]);
    total += fsz[r] * 8;
  }
  double* backup = nullptr;
  DevScalars* sc_backup = nullptr;
  CK(cudaMalloc(&backup, total * sizeof(double)));
  if (cudaMalloc(&sc_backup, sizeof(DevScalars) * b->nruns) != cudaSuccess) {
    cudaFree(backup);
    return MHD_ERR_OOM;
  }
  auto save = [&](bool restore) {
    double* p = backup;
    for (int r = 0; r < b->nruns; r++) {  // U[0]'s 8 fields are contiguous
      size_t bytes = fsz[r] * 8 * sizeof(double);
      if (restore) cudaMemcpyAsync(b->runs[r].U[0].q[0], p, bytes, cudaMemcpyDeviceToDevice, b->stream);
      else cudaMemcpyAsync(p, b->runs[r].U[0].q[0], bytes, cudaMemcpyDeviceToDevice, b->stream);
      p += fsz[r] * 8;
    }
    if (restore) cudaMemcpyAsync(b->sc, sc_backup, sizeof(DevScalars) * b->nruns, cudaMemcpyDeviceToDevice, b->stream);
    else cudaMemcpyAsync(sc_backup, b->sc, sizeof(DevScalars) * b->nruns, cudaMemcpyDeviceToDevice, b->stream);
  };
  save(false);
  const int cand[4] = {8, 16, 32, 64};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bs = b->seglen_small, bl = b->seglen_large;
  int rc = MHD_OK;
  for (int i = 0; i < 4 && rc == MHD_OK; i++)
    for (int j = 0; j < 4 && rc == MHD_OK; j++) {
      b->seglen_small = cand[i];
      b->seglen_large = cand[j];
      set_seglens(b);
      rc = build_tables(b);
      if (rc) break;
      batch_run_step(b);  // warm
      cudaEventRecord(e0, b->stream);
      batch_run_step(b);
      batch_run_step(b);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = MHD_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bs = cand[i]; bl = cand[j]; }
      save(true);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->seglen_small = bs;
  b->seglen_large = bl;
  set_seglens(b);
  if (rc == MHD_OK) rc = build_tables(b);
  cudaStreamSynchronize(b->stream);
  cudaFree(backup);
  cudaFree(sc_backup);
  drop_graph(b);
  if (seglen_small) *seglen_small = bs;
  if (seglen_large) *seglen_large = bl;
  return rc;
}

int mhd_batch_set_seglen(mhd_batch* b, int seglen_small, int seglen_large) {
  if (!b || seglen_small < 1 || seglen_large < 1) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream));
  b->seglen_small = seglen_small;
  b->seglen_large = seglen_large;
  set_seglens(b);
  drop_graph(b);
  return build_tables(b);
}

int mhd_batch_get_times(mhd_batch* b, double* t_out) {
  if (!b || !t_out) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream));
  std::vector<DevScalars> h(b->nruns);
  CK(copy_sync(h.data(), b->sc, sizeof(DevScalars) * b->nruns, cudaMemcpyDeviceToHost, b->stream));
  for (int r = 0; r < b->nruns; r++) t_out[r] = h[r].time;
  return MHD_OK;
}

int mhd_batch_status(mhd_batch* b, int* bad_run, long long* bad_cell) {
  if (!b) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream));
  std::vector<DevScalars> h(b->nruns);
  CK(copy_sync(h.data(), b->sc, sizeof(DevScalars) * b->nruns, cudaMemcpyDeviceToHost, b->stream));
  if (bad_run) *bad_run = -1;
  if (bad_cell) *bad_cell = -1;
  for (int r = 0; r < b->nruns; r++)
    if (h[r].status) {
      if (bad_run) *bad_run = r;
      if (bad_cell) *bad_cell = h[r].bad_cell;
      return h[r].status;
    }
  return MHD_OK;
}

long long mhd_batch_launch_count(const mhd_batch* b) { return b ? b->launches : -1; }

int mhd_batch_profile_steps(mhd_batch* b, int nsteps, double* ms_out, int* launches_out) {
  if (!b || !ms_out || nsteps < 0) return MHD_ERR_ARG;
  for (int r = 0; r < b->nruns; r++)
    if (!b->has_state[r]) return MHD_ERR_STATE;
  for (int k = 0; k < MHD_NKCLASS; k++) {
    ms_out[k] = 0.0;
    if (launches_out) launches_out[k] = 0;
  }
  for (int i = 0; i < 128; i++) CK(cudaEventCreate(&b->prof_ev[i]));
  int rc = MHD_OK;
  for (int s = 0; s < nsteps && rc == MHD_OK; s++) {
    b->prof_on = true;
    b->prof_n = 0;
    prof_mark(b, -1);
    batch_run_step(b);
    b->prof_on = false;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { rc = cuda_err(e); break; }
    for (int i = 1; i < b->prof_n; i++) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, b->prof_ev[i - 1], b->prof_ev[i]);
      ms_out[b->prof_cls[i]] += ms;
      if (launches_out) launches_out[b->prof_cls[i]]++;
    }
  }
  for (int i = 0; i < 128; i++) cudaEventDestroy(b->prof_ev[i]);
  return rc;
}

}  // extern "C"

int mhd_batch_check_guards(mhd_batch* b, int* run, int* field, long long* word) {
  if (!b || !run || !field || !word) return MHD_ERR_ARG;
  std::vector<int> nf(b->nruns, b->guard_fields);
  return guard_check_blocks(b->stream, b->nruns, b->guard_base.data(), nf.data(), b->guard_stride_w.data(),
                            b->guard_used.data(), run, field, word);
}
