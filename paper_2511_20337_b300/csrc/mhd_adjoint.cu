// Adjoint entry points of libmhd (declared in include/mhd.h): the gradient of
// a final-state functional with respect to the initial state, by the
// transpose of every kernel of the step (mhd_adjoint.cuh), with the step
// sizes frozen.
//
// Schedule for n steps with checkpoints every k steps:
//   forward   n steps on the context registers; U^0, U^k, U^2k, ... saved;
//   reverse   for each block of k steps, last block first: recompute its
//             steps from the checkpoint, keeping every stage input, then run
//             the stage transposes backwards through the block.
// The recomputes run on a second stream, with a context of their own for the
// scratch of the forward kernels, while the transposes run on the context's
// stream.  The block storage is double-buffered, and the recompute context
// stays two blocks ahead: it rebuilds the last two blocks first (with the
// step sizes given, beside the forward pass's last block, as soon as that
// block's checkpoint is saved), then block b - 2 once the transposes of block
// b have read their buffers.  Events order each block's transposes after its
// recompute.  At a 256^2 grid both are latency-bound chains of small kernels,
// so the device runs them side by side.  The recompute also keeps each
// stage's primitives (its primitive pass writes them into the block
// storage), so the transposes need no primitive pass of their own.  (The
// profiling run keeps everything in sequence on the context, so that each
// phase's events time only its own kernels.)
// Memory: ceil(n/k) + 2(k*S + 1) states (S = RK stages), 2 k*S ingredient
// and primitive sets, a second context's scratch, plus the scratch of the
// transposes; work: two forward passes and one reverse pass.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mhd.h"
#include "mhd_adjoint.cuh"
#include "mhd_ctx.cuh"
#include "mhd_host.cuh"
#include "mhd_probe.h"

using namespace mhd;

namespace mhd {

struct AdjointState {
  int nsteps = 0, ckpt_every = 0, nck = 0, nstages = 0;
  size_t fe = 0;              // elements per field
  double* pool = nullptr;     // scratch of the transposes
  double* states = nullptr;   // checkpoints, then the block's stage inputs
  size_t state_count = 0;
  double* ings = nullptr;     // UCT ingredients of every stage of the block (ningr ndim fields each)
  int ningr = 5;              // face ingredients per direction: 5, or 6 with the UCT-HLLD d^R
  size_t ing_count = 0;
  double* prims = nullptr;    // primitives of every stage of the block (8 fields each)
  F8 A[4];                    // cotangent accumulators of the stage inputs (A[3]: incoming)
  L6 Lb;                      // cotangent of the stage increment (cells)
  E3 Eb;                      // cotangent of the edge fields
  GE20 GE;                    // edge-local cotangents
  F8 WbL[3], WbR[3];          // per direction: cotangents of the face states (7 used; WbL.q[7] holds the PLM codes)
  F8 Pb;                      // cotangent of the primitives
  L6 T;                       // misfit target (padded cells)
  double* Jcell = nullptr;
  double* scal = nullptr;     // [0] J, [1..] recorded dt
  std::vector<double> dts;
  double J = 0.0;
  bool has_grad = false;
  mhd_ctx* shadow = nullptr;    // the block recomputes' context (own stream and scratch)
  cudaEvent_t ev_fwd = nullptr;           // forward pass done
  cudaEvent_t ev_rec[2] = {nullptr, nullptr};  // recompute into buffer set i done
  cudaEvent_t ev_rev[2] = {nullptr, nullptr};  // transposes reading buffer set i done
};

void adjoint_free(mhd_ctx* c) {
  if (!c || !c->adj) return;
  if (c->adj->shadow) mhd_destroy(c->adj->shadow);
  for (cudaEvent_t e : {c->adj->ev_fwd, c->adj->ev_rec[0], c->adj->ev_rec[1], c->adj->ev_rev[0], c->adj->ev_rev[1]})
    if (e) cudaEventDestroy(e);
  cudaFree(c->adj->pool);
  cudaFree(c->adj->states);
  cudaFree(c->adj->ings);
  cudaFree(c->adj->prims);
  cudaFree(c->adj->Jcell);
  cudaFree(c->adj->scal);
  delete c->adj;
  c->adj = nullptr;
}

}  // namespace mhd

namespace {

constexpr int kScratchFields = 4 * 8 + 6 + 3 + 3 * 20 + 3 * (8 + 8) + 8 + 6;

// The per-cell PLM decisions of the current direction (adj_riemann_kernel ->
// adj_recon_all_kernel), or the WENO-Z / PPM positivity fallbacks
// (adj_face_states_kernel -> adj_recon5_cell_kernel), live in the face-state
// cotangent fields' spare slot 7.
unsigned* plm_codes(const AdjointState* a, int d) { return reinterpret_cast<unsigned*>(a->WbL[d].q[7]); }

F8 state_at(const AdjointState* a, size_t idx) {
  F8 s;
  for (int q = 0; q < 8; q++) s.q[q] = a->states + (idx * 8 + q) * a->fe;
  return s;
}

// The stored primitives of stage idx, laid out like the context's.
F8 prim_at(const AdjointState* a, size_t idx) {
  F8 s;
  for (int q = 0; q < 8; q++) s.q[q] = a->prims + (idx * 8 + q) * a->fe;
  return s;
}

// The stored ingredients of stage idx, laid out like the context's (direction-major).
FaceIngr ing_at(const AdjointState* a, int ndim, size_t idx) {
  FaceIngr g{};
  const size_t ni = (size_t)a->ningr;
  for (int d = 0; d < ndim; d++)
    for (int q = 0; q < a->ningr; q++) g.a[d][q] = a->ings + (idx * ni * ndim + (size_t)d * ni + q) * a->fe;
  return g;
}

int ensure_state(mhd_ctx* c, int nsteps, int k) {
  const int S = c->cfg.rk;
  const int nck = (nsteps + k - 1) / k;
  const size_t need_states = (size_t)nck + 2 * ((size_t)k * S + 1);  // checkpoints, two block buffer sets
  AdjointState* a = c->adj;
  if (!a) {
    a = new (std::nothrow) AdjointState();
    if (!a) return MHD_ERR_OOM;
    c->adj = a;
    a->fe = c->field_elems;
    a->ningr = c->cfg.emf == MHD_EMF_UCT_HLLD ? 6 : 5;
    size_t bytes = a->fe * sizeof(double) * kScratchFields;
    if (cudaMalloc(&a->pool, bytes) != cudaSuccess) { cudaGetLastError(); adjoint_free(c); return MHD_ERR_OOM; }
    CK(cudaMemsetAsync(a->pool, 0, bytes, c->stream));
    double* p = a->pool;
    auto next = [&]() { double* r = p; p += a->fe; return r; };
    for (int r = 0; r < 4; r++)
      for (int q = 0; q < 8; q++) a->A[r].q[q] = next();
    for (int q = 0; q < 6; q++) a->Lb.q[q] = next();
    for (int d = 0; d < 3; d++) a->Eb.e[d] = next();
    for (int C = 0; C < 3; C++)
      for (int m = 0; m < 20; m++) a->GE.q[C][m] = next();
    for (int d = 0; d < 3; d++)
      for (int q = 0; q < 8; q++) {
        a->WbL[d].q[q] = next();
        a->WbR[d].q[q] = next();
      }
    for (int q = 0; q < 8; q++) a->Pb.q[q] = next();
    for (int q = 0; q < 6; q++) a->T.q[q] = next();
    long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
    if (cudaMalloc(&a->Jcell, sizeof(double) * ncell) != cudaSuccess) { cudaGetLastError(); adjoint_free(c); return MHD_ERR_OOM; }
    // the block recomputes' own context, on its own stream, and the events between the two streams
    mhd_config sc = c->cfg;
    sc.stream = nullptr;
    int rc = mhd_create(&sc, &a->shadow);
    if (rc) { adjoint_free(c); return rc; }
    a->shadow->g = c->g;
    a->shadow->seglen = c->seglen;
    // the recomputes run beside the forward and reverse passes: one
    // cooperative grid at a time on the device, the forward's
    a->shadow->fused = false;
    bool ok = true;
    for (cudaEvent_t* e : {&a->ev_fwd, &a->ev_rec[0], &a->ev_rec[1], &a->ev_rev[0], &a->ev_rev[1]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { adjoint_free(c); return MHD_ERR_CUDA; }
  }
  if (a->state_count < need_states) {
    cudaFree(a->states);
    a->states = nullptr;
    a->state_count = 0;
    if (cudaMalloc(&a->states, need_states * 8 * a->fe * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return MHD_ERR_OOM;
    }
    a->state_count = need_states;
  }
  const size_t need_ings = 2 * (size_t)k * S;
  if (a->ing_count < need_ings) {
    cudaFree(a->ings);
    cudaFree(a->prims);
    a->ings = a->prims = nullptr;
    a->ing_count = 0;
    if (cudaMalloc(&a->ings, need_ings * a->ningr * c->g.ndim * a->fe * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&a->prims, need_ings * 8 * a->fe * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return MHD_ERR_OOM;
    }
    a->ing_count = need_ings;
  }
  if (a->nsteps < nsteps || !a->scal) {
    cudaFree(a->scal);
    a->scal = nullptr;
    if (cudaMalloc(&a->scal, sizeof(double) * (nsteps + 1)) != cudaSuccess) { cudaGetLastError(); return MHD_ERR_OOM; }
  }
  a->nsteps = nsteps;
  a->ckpt_every = k;
  a->nck = nck;
  a->nstages = S;
  a->has_grad = false;
  return MHD_OK;
}

int copy_state(mhd_ctx* c, const F8& dst, const F8& src) {
  // each register's 8 fields are contiguous
  CK(cudaMemcpyAsync(dst.q[0], src.q[0], 8 * c->field_elems * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return MHD_OK;
}

void stage_coeffs(int rk, int s, double& c0, double& c1, double& cL) {
  if (s == 0) { c0 = 0.0; c1 = 1.0; cL = 1.0; return; }
  if (rk == 2) { c0 = 0.5; c1 = 0.5; cL = 0.5; return; }
  if (s == 1) { c0 = 0.75; c1 = 0.25; cL = 0.25; return; }
  c0 = 1.0 / 3.0; c1 = 2.0 / 3.0; cL = 2.0 / 3.0;
}

// Transpose of the ghost fill of A: one gather over the shell when every
// axis is periodic (the forward's single shell pass), else the per-axis
// passes backwards -- the outflow axes from the last (normal-field pass, then
// copy pass), then the periodic ones.  H: a scratch field for the normal-field
// transposes.
void adj_ghost_t(mhd_ctx* c, const F8& A, double* H) {
  const Grid& g = c->g;
  bool all_periodic = true;
  for (int d = 0; d < g.ndim; d++) all_periodic = all_periodic && g.periodic[d];
  if (all_periodic) {
    const long long cells = (long long)g.n[0] * g.n[1] * g.n[2];
    if (g.ndim == 2) adj_ghost_shell_kernel<2><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, A);
    else adj_ghost_shell_kernel<3><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, A);
    c->launches++;
    return;
  }
  for (int d = g.ndim - 1; d >= 0; d--) {
    if (g.periodic[d]) continue;
    adj_ghost_outflow_chain_kernel<<<blocks_for(ghost_rows_work(g, d), 128), 128, 0, c->stream>>>(g, A, d, H);
    adj_ghost_outflow_faces_kernel<<<blocks_for(adj_outflow_faces_work(g, d), 256), 256, 0, c->stream>>>(g, A, d,
                                                                                                         H);
    adj_ghost_outflow_copy_kernel<<<blocks_for(pass_rows(g, d), 128), 128, 0, c->stream>>>(g, A, d);
    c->launches += 3;
  }
  for (int d = g.ndim - 1; d >= 0; d--) {
    if (!g.periodic[d]) continue;
    adj_ghost_periodic_kernel<<<blocks_for(pass_rows(g, d) * g.n[d], 256), 256, 0, c->stream>>>(g, A, d);
    c->launches++;
  }
}

// Riemann transpose of direction DIR on stream st (its own face-state
// cotangents and PLM codes); the reconstruction transposes of all directions
// follow in one launch (adj_recon_all_kernel), which adds into Pb in
// direction order.
template <int NDIM, int RS, int RECON, int DIR>
void adj_riemann_dir(mhd_ctx* c, const F8& Xs, const F8& Ps, const F8& As, double dt, cudaStream_t st) {
  AdjointState* a = c->adj;
  const Grid& g = c->g;
  long long faces = 1;
  for (int d = 0; d < 3; d++) faces *= d == DIR ? g.n[d] + 1 : (d < NDIM ? g.n[d] + 2 : 1);
  if constexpr (RECON != RECON_PLM) {
    adj_face_states_kernel<DIR, NDIM, RECON><<<blocks_for(adj_face_states_work<DIR, NDIM>(g), 128), 128, 0, st>>>(
        g, Ps, a->WbL[DIR], a->WbR[DIR], plm_codes(a, DIR));
    c->launches++;
  }
  adj_riemann_kernel<DIR, NDIM, RS, RECON><<<(int)((faces + 127) / 128), 128, 0, st>>>(
      g, Ps, Xs.q[5 + DIR], a->Lb, a->GE, dt, a->WbL[DIR], a->WbR[DIR], As.q[5 + DIR], plm_codes(a, DIR));
  prof_mark(c, MHD_AKCLASS_RIEMANN);
  c->launches++;
}
// Transpose of stage s at the stage input Xs: the cotangent Aout of the
// stage output is distributed to A0 (U^n) and As (the stage input).
// The WENO-Z / PPM reconstruction transpose of direction DIR: the owner-cell
// pass into the window-slot fields T, then the gather into Pb.
template <int NDIM, int RECON, int DIR>
void adj_recon5_dir(mhd_ctx* c, const F8& Ps, const T35& T) {
  AdjointState* a = c->adj;
  const Grid& g = c->g;
  const long long cells = adj_recon5_cells<DIR, NDIM>(g, g.n[DIR] + 2);
  adj_recon5_cell_kernel<DIR, NDIM, RECON><<<blocks_for(cells, 128), 128, 0, c->stream>>>(
      g, Ps, a->WbL[DIR], a->WbR[DIR], plm_codes(a, DIR), T);
  const long long reach = adj_recon5_cells<DIR, NDIM>(g, g.n[DIR] + 6);
  adj_recon5_gather_kernel<DIR, NDIM><<<blocks_for(reach, 128), 128, 0, c->stream>>>(g, T, a->Pb);
  c->launches += 2;
}
template <int NDIM, int RS, int RECON>
int adj_stage_t(mhd_ctx* c, int s, const F8& Xs, const F8& Ps, const FaceIngr& ING, const F8& Aout, const F8& A0,
                const F8& As, double dt) {
  AdjointState* a = c->adj;
  const Grid& g = c->g;
  // what the transposes read of the forward stage -- its input Xs with the
  // ghost cells its fill wrote, its primitives Ps and its UCT ingredients ING
  // -- was kept when the block recompute ran that stage
  double c0, c1, cL;
  stage_coeffs(c->cfg.rk, s, c0, c1, cL);
  const long long edges = edge_work<NDIM>(g);
  const int nbe = blocks_for(edges, 256);
  if (c->prof_on) {  // one launch per kernel class, each timed on its own
    adj_combine_kernel<NDIM><<<nbe, 256, 0, c->stream>>>(g, Aout, A0, As, a->Lb, a->Eb, c0, c1, cL, dt);
    prof_mark(c, MHD_AKCLASS_COMBINE);
    adj_edge_kernel<NDIM, RS == RS_HLLD_UCT><<<nbe, 256, 0, c->stream>>>(g, Xs, ING, a->Eb, a->GE);
    CK(cudaMemsetAsync(a->Pb.q[0], 0, 8 * a->fe * sizeof(double), c->stream));
    c->launches += 2;
  } else {  // the same in one launch
    adj_combine_edge_kernel<NDIM, RS == RS_HLLD_UCT><<<nbe, 256, 0, c->stream>>>(g, Aout, A0, As, a->Lb, a->Eb, c0, c1, cL, dt, Xs,
                                                              ING, a->GE, a->Pb.q[0], 8 * (long long)a->fe);
    c->launches++;
  }
  long long box = (long long)(g.n[0] + 4) * (g.n[1] + 4) * (NDIM == 3 ? g.n[2] + 4 : 1);
  adj_edge_faces_kernel<NDIM><<<blocks_for(box, 256), 256, 0, c->stream>>>(g, a->GE, As);
  prof_mark(c, MHD_AKCLASS_EDGE);
  c->launches++;
  if (split_now(c)) {  // the directions' Riemann transposes side by side (small grids)
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->aux[0], c->ev_fork, 0);
    adj_riemann_dir<NDIM, RS, RECON, 1>(c, Xs, Ps, As, dt, c->aux[0]);
    cudaEventRecord(c->ev_join[0], c->aux[0]);
    if constexpr (NDIM == 3) {
      cudaStreamWaitEvent(c->aux[1], c->ev_fork, 0);
      adj_riemann_dir<NDIM, RS, RECON, 2>(c, Xs, Ps, As, dt, c->aux[1]);
      cudaEventRecord(c->ev_join[1], c->aux[1]);
    }
    adj_riemann_dir<NDIM, RS, RECON, 0>(c, Xs, Ps, As, dt, c->stream);
    cudaStreamWaitEvent(c->stream, c->ev_join[0], 0);
    if constexpr (NDIM == 3) cudaStreamWaitEvent(c->stream, c->ev_join[1], 0);
  } else {
    adj_riemann_dir<NDIM, RS, RECON, 0>(c, Xs, Ps, As, dt, c->stream);
    adj_riemann_dir<NDIM, RS, RECON, 1>(c, Xs, Ps, As, dt, c->stream);
    if constexpr (NDIM == 3) adj_riemann_dir<NDIM, RS, RECON, 2>(c, Xs, Ps, As, dt, c->stream);
  }
  // the reconstruction transposes of every direction (they read only what
  // the Riemann transposes wrote), adding in direction order: PLM in one
  // launch, the five-cell reconstructions in two per direction
  if constexpr (RECON != RECON_PLM) {
    T35 T;
    for (int i = 0; i < 35; i++) T.q[i] = a->GE.q[i / 20][i % 20];
    adj_recon5_dir<NDIM, RECON, 0>(c, Ps, T);
    adj_recon5_dir<NDIM, RECON, 1>(c, Ps, T);
    if constexpr (NDIM == 3) adj_recon5_dir<NDIM, RECON, 2>(c, Ps, T);
    prof_mark(c, MHD_AKCLASS_RECON);
  } else {
    long long box = (long long)(g.n[0] + 4) * (g.n[1] + 4) * (NDIM == 3 ? g.n[2] + 4 : 1);
    adj_recon_all_kernel<NDIM><<<(int)((box + 127) / 128), 128, 0, c->stream>>>(
        g, plm_codes(a, 0), plm_codes(a, 1), plm_codes(a, NDIM == 3 ? 2 : 0), a->WbL[0], a->WbR[0], a->WbL[1],
        a->WbR[1], a->WbL[NDIM == 3 ? 2 : 0], a->WbR[NDIM == 3 ? 2 : 0], a->Pb);
    prof_mark(c, MHD_AKCLASS_RECON);
    c->launches++;
  }
  long long pad = (long long)g.ext[0] * g.ext[1] * g.ext[2];
  adj_c2p_kernel<NDIM><<<blocks_for(pad, 256), 256, 0, c->stream>>>(g, Xs, Ps, a->Pb, As);
  prof_mark(c, MHD_AKCLASS_C2P);
  c->launches++;
  adj_ghost_t(c, As, a->GE.q[0][0]);  // the scratch of the recon transposes, free again
  prof_mark(c, MHD_AKCLASS_GHOST);
  CK(cudaGetLastError());
  return MHD_OK;
}

template <int RECON>
int adj_stage_r(mhd_ctx* c, int s, const F8& Xs, const F8& Ps, const FaceIngr& ING, const F8& Aout, const F8& A0,
                const F8& As, double dt) {
  const int rs = sweep_rs(&c->cfg);
  if (c->g.ndim == 2) {
    if (rs == RS_HLLD_UCT) return adj_stage_t<2, RS_HLLD_UCT, RECON>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
    return rs == RS_HLLD ? adj_stage_t<2, RS_HLLD, RECON>(c, s, Xs, Ps, ING, Aout, A0, As, dt)
                         : adj_stage_t<2, RS_HLL, RECON>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
  }
  if (rs == RS_HLLD_UCT) return adj_stage_t<3, RS_HLLD_UCT, RECON>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
  return rs == RS_HLLD ? adj_stage_t<3, RS_HLLD, RECON>(c, s, Xs, Ps, ING, Aout, A0, As, dt)
                       : adj_stage_t<3, RS_HLL, RECON>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
}
int adj_stage(mhd_ctx* c, int s, const F8& Xs, const F8& Ps, const FaceIngr& ING, const F8& Aout, const F8& A0,
              const F8& As, double dt) {
  switch (c->cfg.recon) {
    case MHD_RECON_WENOZ: return adj_stage_r<RECON_WENOZ>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
    case MHD_RECON_PPM: return adj_stage_r<RECON_PPM>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
    default: return adj_stage_r<RECON_PLM>(c, s, Xs, Ps, ING, Aout, A0, As, dt);
  }
}

int seed(mhd_ctx* c, int functional) {
  AdjointState* a = c->adj;
  const Grid& g = c->g;
  ghost_fill(c, c->U[0]);
  CK(cudaMemsetAsync(a->A[3].q[0], 0, 8 * a->fe * sizeof(double), c->stream));
  double dV = g.dx[0] * g.dx[1] * (g.ndim == 3 ? g.dx[2] : 1.0);
  const int nb = blocks_for(g.ndim == 2 ? edge_work<2>(g) : edge_work<3>(g), 256);
  if (g.ndim == 2) adj_seed_kernel<2><<<nb, 256, 0, c->stream>>>(g, c->U[0], a->A[3], functional, a->T, dV, a->Jcell);
  else adj_seed_kernel<3><<<nb, 256, 0, c->stream>>>(g, c->U[0], a->A[3], functional, a->T, dV, a->Jcell);
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  adj_sum_kernel<<<1, 1024, 0, c->stream>>>(a->Jcell, ncell, 0.5 * dV, a->scal);
  c->launches += 2;
  adj_ghost_t(c, a->A[3], a->GE.q[0][0]);
  CK(cudaGetLastError());
  return MHD_OK;
}


// Device times of one adjoint run, by phase and (reverse phase) by kernel class.
struct Profile {
  double phase_ms[3];  // forward pass, block recomputes, reverse pass
  double class_ms[MHD_NAKCLASS];
  cudaEvent_t e0, e1;
};

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

int adjoint_run(mhd_ctx* c, int nsteps, const double* dts, int ckpt_every, int functional, int mem,
                const double* const* target, double* J_out, double* dts_out, Profile* prof) {
  if (!c || nsteps < 1 || ckpt_every < 1) return MHD_ERR_ARG;
  if (functional != MHD_FUNC_MAGNETIC_ENERGY && functional != MHD_FUNC_MISFIT) return MHD_ERR_ARG;
  if (functional == MHD_FUNC_MISFIT && (!target || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE))) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  const Grid& g = c->g;
  if (c->g.glm) return MHD_ERR_ARG;
  for (int d = 0; d < g.ndim; d++)
    if (g.n[d] < 2 * g.G + 1) return MHD_ERR_ARG;
  if (dts)
    for (int n = 0; n < nsteps; n++)
      if (!(dts[n] > 0.0) || !std::isfinite(dts[n])) return MHD_ERR_ARG;
  const int k = ckpt_every < nsteps ? ckpt_every : nsteps;
  int rc = ensure_state(c, nsteps, k);
  if (rc) return rc;
  AdjointState* a = c->adj;
  const int S = c->cfg.rk;
  if (functional == MHD_FUNC_MISFIT) {
    const int nq = g.ndim == 2 ? 6 : 5;
    for (int q = 0; q < nq; q++) {
      if (!target[q]) return MHD_ERR_ARG;
      int e[3];
      slot_extents(g, q < 5 ? q : 7, e);
      rc = copy_field(g, c->stream, a->T.q[q], target[q], nullptr, e, true);
      if (rc) return rc;
    }
  }

  const size_t base = (size_t)a->nck;  // the two block buffer sets follow the checkpoints
  const size_t set_states = (size_t)k * S + 1, set_ings = (size_t)k * S;
  auto X = [&](int set, int n0, int n, int st) {
    return state_at(a, base + set * set_states + (size_t)(n - n0) * S + st);
  };
  auto ING = [&](int set, int n0, int n, int st) {
    return ing_at(a, g.ndim, set * set_ings + (size_t)(n - n0) * S + st);
  };
  auto PRIM = [&](int set, int n0, int n, int st) { return prim_at(a, set * set_ings + (size_t)(n - n0) * S + st); };
  // block b's stage inputs and UCT ingredients into buffer set `set`,
  // recomputed from its checkpoint by context r on r's stream
  auto recompute = [&](mhd_ctx* r, int b, int set) -> int {
    const int n0 = b * k, n1 = (n0 + k < nsteps) ? n0 + k : nsteps;
    CK(cudaMemcpyAsync(X(set, n0, n0, 0).q[0], state_at(a, b).q[0], 8 * a->fe * sizeof(double),
                       cudaMemcpyDeviceToDevice, r->stream));
    for (int n = n0; n < n1; n++) {
      set_dt_only_kernel<<<1, 1, 0, r->stream>>>(r->sc, a->dts[n]);
      r->launches++;
      for (int st = 0; st < S; st++) {
        F8 out = st + 1 < S ? X(set, n0, n, st + 1) : X(set, n0, n + 1, 0);
        const F8 own = r->P;
        r->P = PRIM(set, n0, n, st);  // the stage's primitive pass writes them where the transposes read them
        run_stage_regs(r, st, X(set, n0, n, 0), X(set, n0, n, st), out, false);
        r->P = own;
        // keep the stage's UCT ingredients (the context's are contiguous, direction-major)
        const FaceIngr keep = ING(set, n0, n, st);
        CK(cudaMemcpyAsync(keep.a[0][0], r->ING.a[0][0], (size_t)a->ningr * g.ndim * a->fe * sizeof(double),
                           cudaMemcpyDeviceToDevice, r->stream));
      }
    }
    return MHD_OK;
  };
  // forward pass with checkpoints; dt frozen (given) or from the CFL condition
  if (prof) CK(cudaEventRecord(prof->e0, c->stream));
  // The recompute context rebuilds the last two blocks ahead of the reverse
  // pass, from their checkpoints: with the step sizes given, as soon as the
  // forward pass has saved the last block's checkpoint (beside the forward
  // pass's remaining steps); otherwise after the forward pass, which records
  // the steps.  It then stays two blocks ahead of the transposes.
  mhd_ctx* r = prof ? c : a->shadow;
  const int last = a->nck - 1;
  const long long l0 = r == c ? 0 : r->launches;
  auto start_recomputes = [&]() -> int {
    if (r != c) {
      CK(cudaEventRecord(a->ev_fwd, c->stream));
      CK(cudaStreamWaitEvent(r->stream, a->ev_fwd, 0));
    }
    for (int b = last; b >= 0 && b >= last - 1; b--) {
      int rc2 = recompute(r, b, b & 1);
      if (rc2) return rc2;
      CK(cudaEventRecord(a->ev_rec[b & 1], r->stream));
    }
    return MHD_OK;
  };
  bool started = false;
  if (dts) a->dts.assign(dts, dts + nsteps);
  for (int n = 0; n < nsteps; n++) {
    if (n % k == 0) {
      rc = copy_state(c, state_at(a, n / k), c->U[0]);
      if (rc) return rc;
      if (dts && !prof && n / k == last) {
        rc = start_recomputes();
        if (rc) return rc;
        started = true;
      }
    }
    if (dts) {
      set_dt_kernel<<<1, 1, 0, c->stream>>>(c->sc, dts[n]);
      c->launches++;
      run_step(c, false);
    } else {
      run_step(c, true);
    }
    record_dt_kernel<<<1, 1, 0, c->stream>>>(c->sc, a->scal + 1, n);
    c->launches++;
  }
  CK(cudaGetLastError());
  if (prof) {
    CK(cudaEventRecord(prof->e1, c->stream));
    CK(cudaEventSynchronize(prof->e1));
    prof->phase_ms[0] = elapsed(prof->e0, prof->e1);
  }
  a->dts.resize(nsteps);
  CK(cudaMemcpyAsync(a->dts.data(), a->scal + 1, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // the recompute passes below repeat the forward's counting: keep its scalars
  DevScalars fwd;
  CK(copy_sync(&fwd, c->sc, sizeof(fwd), cudaMemcpyDeviceToHost, c->stream));
  if (fwd.status) return fwd.status;
  rc = seed(c, functional);
  if (rc) return rc;

  // the stage transposes of block b, backwards, reading buffer set `set`
  F8 Ain = a->A[3];
  auto reverse = [&](int b, int set) -> int {
    const int n0 = b * k, n1 = (n0 + k < nsteps) ? n0 + k : nsteps;
    for (int n = n1 - 1; n >= n0; n--) {
      const double dt = a->dts[n];
      if (prof) {
        c->prof_on = true;
        c->prof_n = 0;
        prof_mark(c, -1);
      }
      for (int st = 0; st < S; st++) CK(cudaMemsetAsync(a->A[st].q[0], 0, 8 * a->fe * sizeof(double), c->stream));
      for (int st = S - 1; st >= 0; st--) {
        const F8& Aout = st == S - 1 ? Ain : a->A[st + 1];
        int rc2 = adj_stage(c, st, X(set, n0, n, st), PRIM(set, n0, n, st), ING(set, n0, n, st), Aout, a->A[0],
                            a->A[st], dt);
        if (rc2) {
          c->prof_on = false;
          return rc2;
        }
      }
      if (prof) {
        c->prof_on = false;
        CK(cudaStreamSynchronize(c->stream));
        for (int i = 1; i < c->prof_n; i++) {
          double ms = elapsed(c->prof_ev[i - 1], c->prof_ev[i]);
          prof->class_ms[c->prof_cls[i]] += ms;
          prof->phase_ms[2] += ms;
        }
      }
      // the cotangent of U^n becomes the incoming one of the step before
      F8 t = Ain;
      Ain = a->A[0];
      a->A[0] = t;
    }
    return MHD_OK;
  };
  if (prof) {  // in sequence on the context, each phase timed on its own
    for (int b = last; b >= 0; b--) {
      CK(cudaEventRecord(prof->e0, c->stream));
      rc = recompute(c, b, 0);
      if (rc) return rc;
      CK(cudaEventRecord(prof->e1, c->stream));
      CK(cudaEventSynchronize(prof->e1));
      prof->phase_ms[1] += elapsed(prof->e0, prof->e1);
      rc = reverse(b, 0);
      if (rc) return rc;
    }
  } else {  // the recompute context two blocks ahead of the transposes
    if (!started) {
      rc = start_recomputes();
      if (rc) return rc;
    }
    for (int b = last; b >= 0; b--) {
      const int set = b & 1;
      CK(cudaStreamWaitEvent(c->stream, a->ev_rec[set], 0));
      rc = reverse(b, set);
      if (rc) return rc;
      CK(cudaEventRecord(a->ev_rev[set], c->stream));
      if (b >= 2) {  // block b - 2 reuses the buffers the transposes of block b just read
        CK(cudaStreamWaitEvent(r->stream, a->ev_rev[set], 0));
        rc = recompute(r, b - 2, set);
        if (rc) return rc;
        CK(cudaEventRecord(a->ev_rec[set], r->stream));
      }
    }
    CK(cudaStreamSynchronize(r->stream));
    c->launches += r->launches - l0;
  }
  a->A[3] = Ain;  // holds dJ/dU^0
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&a->J, a->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  DevScalars h;
  CK(copy_sync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(copy_sync(c->sc, &fwd, sizeof(fwd), cudaMemcpyHostToDevice, c->stream));
  if (h.status) return h.status;
  a->has_grad = true;
  if (J_out) *J_out = a->J;
  if (dts_out) std::memcpy(dts_out, a->dts.data(), sizeof(double) * nsteps);
  return MHD_OK;
}

}  // namespace

namespace {
// The probe of both products, with NC cotangents per face.
template <int NC>
int probe_vjp(int rs, int n, double gamma, const double* in, const double* cot, double* dual, double* hand) {
  double *d_in = nullptr, *d_cot = nullptr, *d_dual = nullptr, *d_hand = nullptr;
  const size_t nin = (size_t)15 * n, ncot = (size_t)NC * n;
  cudaError_t e = cudaMalloc(&d_in, nin * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_cot, ncot * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_dual, nin * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_hand, nin * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, nin * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_cot, cot, ncot * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int nb = (n + 127) / 128;
    if (rs == RS_HLLD_UCT)
      riemann_vjp_probe_kernel<RS_HLLD_UCT, NC><<<nb, 128>>>(n, gamma, d_in, d_cot, d_dual, d_hand);
    else if (rs == RS_HLLD)
      riemann_vjp_probe_kernel<RS_HLLD, NC><<<nb, 128>>>(n, gamma, d_in, d_cot, d_dual, d_hand);
    else riemann_vjp_probe_kernel<RS_HLL, NC><<<nb, 128>>>(n, gamma, d_in, d_cot, d_dual, d_hand);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(dual, d_dual, nin * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hand, d_hand, nin * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_cot);
  cudaFree(d_dual);
  cudaFree(d_hand);
  return cuda_err(e);
}
}  // namespace

extern "C" {

int mhd_adjoint_run(mhd_ctx* c, int nsteps, const double* dts, int ckpt_every, int functional, int mem,
                    const double* const* target, double* J_out, double* dts_out) {
  return adjoint_run(c, nsteps, dts, ckpt_every, functional, mem, target, J_out, dts_out, nullptr);
}

int mhd_adjoint_profile(mhd_ctx* c, int nsteps, const double* dts, int ckpt_every, double* phase_ms,
                        double* class_ms) {
  if (!c || !phase_ms || !class_ms) return MHD_ERR_ARG;
  Profile p{};
  for (int i = 0; i < 128; i++) CK(cudaEventCreate(&c->prof_ev[i]));
  CK(cudaEventCreate(&p.e0));
  CK(cudaEventCreate(&p.e1));
  int rc = adjoint_run(c, nsteps, dts, ckpt_every, MHD_FUNC_MAGNETIC_ENERGY, MHD_MEM_HOST, nullptr, nullptr,
                       nullptr, &p);
  c->prof_on = false;
  for (int i = 0; i < 128; i++) cudaEventDestroy(c->prof_ev[i]);
  cudaEventDestroy(p.e0);
  cudaEventDestroy(p.e1);
  for (int i = 0; i < 3; i++) phase_ms[i] = p.phase_ms[i];
  for (int k = 0; k < MHD_NAKCLASS; k++) class_ms[k] = p.class_ms[k];
  return rc;
}


int mhd_probe_riemann_vjp(int riemann, int n, double gamma, const double* in, const double* cot, double* dual,
                          double* hand) {
  if (n < 1 || !in || !cot || !dual || !hand || !(gamma > 1.0)) return MHD_ERR_ARG;
  if (riemann != MHD_RIEMANN_HLL && riemann != MHD_RIEMANN_HLLD) return MHD_ERR_ARG;
  return probe_vjp<12>(riemann == MHD_RIEMANN_HLLD ? RS_HLLD : RS_HLL, n, gamma, in, cot, dual, hand);
}

int mhd_probe_stage_vjp(mhd_ctx* c, const double* const* U, double dt, const double* const* w,
                        double* const* grad) {
  if (!c || !U || !w || !grad || c->g.glm || !(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_ARG;
  for (int q = 0; q < 8; q++)
    if (!U[q] || !w[q] || !grad[q]) return MHD_ERR_ARG;
  const Grid& g = c->g;
  int rc = ensure_state(c, 1, 1);
  if (rc) return rc;
  AdjointState* a = c->adj;
  const F8 X = state_at(a, 0), Out = state_at(a, 1);
  for (int q = 0; q < 8; q++) {
    int e[3];
    slot_extents(g, q, e);
    rc = copy_field(g, c->stream, X.q[q], U[q], nullptr, e, true);
    if (rc) return rc;
  }
  // the forward stage on the context: X's ghost zones, the primitives in
  // c->P and the face ingredients in c->ING are what the transposes read
  set_dt_only_kernel<<<1, 1, 0, c->stream>>>(c->sc, dt);
  run_stage_regs(c, 0, X, X, Out, false);
  CK(cudaMemsetAsync(a->A[0].q[0], 0, 8 * a->fe * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a->A[3].q[0], 0, 8 * a->fe * sizeof(double), c->stream));
  for (int q = 0; q < 8; q++) {
    int e[3];
    slot_extents(g, q, e);
    rc = copy_field(g, c->stream, a->A[3].q[q], w[q], nullptr, e, true);
    if (rc) return rc;
  }
  rc = adj_stage(c, 0, X, c->P, c->ING, a->A[3], a->A[0], a->A[0], dt);
  if (rc) return rc;
  for (int q = 0; q < 8; q++) {
    int e[3];
    slot_extents(g, q, e);
    rc = copy_field(g, c->stream, a->A[0].q[q], nullptr, grad[q], e, false);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

int mhd_probe_ghost_vjp(mhd_ctx* c, const double* x, const double* abar, double* fx, double* xbar) {
  if (!c || !x || !abar || !fx || !xbar || c->g.glm) return MHD_ERR_ARG;
  const Grid& g = c->g;
  const size_t E = (size_t)g.ext[0] * g.ext[1] * g.ext[2], fe = c->field_elems;
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * (17 * fe)));
  F8 S, A;
  for (int q = 0; q < 8; q++) {
    S.q[q] = d + q * fe;
    A.q[q] = d + (8 + q) * fe;
  }
  double* H = d + 16 * fe;
  int rc = MHD_OK;
  for (int q = 0; q < 8 && rc == MHD_OK; q++)
    if (cudaMemcpyAsync(S.q[q], x + q * E, E * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(A.q[q], abar + q * E, E * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      rc = MHD_ERR_CUDA;
  if (rc == MHD_OK) {
    ghost_fill(c, S);
    adj_ghost_t(c, A, H);
    if (cudaGetLastError() != cudaSuccess) rc = MHD_ERR_CUDA;
  }
  for (int q = 0; q < 8 && rc == MHD_OK; q++)
    if (cudaMemcpyAsync(fx + q * E, S.q[q], E * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(xbar + q * E, A.q[q], E * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      rc = MHD_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess && rc == MHD_OK) rc = MHD_ERR_CUDA;
  cudaFree(d);
  return rc;
}

int mhd_probe_riemann_vjp_emf(int riemann, int emf, int n, double gamma, const double* in, const double* cot,
                              double* dual, double* hand) {
  if (n < 1 || !in || !cot || !dual || !hand || !(gamma > 1.0)) return MHD_ERR_ARG;
  if (riemann != MHD_RIEMANN_HLL && riemann != MHD_RIEMANN_HLLD) return MHD_ERR_ARG;
  if (emf != MHD_EMF_UCT_HLL && !(emf == MHD_EMF_UCT_HLLD && riemann == MHD_RIEMANN_HLLD)) return MHD_ERR_ARG;
  mhd_config cfg{};
  cfg.riemann = riemann;
  cfg.emf = emf;
  return probe_vjp<13>(sweep_rs(&cfg), n, gamma, in, cot, dual, hand);
}

int mhd_adjoint_grad_conserved(mhd_ctx* c, int mem, double* const* gU, double* const* gB) {
  if (!c || !gU || !gB || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  if (!c->adj || !c->adj->has_grad) return MHD_ERR_STATE;
  AdjointState* a = c->adj;
  for (int q = 0; q < 8; q++) {
    double* dst = q < 5 ? gU[q] : gB[q - 5];
    if (!dst) return MHD_ERR_ARG;
    int e[3];
    slot_extents(c->g, q, e);
    int rc = copy_field(c->g, c->stream, a->A[3].q[q], nullptr, dst, e, false);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

int mhd_adjoint_grad_prim(mhd_ctx* c, int mem, double* grad_rho, double* const* grad_v) {
  if (!c || !grad_rho || !grad_v || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  for (int q = 0; q < 3; q++)
    if (!grad_v[q]) return MHD_ERR_ARG;
  if (!c->adj || !c->adj->has_grad) return MHD_ERR_STATE;
  AdjointState* a = c->adj;
  const Grid& g = c->g;
  // primitives of U^0 (the first checkpoint)
  F8 X0 = state_at(a, (size_t)a->nck);
  int rc = copy_state(c, X0, state_at(a, 0));
  if (rc) return rc;
  ghost_fill(c, X0);
  prim(c, X0, false);
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  F8 out = a->Pb;
  if (g.ndim == 2) adj_to_prim_kernel<2><<<blocks_for(ncell, 256), 256, 0, c->stream>>>(g, a->A[3], c->P, out);
  else adj_to_prim_kernel<3><<<blocks_for(ncell, 256), 256, 0, c->stream>>>(g, a->A[3], c->P, out);
  c->launches++;
  CK(cudaGetLastError());
  double* dst[4] = {grad_rho, grad_v[0], grad_v[1], grad_v[2]};
  for (int q = 0; q < 4; q++) {
    int e[3];
    slot_extents(g, 0, e);
    rc = copy_field(g, c->stream, out.q[q], nullptr, dst[q], e, false);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

}  // extern "C"
