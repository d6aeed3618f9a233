// C-ABI of libmhd (declared in include/mhd.h): context management, state
// import/export and the orchestration of the RK stages of one time step.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "mhd.h"
#include "mhd_ctx.cuh"
#include "mhd_host.cuh"
#include "mhd_kernels.cuh"
#include "mhd_probe.h"

using namespace mhd;

namespace mhd {

void prof_mark(mhd_ctx* c, int cls) {
  if (!c->prof_on || c->prof_n >= 128) return;
  cudaEventRecord(c->prof_ev[c->prof_n], c->stream);
  c->prof_cls[c->prof_n] = cls;
  c->prof_n++;
}

// --- launch helpers ---
void ghost_fill(mhd_ctx* c, const F8& S) {
  const Grid& g = c->g;
  bool all_periodic = true;
  for (int d = 0; d < g.ndim; d++) all_periodic = all_periodic && g.periodic[d];
  if (all_periodic) {  // one pass over the ghost shell
    if (g.ndim == 2) ghost_shell_kernel<2><<<blocks_for(ghost_shell_work<2>(g), 256), 256, 0, c->stream>>>(g, S);
    else ghost_shell_kernel<3><<<blocks_for(ghost_shell_work<3>(g), 256), 256, 0, c->stream>>>(g, S);
    c->launches++;
    prof_mark(c, MHD_KCLASS_GHOST);
    return;
  }
  for (int pass = 0; pass < 2; pass++)
    for (int d = 0; d < g.ndim; d++) {
      if ((pass == 0) != (g.periodic[d] != 0)) continue;
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      long long rows = (long long)(g.hi(t1) - g.lo(t1) + 1) * (g.hi(t2) - g.lo(t2) + 1);
      long long work = rows * (2 * g.G + 1);
      if (g.periodic[d]) {
        ghost_periodic_kernel<<<blocks_for(work, 256), 256, 0, c->stream>>>(g, S, d);
        c->launches++;
        prof_mark(c, MHD_KCLASS_GHOST);
      } else {
        ghost_outflow_copy_kernel<<<blocks_for(work, 256), 256, 0, c->stream>>>(g, S, d);
        prof_mark(c, MHD_KCLASS_GHOST);
        ghost_outflow_normal_kernel<<<blocks_for(rows, 128), 128, 0, c->stream>>>(g, S, d);
        prof_mark(c, MHD_KCLASS_GHOST);
        c->launches += 2;
      }
    }
}

void prim(mhd_ctx* c, const F8& S, bool cfl, bool fast) {
  const Grid& g = c->g;
  long long work = (long long)(g.n[0] + 2 * g.G) * (g.n[1] + 2 * g.G) * (g.ndim == 3 ? g.n[2] + 2 * g.G : 1);
  int nb = blocks_for(work, 256);
  if (g.ndim == 2) {
    if (cfl) prim_kernel<2, true, false><<<nb, 256, 0, c->stream>>>(g, S, c->P, c->sc, c->lam);
    else if (fast) prim_kernel<2, false, true><<<nb, 256, 0, c->stream>>>(g, S, c->P, c->sc, c->lam);
    else prim_kernel<2, false, false><<<nb, 256, 0, c->stream>>>(g, S, c->P, c->sc, c->lam);
  } else {
    if (cfl) prim_kernel<3, true, false><<<nb, 256, 0, c->stream>>>(g, S, c->P, c->sc, c->lam);
    else if (fast) prim_kernel<3, false, true><<<nb, 256, 0, c->stream>>>(g, S, c->P, c->sc, c->lam);
    else prim_kernel<3, false, false><<<nb, 256, 0, c->stream>>>(g, S, c->P, c->sc, c->lam);
  }
  c->launches++;
  prof_mark(c, MHD_KCLASS_PRIM);
  if (cfl) {  // the IEEE decision among the candidates, and dt
    const long long cells = (long long)g.n[0] * g.n[1] * g.n[2];
    if (g.ndim == 2) cfl_exact_kernel<2><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, c->P, c->lam, c->sc);
    else cfl_exact_kernel<3><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, c->P, c->lam, c->sc);
    c->launches++;
    prof_mark(c, MHD_KCLASS_PRIM);
  }
}

bool split_now(const mhd_ctx* c) { return c->split && !c->prof_on; }

// One direction's sweep on stream st into the increment target T: mode 0
// writes -dt/dx dF, 1 adds it, 2 stores the raw difference dF (split sweeps).
template <int DIR, int NDIM, int RECON, int RS>
void sweep_one(mhd_ctx* c, const F8& S, cudaStream_t st, const L6& T, int mode) {
  const Grid& g = c->g;
  const long long threads = sweep_work<DIR, NDIM>(g, c->seglen);
  const int nb = (int)((threads + kSweepThreads - 1) / kSweepThreads);
  if constexpr (DIR == 0) {
    if (sweep_staged<DIR, NDIM>(g)) {
      sweep_kernel<DIR, NDIM, RECON, RS, true><<<nb, kSweepThreads, kXStageBytes, st>>>(
          g, c->P, S.q[5 + DIR], T, c->ING, c->sc, c->seglen, mode);
      c->launches++;
      prof_mark(c, MHD_KCLASS_SWEEP_X + DIR);
      return;
    }
  }
  sweep_kernel<DIR, NDIM, RECON, RS><<<nb, kSweepThreads, 0, st>>>(g, c->P, S.q[5 + DIR], T, c->ING, c->sc,
                                                                   c->seglen, mode);
  c->launches++;
  prof_mark(c, MHD_KCLASS_SWEEP_X + DIR);
}

template <int NDIM, int RECON, int RS>
void sweeps_t(mhd_ctx* c, const F8& S) {
  if (split_now(c)) {  // y (and z) beside x; the main stream waits for both
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->aux[0], c->ev_fork, 0);
    sweep_one<1, NDIM, RECON, RS>(c, S, c->aux[0], c->D[0], 2);
    cudaEventRecord(c->ev_join[0], c->aux[0]);
    if constexpr (NDIM == 3) {
      cudaStreamWaitEvent(c->aux[1], c->ev_fork, 0);
      sweep_one<2, NDIM, RECON, RS>(c, S, c->aux[1], c->D[1], 2);
      cudaEventRecord(c->ev_join[1], c->aux[1]);
    }
    sweep_one<0, NDIM, RECON, RS>(c, S, c->stream, c->L, 0);
    cudaStreamWaitEvent(c->stream, c->ev_join[0], 0);
    if constexpr (NDIM == 3) cudaStreamWaitEvent(c->stream, c->ev_join[1], 0);
    return;
  }
  sweep_one<0, NDIM, RECON, RS>(c, S, c->stream, c->L, 0);
  sweep_one<1, NDIM, RECON, RS>(c, S, c->stream, c->L, 1);
  if constexpr (NDIM == 3) sweep_one<2, NDIM, RECON, RS>(c, S, c->stream, c->L, 1);
}

// The staged x sweep uses more than the default 48 KB of dynamic shared
// memory; the attribute is set once per context, outside any graph capture.
template <int NDIM, int RECON, int RS>
cudaError_t allow_stage_t() {
  return cudaFuncSetAttribute(sweep_kernel<0, NDIM, RECON, RS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kXStageBytes);
}
// The sweeps' Riemann-solver template value of a configuration.
int sweep_rs(const mhd_config* cfg) {
  if (cfg->riemann != MHD_RIEMANN_HLLD) return RS_HLL;
  return cfg->emf == MHD_EMF_UCT_HLLD ? RS_HLLD_UCT : RS_HLLD;
}
template <int NDIM, int RECON>
cudaError_t allow_stage_r(int rs) {
  if (rs == RS_HLLD_UCT) return allow_stage_t<NDIM, RECON, RS_HLLD_UCT>();
  return rs == RS_HLLD ? allow_stage_t<NDIM, RECON, RS_HLLD>() : allow_stage_t<NDIM, RECON, RS_HLL>();
}
template <int NDIM>
cudaError_t allow_stage_n(int r, int rs) {
  if (r == MHD_RECON_PLM) return allow_stage_r<NDIM, RECON_PLM>(rs);
  if (r == MHD_RECON_WENOZ) return allow_stage_r<NDIM, RECON_WENOZ>(rs);
  return allow_stage_r<NDIM, RECON_PPM>(rs);
}
cudaError_t allow_stage(const mhd_config* cfg) {
  return cfg->ndim == 2 ? allow_stage_n<2>(cfg->recon, sweep_rs(cfg)) : allow_stage_n<3>(cfg->recon, sweep_rs(cfg));
}

template <int NDIM, int RECON>
void sweeps_r(mhd_ctx* c, const F8& S) {
  const int rs = sweep_rs(&c->cfg);
  if (rs == RS_HLLD_UCT) sweeps_t<NDIM, RECON, RS_HLLD_UCT>(c, S);
  else if (rs == RS_HLLD) sweeps_t<NDIM, RECON, RS_HLLD>(c, S);
  else sweeps_t<NDIM, RECON, RS_HLL>(c, S);
}
template <int NDIM>
void sweeps_n(mhd_ctx* c, const F8& S) {
  const int r = c->cfg.recon;
  if (r == MHD_RECON_PLM) sweeps_r<NDIM, RECON_PLM>(c, S);
  else if (r == MHD_RECON_WENOZ) sweeps_r<NDIM, RECON_WENOZ>(c, S);
  else sweeps_r<NDIM, RECON_PPM>(c, S);
}

void emf(mhd_ctx* c, const F8& S) {
  const Grid& g = c->g;
  long long work = (long long)(g.n[0] + 1) * (g.n[1] + 1) * (g.ndim == 3 ? g.n[2] + 1 : 1);
  int nb = blocks_for(work, 256);
  const bool hlld = c->cfg.emf == MHD_EMF_UCT_HLLD;
  if (g.ndim == 2) {
    if (hlld) emf_kernel<2, true><<<nb, 256, 0, c->stream>>>(g, S, c->ING, c->E);
    else emf_kernel<2, false><<<nb, 256, 0, c->stream>>>(g, S, c->ING, c->E);
  } else {
    if (hlld) emf_kernel<3, true><<<nb, 256, 0, c->stream>>>(g, S, c->ING, c->E);
    else emf_kernel<3, false><<<nb, 256, 0, c->stream>>>(g, S, c->ING, c->E);
  }
  c->launches++;
  prof_mark(c, MHD_KCLASS_EMF);
}

void ct_rk(mhd_ctx* c, const F8& U0, const F8& Us, const F8& Out, int mode) {
  const Grid& g = c->g;
  long long work = (long long)(g.n[0] + 1) * (g.n[1] + 1) * (g.ndim == 3 ? g.n[2] + 1 : 1);
  int nb = blocks_for(work, 256);
  if (split_now(c)) {
    if (g.ndim == 2) ct_rk_split_kernel<2><<<nb, 256, 0, c->stream>>>(g, U0, Us, Out, c->L, c->D[0], c->D[1], c->E, c->sc, mode);
    else ct_rk_split_kernel<3><<<nb, 256, 0, c->stream>>>(g, U0, Us, Out, c->L, c->D[0], c->D[1], c->E, c->sc, mode);
  } else if (g.ndim == 2) {
    ct_rk_kernel<2><<<nb, 256, 0, c->stream>>>(g, U0, Us, Out, c->L, c->E, c->sc, mode);
  } else {
    ct_rk_kernel<3><<<nb, 256, 0, c->stream>>>(g, U0, Us, Out, c->L, c->E, c->sc, mode);
  }
  c->launches++;
  prof_mark(c, MHD_KCLASS_CT_RK);
}

void sweeps(mhd_ctx* c, const F8& S) {
  if (c->g.ndim == 2) sweeps_n<2>(c, S);
  else sweeps_n<3>(c, S);
}

int stage_mode(int rk, int s) {
  return s == 0 ? COMB_FIRST : (rk == 2 ? COMB_RK2_FINAL : (s == 1 ? COMB_RK3_SECOND : COMB_RK3_FINAL));
}

void run_stage_regs(mhd_ctx* c, int s, const F8& U0, const F8& Us, const F8& Out, bool cfl) {
  if (fused_now(c)) {
    coop_stage(c, s, U0, Us, Out, cfl);
    return;
  }
  ghost_fill(c, Us);
  prim(c, Us, cfl, s > 0);
  sweeps(c, Us);
  emf(c, Us);
  ct_rk(c, U0, Us, Out, stage_mode(c->cfg.rk, s));
}

// --- divergence cleaning (GLM) helpers ---
void glm_ghost_fill(mhd_ctx* c, const F9& S) {
  const Grid& g = c->g;
  for (int pass = 0; pass < 2; pass++)
    for (int d = 0; d < g.ndim; d++) {
      if ((pass == 0) != (g.periodic[d] != 0)) continue;
      glm_ghost_kernel<<<blocks_for(ghost_layers_work(g, d), 256), 256, 0, c->stream>>>(g, S, d);
      c->launches++;
      prof_mark(c, MHD_KCLASS_GHOST);
    }
}

void glm_prim(mhd_ctx* c, const F9& S, bool cfl) {
  const Grid& g = c->g;
  int nb = blocks_for(g.ndim == 2 ? prim_work<2>(g) : prim_work<3>(g), 256);
  if (g.ndim == 2) {
    if (cfl) glm_prim_kernel<2, true><<<nb, 256, 0, c->stream>>>(g, S, c->GP, c->sc);
    else glm_prim_kernel<2, false><<<nb, 256, 0, c->stream>>>(g, S, c->GP, c->sc);
  } else {
    if (cfl) glm_prim_kernel<3, true><<<nb, 256, 0, c->stream>>>(g, S, c->GP, c->sc);
    else glm_prim_kernel<3, false><<<nb, 256, 0, c->stream>>>(g, S, c->GP, c->sc);
  }
  c->launches++;
  prof_mark(c, MHD_KCLASS_PRIM);
}

template <int DIR, int NDIM, int RECON, int RS>
void glm_sweep_one(mhd_ctx* c) {
  const long long threads = glm_sweep_work<DIR, NDIM>(c->g, c->seglen);
  glm_sweep_kernel<DIR, NDIM, RECON, RS><<<(int)((threads + 127) / 128), 128, 0, c->stream>>>(
      c->g, c->GP, c->GL, c->sc, c->seglen, DIR > 0 ? 1 : 0);
  c->launches++;
  prof_mark(c, MHD_KCLASS_SWEEP_X + DIR);
}
template <int NDIM, int RECON, int RS>
void glm_sweeps_t(mhd_ctx* c) {
  glm_sweep_one<0, NDIM, RECON, RS>(c);
  glm_sweep_one<1, NDIM, RECON, RS>(c);
  if constexpr (NDIM == 3) glm_sweep_one<2, NDIM, RECON, RS>(c);
}
template <int NDIM>
void glm_sweeps_n(mhd_ctx* c) {
  int r = c->cfg.recon, s = c->cfg.riemann;
  const bool hlld = s == MHD_RIEMANN_HLLD;
  if (r == MHD_RECON_PLM) hlld ? glm_sweeps_t<NDIM, RECON_PLM, RS_HLLD>(c) : glm_sweeps_t<NDIM, RECON_PLM, RS_HLL>(c);
  else if (r == MHD_RECON_WENOZ)
    hlld ? glm_sweeps_t<NDIM, RECON_WENOZ, RS_HLLD>(c) : glm_sweeps_t<NDIM, RECON_WENOZ, RS_HLL>(c);
  else hlld ? glm_sweeps_t<NDIM, RECON_PPM, RS_HLLD>(c) : glm_sweeps_t<NDIM, RECON_PPM, RS_HLL>(c);
}

void glm_run_stage(mhd_ctx* c, int s, bool cfl) {
  const Grid& g = c->g;
  const int rk = c->cfg.rk;
  const F9& Us = s == 0 ? c->GU[0] : (s == 1 ? c->GU[1] : c->GU[2]);
  const F9& Out = s == 0 ? c->GU[1] : ((rk == 2 || s == 2) ? c->GU[0] : c->GU[2]);
  glm_ghost_fill(c, Us);
  glm_prim(c, Us, cfl);
  if (g.ndim == 2) glm_sweeps_n<2>(c);
  else glm_sweeps_n<3>(c);
  double dh = g.dx[0];
  for (int d = 1; d < g.ndim; d++) dh = g.dx[d] < dh ? g.dx[d] : dh;
  const long long cells = (long long)g.n[0] * g.n[1] * g.n[2];
  const int last = s == rk - 1;
  if (g.ndim == 2)
    glm_combine_kernel<2><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, c->GU[0], Us, Out, c->GL, c->sc,
                                                                         stage_mode(rk, s), last, c->cfg.glm_alpha, dh);
  else
    glm_combine_kernel<3><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, c->GU[0], Us, Out, c->GL, c->sc,
                                                                         stage_mode(rk, s), last, c->cfg.glm_alpha, dh);
  c->launches++;
  prof_mark(c, MHD_KCLASS_CT_RK);
}

// One RK stage s of the step on the context's registers; cfl = compute this
// step's dt in the primitive pass.
void run_stage(mhd_ctx* c, int s, bool cfl) {
  if (c->g.glm) {
    glm_run_stage(c, s, cfl);
    return;
  }
  const int rk = c->cfg.rk;
  const F8& Us = s == 0 ? c->U[0] : (s == 1 ? c->U[1] : c->U[2]);
  const F8& Out = s == 0 ? c->U[1] : ((rk == 2 || s == 2) ? c->U[0] : c->U[2]);
  run_stage_regs(c, s, c->U[0], Us, Out, cfl);
}

void divb_check(mhd_ctx* c, double tol) {
  const Grid& g = c->g;
  const long long cells = (long long)g.n[0] * g.n[1] * g.n[2];
  if (g.ndim == 2) divb_kernel<2><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, c->U[0], c->sc);
  else divb_kernel<3><<<blocks_for(cells, 256), 256, 0, c->stream>>>(g, c->U[0], c->sc);
  divb_finish_kernel<<<1, 1, 0, c->stream>>>(c->sc, tol);
  c->launches += 2;
  prof_mark(c, MHD_KCLASS_OTHER);
}

void run_step(mhd_ctx* c, bool device_dt) {
  for (int s = 0; s < c->cfg.rk; s++) run_stage(c, s, device_dt && s == 0);
  if (c->divb_tol > 0.0) divb_check(c, c->divb_tol);
}

}  // namespace mhd

// Default sweep segment length: each segment repeats one face and one
// reconstruction at its end, so long segments waste less, while short ones
// give more threads.  Take the longest (2..256) that still leaves about eight
// waves of 384-thread SM loads in the sweep with the fewest faces.
static long long faces_per_thread_target(const Grid& g) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  long long fewest = LLONG_MAX;
  for (int d = 0; d < g.ndim; d++) {
    long long faces = g.n[d] + 1;
    for (int t = 0; t < g.ndim; t++)
      if (t != d) faces *= g.n[t] + 2;
    fewest = faces < fewest ? faces : fewest;
  }
  return fewest / (8LL * sms * 384);
}
static int default_seglen(const Grid& g) {
  const long long per_thread = faces_per_thread_target(g);
  return (int)(per_thread < 2 ? 2 : (per_thread > 256 ? 256 : per_thread));
}
// Sweeps side by side when even segments of 2 faces leave fewer than about
// eight waves of threads in one sweep (CT only).
static bool split_sweeps(const Grid& g) { return !g.glm && g.ndim > 1 && faces_per_thread_target(g) < 2; }

extern "C" {

const char* mhd_strerror(int code) {
  switch (code) {
    case MHD_OK: return "ok";
    case MHD_ERR_ARG: return "invalid argument";
    case MHD_ERR_CUDA: return "CUDA runtime error";
    case MHD_ERR_OOM: return "device out of memory";
    case MHD_ERR_UNPHYSICAL: return "non-positive density or pressure";
    case MHD_ERR_TIMEOUT: return "device-side wait timed out";
    case MHD_ERR_STATE: return "no state set";
    case MHD_ERR_TOO_LARGE: return "grid exceeds the fixed scratch of mhd_step_noalloc";
    case MHD_ERR_DIVB: return "discrete div B above the monitor's tolerance";
    case MHD_ERR_GUARD: return "a guard word beside a device array was overwritten";
    default: return "unknown error";
  }
}

int mhd_create(const mhd_config* cfg, mhd_ctx** out) {
  if (!out) return MHD_ERR_ARG;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  Grid g = make_grid(cfg);
  long long elems = (long long)g.ext[0] * g.ext[1] * g.ext[2];
  if (elems > (long long)INT_MAX - 1) return MHD_ERR_ARG;
  mhd_ctx* c = new (std::nothrow) mhd_ctx();
  if (!c) return MHD_ERR_OOM;
  c->cfg = *cfg;
  c->g = g;
  c->seglen = default_seglen(g);
  c->split = split_sweeps(g);
  c->field_used = elems;
  c->field_elems = (size_t)guard_stride(elems);
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
    c->own_stream = false;
  } else {
    // a blocking stream: ordered with the legacy default stream, and capturable
    if (cudaStreamCreate(&c->stream) != cudaSuccess) { delete c; return MHD_ERR_CUDA; }
    c->own_stream = true;
  }
  // CT: 3 registers of 8, primitives 8, increment 6, ingredients 15 (18 with
  // the UCT-HLLD weights), edges 3; GLM: 3 registers of 9, primitives 9,
  // increment 9 (+ the CFL rates; + the raw flux differences of the split y
  // and z sweeps)
  const int ningr = cfg->emf == MHD_EMF_UCT_HLLD ? 6 : 5;
  const int nfields = (g.glm ? 3 * 9 + 9 + 9 : 3 * 8 + 8 + 6 + 3 * ningr + 3) + 1 + (c->split ? 6 * (g.ndim - 1) : 0);
  c->pool_fields = nfields;
  size_t bytes = (size_t)guard_block_words(nfields, (long long)c->field_elems) * sizeof(double);
  if (cudaMalloc(&c->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return MHD_ERR_OOM;
  }
  cudaMemsetAsync(c->pool, 0, bytes, c->stream);
  guard_fill(c->stream, c->pool, nfields, (long long)c->field_elems, elems);
  double* p = c->pool + kGuardWords;
  auto next = [&]() { double* r = p; p += c->field_elems; return r; };
  if (g.glm) {
    c->reg_fields = 9;
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 9; q++) {
        c->GU[r].q[q] = next();
        if (q < 8) c->U[r].q[q] = c->GU[r].q[q];
      }
    for (int q = 0; q < 9; q++) c->GP.q[q] = next();
    for (int q = 0; q < 9; q++) c->GL.q[q] = next();
  } else {
    c->reg_fields = 8;
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 8; q++) c->U[r].q[q] = next();
    for (int q = 0; q < 8; q++) c->P.q[q] = next();
    for (int q = 0; q < 6; q++) c->L.q[q] = next();
    for (int d = 0; d < 3; d++)
      for (int q = 0; q < ningr; q++) c->ING.a[d][q] = next();
    for (int d = 0; d < 3; d++) c->E.e[d] = next();
  }
  c->lam = next();
  if (c->split)
    for (int d = 0; d < g.ndim - 1; d++)
      for (int q = 0; q < 6; q++) c->D[d].q[q] = next();
  if (cudaMalloc(&c->sc, sizeof(DevScalars)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->pool);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return MHD_ERR_OOM;
  }
  DevScalars h;
  reset_scalars_host(&h);
  cudaMemcpyAsync(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    mhd_destroy(c);
    return MHD_ERR_CUDA;
  }
  if (allow_stage(cfg) != cudaSuccess) {
    mhd_destroy(c);
    return MHD_ERR_CUDA;
  }
  if (c->split) {
    bool ok = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int d = 0; d < 2 && ok; d++)
      ok = cudaStreamCreateWithFlags(&c->aux[d], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->ev_join[d], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      mhd_destroy(c);
      return MHD_ERR_CUDA;
    }
  }
  rc = coop_init(c);
  if (rc) {
    mhd_destroy(c);
    return rc;
  }
  c->launches_per_step = -1;
  *out = c;
  return MHD_OK;
}

int mhd_destroy(mhd_ctx* c) {
  if (!c) return MHD_OK;
  cudaStreamSynchronize(c->stream);
  if (c->graph_ready) cudaGraphExecDestroy(c->graph);
  adjoint_free(c);
  coop_free(c);
  cudaFree(c->pool);
  cudaFree(c->sc);
  for (int d = 0; d < 2; d++) {
    if (c->aux[d]) cudaStreamDestroy(c->aux[d]);
    if (c->ev_join[d]) cudaEventDestroy(c->ev_join[d]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return MHD_OK;
}

static int set_common_faces(mhd_ctx* c, const double* const* B) {
  for (int q = 5; q < 8; q++) {
    int e[3];
    slot_extents(c->g, q, e);
    int rc = copy_field(c->g, c->stream, c->U[0].q[q], B[q - 5], nullptr, e, true);
    if (rc) return rc;
  }
  return MHD_OK;
}

static int reset_time(mhd_ctx* c) {
  CK(cudaMemcpyAsync(c->sc, reset_scalars_source(), sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream));
  return MHD_OK;
}

int mhd_set_conserved(mhd_ctx* c, int mem, const double* const* U, const double* const* B) {
  if (!c || !U || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  for (int q = 0; q < 5; q++)
    if (!U[q]) return MHD_ERR_ARG;
  for (int q = 0; q < 3; q++)
    if (!B[q]) return MHD_ERR_ARG;
  for (int q = 0; q < 5; q++) {
    int e[3];
    slot_extents(c->g, q, e);
    int rc = copy_field(c->g, c->stream, c->U[0].q[q], U[q], nullptr, e, true);
    if (rc) return rc;
  }
  int rc = set_common_faces(c, B);
  if (rc) return rc;
  if (c->g.glm) CK(cudaMemsetAsync(c->GU[0].q[8], 0, c->field_used * sizeof(double), c->stream));
  c->has_state = true;
  return reset_time(c);
}

int mhd_set_prim(mhd_ctx* c, int mem, const double* rho, const double* const* v, const double* p,
                 const double* const* B) {
  if (!c || !rho || !v || !p || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  const double* cells[5] = {rho, v[0], v[1], v[2], p};
  for (int q = 0; q < 5; q++) {
    if (!cells[q]) return MHD_ERR_ARG;
    int e[3];
    slot_extents(c->g, q, e);
    int rc = copy_field(c->g, c->stream, c->U[0].q[q], cells[q], nullptr, e, true);
    if (rc) return rc;
  }
  int rc = set_common_faces(c, B);
  if (rc) return rc;
  long long work = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
  if (c->g.glm) {
    CK(cudaMemsetAsync(c->GU[0].q[8], 0, c->field_used * sizeof(double), c->stream));
    if (c->g.ndim == 2) glm_prim_to_cons_kernel<2><<<blocks_for(work, 256), 256, 0, c->stream>>>(c->g, c->GU[0]);
    else glm_prim_to_cons_kernel<3><<<blocks_for(work, 256), 256, 0, c->stream>>>(c->g, c->GU[0]);
  } else if (c->g.ndim == 2) {
    prim_to_cons_kernel<2><<<blocks_for(work, 256), 256, 0, c->stream>>>(c->g, c->U[0]);
  } else {
    prim_to_cons_kernel<3><<<blocks_for(work, 256), 256, 0, c->stream>>>(c->g, c->U[0]);
  }
  c->launches++;
  CK(cudaGetLastError());
  c->has_state = true;
  return reset_time(c);
}

int mhd_status(mhd_ctx* c, long long* bad_cell) {
  if (!c) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  DevScalars h;
  CK(copy_sync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  if (bad_cell) *bad_cell = h.status && h.status != MHD_ERR_TIMEOUT ? h.bad_cell : -1;
  if (h.status) {
    int st = h.status;
    h.status = 0;
    h.bad_cell = LLONG_MAX;
    CK(copy_sync(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    if (st == MHD_ERR_TIMEOUT) {
      int rc = coop_clear(c);
      if (rc) return rc;
    }
    return st;
  }
  return MHD_OK;
}

int mhd_get_conserved(mhd_ctx* c, int mem, double* const* U, double* const* B) {
  if (!c || !U || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  if (!c->g.glm) ghost_fill(c, c->U[0]);  // the duplicate last face of periodic axes
  for (int q = 0; q < 8; q++) {
    double* dst = q < 5 ? U[q] : B[q - 5];
    if (!dst) return MHD_ERR_ARG;
    int e[3];
    slot_extents(c->g, q, e);
    int rc = copy_field(c->g, c->stream, c->U[0].q[q], nullptr, dst, e, false);
    if (rc) return rc;
  }
  CK(cudaGetLastError());
  return mhd_status(c, nullptr);
}

int mhd_set_boundaries(mhd_ctx* c, const int bc[6]) {
  if (!c || !bc) return MHD_ERR_ARG;
  mhd_config t = c->cfg;
  for (int s = 0; s < 6; s++) t.bc[s] = bc[s];
  int rc = validate(&t);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->cfg = t;
  for (int d = 0; d < c->g.ndim; d++) c->g.periodic[d] = t.bc[2 * d] == MHD_BC_PERIODIC;
  if (c->graph_ready) {
    cudaGraphExecDestroy(c->graph);
    c->graph_ready = false;
  }
  return MHD_OK;
}

int mhd_cfl_dt(mhd_ctx* c, double* dt_out) {
  if (!c || !dt_out) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  // evaluate the rate without touching the accumulated time
  DevScalars before;
  CK(cudaStreamSynchronize(c->stream));
  CK(copy_sync(&before, c->sc, sizeof(before), cudaMemcpyDeviceToHost, c->stream));
  if (c->g.glm) {
    glm_ghost_fill(c, c->GU[0]);
    glm_prim(c, c->GU[0], true);
  } else {
    ghost_fill(c, c->U[0]);
    prim(c, c->U[0], true);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  DevScalars after;
  CK(copy_sync(&after, c->sc, sizeof(after), cudaMemcpyDeviceToHost, c->stream));
  *dt_out = after.dt;
  after.dt = before.dt;
  after.time = before.time;
  CK(copy_sync(c->sc, &after, sizeof(after), cudaMemcpyHostToDevice, c->stream));
  return after.status ? after.status : MHD_OK;
}

int mhd_step(mhd_ctx* c, double dt) {
  if (!c || !(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  set_dt_kernel<<<1, 1, 0, c->stream>>>(c->sc, dt);
  c->launches++;
  prof_mark(c, MHD_KCLASS_OTHER);
  run_step(c, false);
  CK(cudaGetLastError());
  return MHD_OK;
}

int mhd_advance(mhd_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  if (nsteps == 0) return MHD_OK;
  if (!c->graph_ready) {
    long long before = c->launches;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    run_step(c, true);
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (e != cudaSuccess) return cuda_err(e);
    e = cudaGraphInstantiate(&c->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_err(e);
    c->graph_ready = true;
    c->launches_per_step = (int)(c->launches - before);
    c->launches = before;
  }
  for (int s = 0; s < nsteps; s++) {
    CK(cudaGraphLaunch(c->graph, c->stream));
    c->launches += c->launches_per_step;
  }
  return MHD_OK;
}

}  // extern "C"

// Set the simulation time (a resumed run).
static __global__ void set_time_kernel(DevScalars* sc, double t) { sc->time = t; }

extern "C" {

int mhd_set_divb_check(mhd_ctx* c, double tol) {
  if (!c || !(tol >= 0.0) || !std::isfinite(tol) || c->g.glm) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->divb_tol = tol;
  if (c->graph_ready) {  // the captured step changes
    cudaGraphExecDestroy(c->graph);
    c->graph_ready = false;
  }
  return MHD_OK;
}

int mhd_divb(mhd_ctx* c, double* rel_out) {
  if (!c || !rel_out || c->g.glm) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  ghost_fill(c, c->U[0]);
  divb_check(c, 0.0);
  CK(cudaGetLastError());
  DevScalars h;
  CK(copy_sync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  *rel_out = h.divb_rel;
  return MHD_OK;
}

}  // extern "C"

extern "C" {

int mhd_set_time(mhd_ctx* c, double t) {
  if (!c || !(t == t)) return MHD_ERR_ARG;
  set_time_kernel<<<1, 1, 0, c->stream>>>(c->sc, t);
  CK(cudaGetLastError());
  return MHD_OK;
}

int mhd_get_time(mhd_ctx* c, double* t_out) {
  if (!c || !t_out) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  DevScalars h;
  CK(copy_sync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  *t_out = h.time;
  return MHD_OK;
}

int mhd_last_dt(mhd_ctx* c, double* dt_out) {
  if (!c || !dt_out) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  DevScalars h;
  CK(copy_sync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  *dt_out = h.dt;
  return MHD_OK;
}

long long mhd_launch_count(const mhd_ctx* c) { return c ? c->launches : -1; }

int mhd_set_psi(mhd_ctx* c, int mem, const double* psi) {
  if (!c || !psi || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE) || !c->g.glm) return MHD_ERR_ARG;
  int e[3];
  slot_extents(c->g, 0, e);
  return copy_field(c->g, c->stream, c->GU[0].q[8], psi, nullptr, e, true);
}

int mhd_get_psi(mhd_ctx* c, int mem, double* psi) {
  if (!c || !psi || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE) || !c->g.glm) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  int e[3];
  slot_extents(c->g, 0, e);
  int rc = copy_field(c->g, c->stream, c->GU[0].q[8], nullptr, psi, e, false);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

int mhd_set_seglen(mhd_ctx* c, int seglen) {
  if (!c || seglen < 1) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->seglen = seglen;
  if (c->graph_ready) {  // the captured sweeps carry the old segment length
    cudaGraphExecDestroy(c->graph);
    c->graph_ready = false;
  }
  return MHD_OK;
}

int mhd_get_seglen(const mhd_ctx* c, int* seglen_out) {
  if (!c || !seglen_out) return MHD_ERR_ARG;
  *seglen_out = c->seglen;
  return MHD_OK;
}

int mhd_autotune(mhd_ctx* c, int* seglen_out) {
  if (!c) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  CK(cudaStreamSynchronize(c->stream));
  DevScalars sc_h;
  CK(copy_sync(&sc_h, c->sc, sizeof(sc_h), cudaMemcpyDeviceToHost, c->stream));
  const size_t bytes = (size_t)c->reg_fields * c->field_elems * sizeof(double);  // U[0]'s fields are contiguous
  double* backup = nullptr;
  CK(cudaMalloc(&backup, bytes));
  CK(cudaMemcpyAsync(backup, c->U[0].q[0], bytes, cudaMemcpyDeviceToDevice, c->stream));
  int longest = 0;  // faces per pencil along the longest axis
  for (int d = 0; d < c->g.ndim; d++) longest = c->g.n[d] + 1 > longest ? c->g.n[d] + 1 : longest;
  // powers of two and lengths between them, plus the lengths that split the
  // longest pencil into 4..12 equal segments: the segment count sets how many
  // waves of blocks a sweep takes and how short its last segment is
  int cand[32], ncand = 0;
  for (int s : {2, 4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64, 96, 128}) cand[ncand++] = s;
  for (int k = 4; k <= 12; k++) cand[ncand++] = (longest + k - 1) / k;
  std::sort(cand, cand + ncand);
  ncand = (int)(std::unique(cand, cand + ncand) - cand);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int pick = c->seglen, rc = MHD_OK;
  bool pick_fused = c->fused;
  // both launch forms where the fused stage is available (2D CT grids)
  const int nforms = c->bar ? 2 : 1;
  for (int f = 0; f < nforms && rc == MHD_OK; f++) {
    if (c->bar) c->fused = f == 1;
    for (int i = 0; i < ncand && rc == MHD_OK; i++) {
      if (cand[i] > 2 * longest) break;
      c->seglen = cand[i];
      run_step(c, true);  // warm
      cudaEventRecord(e0, c->stream);
      run_step(c, true);
      run_step(c, true);
      cudaEventRecord(e1, c->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { rc = cuda_err(e); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; pick = cand[i]; pick_fused = c->fused; }
      cudaMemcpyAsync(c->U[0].q[0], backup, bytes, cudaMemcpyDeviceToDevice, c->stream);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(c->stream);
  cudaFree(backup);
  CK(copy_sync(c->sc, &sc_h, sizeof(sc_h), cudaMemcpyHostToDevice, c->stream));
  c->seglen = pick;
  c->fused = pick_fused;
  if (c->graph_ready) {
    cudaGraphExecDestroy(c->graph);
    c->graph_ready = false;
  }
  if (seglen_out) *seglen_out = pick;
  return rc;
}

int mhd_counters(mhd_ctx* c, long long* recon_fallbacks, long long* pressure_floors) {
  if (!c) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  DevScalars h;
  CK(copy_sync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  if (recon_fallbacks) *recon_fallbacks = (long long)h.fallbacks;
  if (pressure_floors) *pressure_floors = (long long)h.floors;
  return MHD_OK;
}

int mhd_profile_steps(mhd_ctx* c, int nsteps, double* ms_out, int* launches_out) {
  if (!c || !ms_out || nsteps < 0) return MHD_ERR_ARG;
  if (!c->has_state) return MHD_ERR_STATE;
  for (int k = 0; k < MHD_NKCLASS; k++) {
    ms_out[k] = 0.0;
    if (launches_out) launches_out[k] = 0;
  }
  for (int i = 0; i < 128; i++) CK(cudaEventCreate(&c->prof_ev[i]));
  int rc = MHD_OK;
  for (int s = 0; s < nsteps && rc == MHD_OK; s++) {
    c->prof_on = true;
    c->prof_n = 0;
    prof_mark(c, -1);
    run_step(c, true);
    c->prof_on = false;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { rc = cuda_err(e); break; }
    for (int i = 1; i < c->prof_n; i++) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->prof_ev[i - 1], c->prof_ev[i]);
      ms_out[c->prof_cls[i]] += ms;
      if (launches_out) launches_out[c->prof_cls[i]]++;
    }
  }
  for (int i = 0; i < 128; i++) cudaEventDestroy(c->prof_ev[i]);
  return rc;
}

}  // extern "C"

namespace {
// Eight independent chains of dependent FP64 instructions per thread, in one of
// the instruction forms of MHD_FP64_FORM_*; the result is stored so the chains
// are live.  The operands a, b come from device memory (registers), except in
// the constant-operand form, where they are literals.
template <int FORM>
__global__ void fp64_probe_kernel(double* out, const double* __restrict__ ab, int iters) {
  const double a = ab[0], b = ab[1];
  const double b2 = ab[2], b3 = ab[3];
  double c[8];
#pragma unroll
  for (int q = 0; q < 8; q++) c[q] = threadIdx.x * 1e-3 + q;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (FORM == MHD_FP64_FORM_DMUL) c[q] = c[q] * a;
      else if (FORM == MHD_FP64_FORM_DADD) c[q] = c[q] + b;
      else if (FORM == MHD_FP64_FORM_DFMA_DISTINCT) c[q] = fma(c[q], a, (q & 1) ? b3 : ((q & 2) ? b2 : b));
      else if (FORM == MHD_FP64_FORM_DFMA_CONST) c[q] = fma(c[q], 0.999999, 1e-7);  // literal operands
      else c[q] = fma(c[q], a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
}
template <int FORM>
float time_probe(double* buf, const double* ab, int blocks, int threads, int iters) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 5; rep++) {
    cudaEventRecord(e0, 0);
    fp64_probe_kernel<FORM><<<blocks, threads>>>(buf, ab, iters);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}
// Rates of the forms in GFLOP/s equivalents (2 flops per FP64 instruction).
int probe_forms(double* rates, int nforms) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8, iters = 4096;
  double *buf = nullptr, *ab = nullptr;
  CK(cudaMalloc(&buf, sizeof(double) * threads * blocks));
  if (cudaMalloc(&ab, 4 * sizeof(double)) != cudaSuccess) {
    cudaFree(buf);
    return MHD_ERR_OOM;
  }
  const double h[4] = {0.999999, 1e-7, 2e-7, 3e-7};
  cudaError_t e = cudaMemcpy(ab, h, sizeof(h), cudaMemcpyHostToDevice);
  const double inst = 8.0 * iters * (double)threads * blocks;
  float ms[MHD_FP64_NFORMS] = {};
  if (e == cudaSuccess) {
    ms[0] = time_probe<0>(buf, ab, blocks, threads, iters);
    if (nforms > 1) {
      ms[1] = time_probe<1>(buf, ab, blocks, threads, iters);
      ms[2] = time_probe<2>(buf, ab, blocks, threads, iters);
      ms[3] = time_probe<3>(buf, ab, blocks, threads, iters);
      ms[4] = time_probe<4>(buf, ab, blocks, threads, iters);
    }
    e = cudaGetLastError();
  }
  cudaFree(buf);
  cudaFree(ab);
  if (e != cudaSuccess) return cuda_err(e);
  for (int f = 0; f < nforms; f++) rates[f] = 2.0 * inst / (ms[f] * 1e-3) / 1e9;
  return MHD_OK;
}
}  // namespace

// Both CFL rates of n primitive states (rho, vx, vy, vz, bx, by, bz, p each).
template <int NDIM>
static __global__ void cfl_rate_probe_kernel(mhd::Grid g, int n, const double* __restrict__ prim, double* near_out,
                                             double* ieee_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double* w = prim + (size_t)8 * t;
  mhd::Prim8 V;
  V.rho = w[0]; V.vx = w[1]; V.vy = w[2]; V.vz = w[3];
  V.bx = w[4]; V.by = w[5]; V.bz = w[6]; V.p = w[7];
  near_out[t] = mhd::cfl_rate_near_ieee<NDIM>(g, V);
  ieee_out[t] = mhd::cfl_rate_ieee<NDIM>(g, V);
}

// The sweeps' Riemann solver at n faces: in[15] = left (rho, u, v, w, b1, b2,
// p), right (same), b_n; out F[7] and the UCT ingredients ing[6].
template <int RS>
static __global__ void riemann_probe_kernel(int n, double gamma, const double* __restrict__ in,
                                            double* __restrict__ F_out, double* __restrict__ ing_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double* x = in + (size_t)15 * t;
  mhd::W7 L = {x[0], x[1], x[2], x[3], x[4], x[5], x[6]};
  mhd::W7 R = {x[7], x[8], x[9], x[10], x[11], x[12], x[13]};
  mhd::Flux7 F;
  mhd::Ingr ing;
  ing.dr = 0.0;
  const double igm1 = 1.0 / (gamma - 1.0);
  if (RS == mhd::RS_HLL) mhd::riemann_hll(L, R, x[14], gamma, igm1, F, ing);
  else mhd::riemann_hlld<double, RS == mhd::RS_HLLD_UCT>(L, R, x[14], gamma, igm1, F, ing);
  if (RS != mhd::RS_HLLD_UCT) ing.dr = ing.dd;
  for (int q = 0; q < 7; q++) F_out[(size_t)7 * t + q] = F.f[q];
  const double v6[6] = {ing.ap, ing.am, ing.dd, ing.uL, ing.uR, ing.dr};
  for (int q = 0; q < 6; q++) ing_out[(size_t)6 * t + q] = v6[q];
}

extern "C" {

int mhd_probe_riemann(int riemann, int emf, int n, double gamma, const double* in, double* F, double* ing) {
  if (n < 1 || !in || !F || !ing || !(gamma > 1.0)) return MHD_ERR_ARG;
  if (riemann != MHD_RIEMANN_HLL && riemann != MHD_RIEMANN_HLLD) return MHD_ERR_ARG;
  if (emf != MHD_EMF_UCT_HLL && emf != MHD_EMF_UCT_HLLD) return MHD_ERR_ARG;
  if (emf == MHD_EMF_UCT_HLLD && riemann != MHD_RIEMANN_HLLD) return MHD_ERR_ARG;
  double *d_in = nullptr, *d_F = nullptr, *d_ing = nullptr;
  cudaError_t e = cudaMalloc(&d_in, sizeof(double) * 15 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_F, sizeof(double) * 7 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_ing, sizeof(double) * 6 * (size_t)n);
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, sizeof(double) * 15 * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int nb = (n + 127) / 128;
    if (riemann == MHD_RIEMANN_HLL) riemann_probe_kernel<mhd::RS_HLL><<<nb, 128>>>(n, gamma, d_in, d_F, d_ing);
    else if (emf == MHD_EMF_UCT_HLLD)
      riemann_probe_kernel<mhd::RS_HLLD_UCT><<<nb, 128>>>(n, gamma, d_in, d_F, d_ing);
    else riemann_probe_kernel<mhd::RS_HLLD><<<nb, 128>>>(n, gamma, d_in, d_F, d_ing);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(F, d_F, sizeof(double) * 7 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ing, d_ing, sizeof(double) * 6 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_F);
  cudaFree(d_ing);
  return cuda_err(e);
}

int mhd_probe_fp64(double* gflops_out) {
  if (!gflops_out) return MHD_ERR_ARG;
  return probe_forms(gflops_out, 1);
}

int mhd_probe_fp64_forms(double* rates) {
  if (!rates) return MHD_ERR_ARG;
  return probe_forms(rates, MHD_FP64_NFORMS);
}

int mhd_probe_cfl_rate(int ndim, double gamma, const double* dx, int n, const double* prim, double* near_out,
                       double* ieee_out) {
  if ((ndim != 2 && ndim != 3) || !(gamma > 1.0) || !dx || n < 1 || !prim || !near_out || !ieee_out)
    return MHD_ERR_ARG;
  mhd::Grid g{};
  g.ndim = ndim;
  g.gamma = gamma;
  for (int d = 0; d < 3; d++) {
    if (!(dx[d] > 0.0)) return MHD_ERR_ARG;
    g.dx[d] = dx[d];
    g.idx[d] = 1.0 / dx[d];
  }
  double *d_prim = nullptr, *d_near = nullptr, *d_ieee = nullptr;
  cudaError_t e = cudaMalloc(&d_prim, sizeof(double) * 8 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_near, sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_ieee, sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = cudaMemcpy(d_prim, prim, sizeof(double) * 8 * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int nb = (n + 255) / 256;
    if (ndim == 3) cfl_rate_probe_kernel<3><<<nb, 256>>>(g, n, d_prim, d_near, d_ieee);
    else cfl_rate_probe_kernel<2><<<nb, 256>>>(g, n, d_prim, d_near, d_ieee);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(near_out, d_near, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ieee_out, d_ieee, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d_prim);
  cudaFree(d_near);
  cudaFree(d_ieee);
  return cuda_err(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single step.  All scratch lives in one file-scope device
// array; host code reaches it only through the address cudaGetSymbolAddress
// returns (the array's name is a host-side stand-in in host code).
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocDoubles = MHD_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kNoAllocFields = 3 * 8 + 8 + 6 + 15 + 3 + 1;  // mhd_create's carve-up (CT, UCT-HLL); +3 for UCT-HLLD
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};  // device address of the array, per device

// Once per device, with that device current: look up the array's device address.
int noalloc_scratch(double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MHD_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    double* p = nullptr;
    CK(cudaGetSymbolAddress((void**)&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_step_noalloc(const mhd_config* cfg, double* const* U, double* const* B, double dt) {
  int rc = validate(cfg);
  if (rc) return rc;
  if (cfg->divb != MHD_DIVB_CT) return MHD_ERR_ARG;
  if (!U || !B || !(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_ARG;
  for (int q = 0; q < 5; q++)
    if (!U[q]) return MHD_ERR_ARG;
  for (int q = 0; q < 3; q++)
    if (!B[q]) return MHD_ERR_ARG;
  Grid g = make_grid(cfg);
  long long elems = (long long)g.ext[0] * g.ext[1] * g.ext[2];
  long long field = (elems + 31) / 32 * 32;  // 256-byte aligned fields
  long long sc_doubles = (long long)((sizeof(DevScalars) + 255) / 256 * 256 / sizeof(double));
  const int ningr = cfg->emf == MHD_EMF_UCT_HLLD ? 6 : 5;
  long long need = field * (kNoAllocFields + 3 * (ningr - 5)) + sc_doubles;
  if (need > (long long)kNoAllocDoubles) return MHD_ERR_TOO_LARGE;
  double* base = nullptr;
  rc = noalloc_scratch(&base);
  if (rc) return rc;

  CK(allow_stage(cfg));
  // a context on the stack whose arrays are carved out of the static scratch
  mhd_ctx c{};
  c.cfg = *cfg;
  c.g = g;
  c.stream = (cudaStream_t)cfg->stream;
  c.own_stream = false;
  c.field_elems = (size_t)field;
  c.field_used = elems;
  c.pool = base;
  c.seglen = 16;
  double* p = base;
  auto next = [&]() { double* r = p; p += field; return r; };
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 8; q++) c.U[r].q[q] = next();
  for (int q = 0; q < 8; q++) c.P.q[q] = next();
  for (int q = 0; q < 6; q++) c.L.q[q] = next();
  for (int d = 0; d < 3; d++)
    for (int q = 0; q < ningr; q++) c.ING.a[d][q] = next();
  for (int d = 0; d < 3; d++) c.E.e[d] = next();
  c.lam = next();
  c.sc = reinterpret_cast<DevScalars*>(p);
  c.has_state = true;

  // the array keeps the previous call's contents: clear what this call uses,
  // then set the device scalars (bad_cell starts at the largest index)
  CK(cudaMemsetAsync(base, 0, (size_t)need * sizeof(double), c.stream));
  CK(cudaMemcpyAsync(c.sc, reset_scalars_source(), sizeof(DevScalars), cudaMemcpyHostToDevice, c.stream));
  for (int q = 0; q < 8; q++) {
    int e[3];
    slot_extents(g, q, e);
    rc = copy_field(c.g, c.stream, c.U[0].q[q], q < 5 ? U[q] : B[q - 5], nullptr, e, true);
    if (rc) return rc;
  }
  set_dt_kernel<<<1, 1, 0, c.stream>>>(c.sc, dt);
  run_step(&c, false);
  ghost_fill(&c, c.U[0]);  // the duplicate last face of periodic axes
  CK(cudaGetLastError());
  // a step that met a non-positive density or pressure leaves the caller's
  // arrays as they were: the status is read before anything is copied back
  DevScalars h;
  CK(copy_sync(&h, c.sc, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
  if (h.status) return h.status;
  for (int q = 0; q < 8; q++) {
    int e[3];
    slot_extents(g, q, e);
    rc = copy_field(c.g, c.stream, c.U[0].q[q], nullptr, q < 5 ? U[q] : B[q - 5], e, false);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c.stream));
  return MHD_OK;
}
