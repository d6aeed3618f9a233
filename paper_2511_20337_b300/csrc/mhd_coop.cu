// The fused stage of 2D constrained-transport grids (mhd_coop.cuh): context
// set-up, the cooperative launch of one RK stage, and the entry points of
// include/mhd.h that switch it, bound its waits and inject a missing arrival.
#include <cmath>

#include "mhd.h"
#include "mhd_coop.cuh"
#include "mhd_ctx.cuh"
#include "mhd_host.cuh"

using namespace mhd;

namespace mhd {

constexpr unsigned long long kDefaultWaitNs = 1000000000ull;  // 1 s
// Fused by default up to 256^2 cells: measured (PLM + HLLD + RK2, each form
// at its best segment length) level with or faster than the per-phase
// launches from 64^2 to 256^2 and within +-7 % above; mhd_autotune decides
// for any eligible grid.
constexpr long long kFusedDefaultCells = 256LL * 256;

template <int RECON, int RS>
void* coop_fn() {
  return (void*)coop_stage_kernel<RECON, RS>;
}
// The kernel of a configuration (reconstruction x the sweeps' solver).
static void* coop_kernel_of(const mhd_config& cfg) {
  const int rs = sweep_rs(&cfg);
  switch (cfg.recon) {
    case MHD_RECON_PLM:
      return rs == RS_HLL ? coop_fn<RECON_PLM, RS_HLL>()
                          : (rs == RS_HLLD ? coop_fn<RECON_PLM, RS_HLLD>() : coop_fn<RECON_PLM, RS_HLLD_UCT>());
    case MHD_RECON_WENOZ:
      return rs == RS_HLL ? coop_fn<RECON_WENOZ, RS_HLL>()
                          : (rs == RS_HLLD ? coop_fn<RECON_WENOZ, RS_HLLD>() : coop_fn<RECON_WENOZ, RS_HLLD_UCT>());
    default:
      return rs == RS_HLL ? coop_fn<RECON_PPM, RS_HLL>()
                          : (rs == RS_HLLD ? coop_fn<RECON_PPM, RS_HLLD>() : coop_fn<RECON_PPM, RS_HLLD_UCT>());
  }
}

static CoopBar bar_reset(unsigned long long limit_ns) {
  CoopBar h{};
  h.skip_block = -1;
  h.skip_at = -1;
  h.limit_ns = limit_ns;
  return h;
}

// 2D CT grids with the side-by-side sweeps' buffers qualify; the launch takes
// every block the device can hold at once (the cooperative limit).  On by
// default for grids up to kFusedDefaultCells.
int coop_init(mhd_ctx* c) {
  c->fused = false;
  c->coop_blocks = 0;
  c->coop_limit_ns = kDefaultWaitNs;
  if (c->g.ndim != 2 || c->g.glm || !c->split) return MHD_OK;
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop) return MHD_OK;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_kernel_of(c->cfg), kCoopThreads, 0));
  if (per_sm < 1) return MHD_OK;
  if (cudaMalloc(&c->bar, sizeof(CoopBar)) != cudaSuccess) {
    cudaGetLastError();
    return MHD_ERR_OOM;
  }
  const CoopBar h = bar_reset(c->coop_limit_ns);
  CK(copy_sync(c->bar, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  c->coop_blocks = per_sm * sms;
  c->fused = (long long)c->g.n[0] * c->g.n[1] <= kFusedDefaultCells;
  return MHD_OK;
}

void coop_free(mhd_ctx* c) {
  if (c->bar) cudaFree(c->bar);
  c->bar = nullptr;
}

bool fused_now(const mhd_ctx* c) { return c->fused && !c->prof_on; }

// One RK stage as one cooperative launch.
void coop_stage(mhd_ctx* c, int s, const F8& U0, const F8& Us, const F8& Out, bool cfl) {
  CoopStage a;
  a.g = c->g;
  a.U0 = U0;
  a.Us = Us;
  a.Out = Out;
  a.P = c->P;
  a.L = c->L;
  a.D = c->D[0];
  a.ING = c->ING;
  a.E = c->E;
  a.sc = c->sc;
  a.lam = c->lam;
  a.bar = c->bar;
  a.seglen = c->seglen;
  a.mode = stage_mode(c->cfg.rk, s);
  a.cfl = cfl ? 1 : 0;
  a.fast = s > 0 ? 1 : 0;
  // all axes periodic: each stage leaves the periodic images of its output,
  // which is the next stage's input, so the stages after the first skip
  // their ghost phase (the first keeps it: the host may have set U^n)
  const bool periodic = c->g.periodic[0] && c->g.periodic[1];
  a.ghost_out = periodic && s + 1 < c->cfg.rk ? 1 : 0;
  a.ghost_in = periodic && s > 0 ? 1 : 0;
  void* args[] = {&a};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)c->coop_blocks);
  lc.blockDim = dim3(kCoopThreads);
  lc.dynamicSmemBytes = 0;
  lc.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaLaunchKernelExC(&lc, coop_kernel_of(c->cfg), args);
  c->launches++;
}

// After a wait gave up: the barrier back to its initial state (the limit and
// no injected skip).  The stream must be idle.
int coop_clear(mhd_ctx* c) {
  if (!c->bar) return MHD_OK;
  const CoopBar h = bar_reset(c->coop_limit_ns);
  CK(copy_sync(c->bar, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  return MHD_OK;
}

}  // namespace mhd

extern "C" {

int mhd_set_fused(mhd_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return MHD_ERR_ARG;
  if (on && !c->bar) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->fused = on != 0;
  if (c->graph_ready) {  // the captured step holds the other launch sequence
    cudaGraphExecDestroy(c->graph);
    c->graph_ready = false;
  }
  return MHD_OK;
}

int mhd_get_fused(const mhd_ctx* c, int* on_out, int* blocks_out) {
  if (!c || !on_out) return MHD_ERR_ARG;
  *on_out = c->fused ? 1 : 0;
  if (blocks_out) *blocks_out = c->coop_blocks;
  return MHD_OK;
}

int mhd_set_wait_limit(mhd_ctx* c, double seconds) {
  if (!c || !(seconds > 0.0) || !(seconds <= 60.0)) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->coop_limit_ns = (unsigned long long)std::llround(seconds * 1e9);
  if (c->coop_limit_ns < 1) c->coop_limit_ns = 1;
  if (!c->bar) return MHD_OK;
  unsigned long long v = c->coop_limit_ns;
  CK(copy_sync(&c->bar->limit_ns, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
  return MHD_OK;
}

int mhd_inject_skip_arrive(mhd_ctx* c, int block, int barrier) {
  if (!c || !c->bar || block < -1 || barrier < -1) return MHD_ERR_ARG;
  if (block >= c->coop_blocks) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  int v[2] = {block, block < 0 ? -1 : barrier};
  CK(copy_sync(&c->bar->skip_block, v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
  return MHD_OK;
}

int mhd_fused_waits(mhd_ctx* c, int* waits_out) {
  if (!c || !waits_out) return MHD_ERR_ARG;
  *waits_out = 0;
  if (!c->bar) return MHD_OK;
  CK(cudaStreamSynchronize(c->stream));
  CK(copy_sync(waits_out, &c->bar->waits, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return MHD_OK;
}

}  // extern "C"
