// One launch per RK stage for 2D constrained-transport grids (the fused
// stage): a cooperative kernel runs the phases of a stage -- ghost fill,
// primitive recovery with the CFL candidates, the x and y sweeps side by side
// with the CFL decision, the UCT edge fields, CT + RK combine -- as
// grid-stride loops over the same item functions as the per-phase kernels,
// separated by grid barriers.  The arithmetic and its order are those of the
// side-by-side sweep path (the y sweep's raw flux differences combined with
// the x increment in the CT + RK item), so the state is the same to the bit.
//
// The barrier waits are bounded: a wait that runs past the context's limit
// marks the barrier as given up and sets MHD_ERR_TIMEOUT in the device
// status, and every block of the launch returns at its next barrier.  The
// mark stays until the host clears it, so later stage launches return at once
// and the state keeps the last completed step (each stage writes its output
// register only in its last phase, after its last barrier).
#pragma once
#include "mhd.h"
#include "mhd_kernels.cuh"

namespace mhd {

constexpr int kCoopThreads = 256;

// Grid barrier of one context's fused stage (device memory, 32 bytes).
// Arrivals are counted over the whole launch: barrier k (from 0) is complete
// once count reaches (k + 1) * gridDim.x.  A wait that gives up sets the
// kCoopAbort bit of count (arrivals never reach it), which ends every other
// wait at once and marks the launch (and, until the host clears it, every
// later one) as given up.  The last block to finish a completed launch zeroes
// count and exits.
constexpr unsigned int kCoopAbort = 0x40000000u;
struct CoopBar {
  unsigned int count;           // arrivals since the launch began (| kCoopAbort once given up)
  unsigned int exits;           // blocks that finished the launch
  int pad;
  int skip_block;               // fault injection: this block does not arrive at barrier skip_at (-1: off)
  int skip_at;
  int waits;                    // barriers per stage of the last launch (written by block 0)
  unsigned long long limit_ns;  // bound of every wait
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier k of the launch; every thread of every block calls it.  Thread 0
// arrives for its block with a release add (bar.sync has ordered the block's
// writes before it), polls with relaxed loads and ends with an acquire load;
// the closing bar.sync then orders every thread's later loads after that
// acquire, so they see what other blocks wrote before the barrier (measured
// at 1.20 us on 148 blocks, as fast as a cooperative-groups grid sync).
// skip_at: the barrier this block does not arrive at (fault injection; -1
// none), read once per launch.  Returns false on every thread of the block
// when the launch has given up.
__device__ __forceinline__ bool coop_sync(CoopBar* b, DevScalars* sc, int k, int skip_at) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (k != skip_at) red_release_add_u32(&b->count, 1u);
    const unsigned int target = (unsigned int)(k + 1) * gridDim.x;
    unsigned long long t0 = 0;
    unsigned int polls = 0;
    while (ld_relaxed_u32(&b->count) < target) {
      if ((++polls & 63u) != 0u) continue;  // the clock every 64 polls
      const unsigned long long t = global_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > b->limit_ns) {
        // the mark is a bit, set once however many waits run out together
        // (adding it would carry out of the word after four of them)
        if ((atomicOr(&b->count, kCoopAbort) & kCoopAbort) == 0u) atomicExch(&sc->status, MHD_ERR_TIMEOUT);
        break;
      }
    }
    // also false for a block that completed the barrier after the others gave up
    ok = ld_acquire_u32(&b->count) < kCoopAbort;
  }
  __syncthreads();
  return ok != 0;
}

// A device scalar that one block wrote before the last barrier and every
// block reads, as a strong load at device scope (not kept in the L1 from the
// stale copy the sweep items read).
__device__ __forceinline__ double ld_strong_f64(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_strong_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The end of a launch that completed: the last block out zeroes the counts.
__device__ __forceinline__ void coop_exit(CoopBar* b) {
  if (threadIdx.x == 0) {
    if (atomicAdd(&b->exits, 1u) == gridDim.x - 1) {
      b->count = 0u;
      b->exits = 0u;
    }
  }
}

// Arguments of one fused stage: Out = combine(U0, Us, L(Us)) as run_stage_regs.
struct CoopStage {
  Grid g;
  F8 U0, Us, Out, P;
  L6 L, D;          // x sweep: stage increment; y sweep: raw flux differences
  FaceIngr ING;
  E3 E;
  DevScalars* sc;
  double* lam;      // near-IEEE CFL rates (cfl)
  CoopBar* bar;
  int seglen, mode, cfl, fast;
  int ghost_in;     // Us's ghost zones are already filled (the previous fused stage's images)
  int ghost_out;    // write the periodic images of Out (all axes periodic)
};

template <int RECON, int RS>
static __global__ void __launch_bounds__(kCoopThreads, 1) coop_stage_kernel(CoopStage a) {
  constexpr bool EMF_HLLD = RS == RS_HLLD_UCT;
  __shared__ int live;
  int skip_at = -1;  // thread 0's injected missing arrival
  if (threadIdx.x == 0) {
    live = ld_relaxed_u32(&a.bar->count) < kCoopAbort;
    if (a.bar->skip_block == (int)blockIdx.x) skip_at = a.bar->skip_at;
  }
  __syncthreads();
  if (!live) return;
  const Grid& g = a.g;
  // Item ids go out a warp at a time, round-robin over the blocks (one per
  // SM): the phases with fewer items than threads then spread over every SM
  // and sub-partition instead of filling the first blocks, and a warp's 32
  // items stay consecutive (coalesced).
  const long long T = (long long)gridDim.x * blockDim.x;
  const long long t0 = ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
  int k = 0;
  // ghost zones of Us: periodic axes, then outflow axes (copy, then the normal field)
  if (a.ghost_in) {
    // the previous stage of this step wrote them with its output
  } else if (g.periodic[0] && g.periodic[1]) {
    const long long w = ghost_shell_work<2>(g);
    for (long long id = t0; id < w; id += T) ghost_shell_item<2>(g, a.Us, id);
    if (!coop_sync(a.bar, a.sc, k++, skip_at)) return;
  } else {
    for (int pass = 0; pass < 2; pass++)
      for (int d = 0; d < 2; d++) {
        if ((pass == 0) != (g.periodic[d] != 0)) continue;
        const long long w = ghost_layers_work(g, d);
        if (g.periodic[d]) {
          for (long long id = t0; id < w; id += T) ghost_periodic_item(g, a.Us, d, id);
        } else {
          for (long long id = t0; id < w; id += T) ghost_outflow_copy_item(g, a.Us, d, id);
          if (!coop_sync(a.bar, a.sc, k++, skip_at)) return;
          const long long r = ghost_rows_work(g, d);
          for (long long id = t0; id < r; id += T) ghost_outflow_normal_item(g, a.Us, d, id);
        }
        if (!coop_sync(a.bar, a.sc, k++, skip_at)) return;
      }
  }
  // primitives (+ the near-IEEE CFL rates and their maximum)
  {
    const long long w = prim_work<2>(g);
    double lam_max = 0.0;
    const int nxp = g.n[0] + 2 * g.G;
    for (long long id = t0; id < w; id += T) {
      if (a.fast) prim_item<2, false, true>(g, a.Us, a.P, a.sc, id);
      else prim_item<2, false, false>(g, a.Us, a.P, a.sc, id);
      if (a.cfl) {
        const int i = (int)(id % nxp) - g.G, j = (int)(id / nxp) - g.G;
        if (i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1]) {
          const int c = g.at(i, j, 0);
          Prim8 V;
          V.rho = a.P.q[0][c]; V.vx = a.P.q[1][c]; V.vy = a.P.q[2][c]; V.vz = a.P.q[3][c];
          V.bx = a.P.q[4][c]; V.by = a.P.q[5][c]; V.bz = a.P.q[6][c]; V.p = a.P.q[7][c];
          const double lam = cfl_rate_near_ieee<2>(g, V);
          a.lam[c] = lam;
          lam_max = (lam > lam_max) ? lam : lam_max;
        }
      }
    }
    if (a.cfl) block_max_into(lam_max, &a.sc->lapx_bits);
    if (!coop_sync(a.bar, a.sc, k++, skip_at)) return;
  }
  // the x and y sweeps side by side, both storing raw flux differences (x in
  // L, y in D), so that no sweep needs this step's dt.  The x items go to one
  // group of blocks and the y items to the rest, in proportion to their
  // counts, so that each SM runs one sweep body.  Then, over every block, the
  // CFL step: the IEEE rate of the candidates within 4e-13 of the maximum.
  {
    const long long nxi = sweep_work<0, 2>(g, a.seglen), nyi = sweep_work<1, 2>(g, a.seglen);
    int gx = (int)((nxi * gridDim.x + (nxi + nyi) / 2) / (nxi + nyi));
    gx = gx < 1 ? 1 : (gx > (int)gridDim.x - 1 ? (int)gridDim.x - 1 : gx);
    const bool xb = (int)blockIdx.x < gx;
    const int gb = xb ? gx : (int)gridDim.x - gx;
    const int bi = xb ? (int)blockIdx.x : (int)blockIdx.x - gx;
    const long long Tg = (long long)gb * blockDim.x;
    const long long tg = ((long long)(threadIdx.x >> 5) * gb + bi) * 32 + (threadIdx.x & 31);
    if (xb) {
      for (long long id = tg; id < nxi; id += Tg)
        sweep_item_direct<0, 2, RECON, RS>(g, a.P, a.Us.q[5], a.L, a.ING, a.sc, a.seglen, 2, id);
    } else {
      for (long long id = tg; id < nyi; id += Tg)
        sweep_item_direct<1, 2, RECON, RS>(g, a.P, a.Us.q[6], a.D, a.ING, a.sc, a.seglen, 2, id);
    }
    if (a.cfl) {
      const double M = __longlong_as_double((long long)ld_strong_u64(&a.sc->lapx_bits));
      const double Tm = M * (1.0 - 4e-13);
      const long long w = (long long)g.n[0] * g.n[1];
      double lam_max = 0.0;
      for (long long id = t0; id < w; id += T) {
        const int c = g.at((int)(id % g.n[0]), (int)(id / g.n[0]), 0);
        if (a.lam[c] >= Tm) {
          Prim8 V;
          V.rho = a.P.q[0][c]; V.vx = a.P.q[1][c]; V.vy = a.P.q[2][c]; V.vz = a.P.q[3][c];
          V.bx = a.P.q[4][c]; V.by = a.P.q[5][c]; V.bz = a.P.q[6][c]; V.p = a.P.q[7][c];
          const double lam = cfl_rate_ieee<2>(g, V);
          lam_max = (lam > lam_max) ? lam : lam_max;
        }
      }
      cfl_block_finish(lam_max, a.sc, g.cfl, gridDim.x);
    }
    if (!coop_sync(a.bar, a.sc, k++, skip_at)) return;
  }
  // UCT edge fields
  {
    const long long w = edge_work<2>(g);
    for (long long id = t0; id < w; id += T) emf_item<2, EMF_HLLD>(g, a.Us, a.ING, a.E, id);
    if (!coop_sync(a.bar, a.sc, k++, skip_at)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.bar->waits = k;
  // CT + RK combine (the stage's only write of its output register).  The x
  // increment fmul(-dt/dx, D_x) is the value the x sweep stores when it
  // scales its own differences (accumulate mode 0), formed in the same two
  // roundings, so the combine is that of the side-by-side sweeps to the bit.
  {
    const long long w = edge_work<2>(g);
    const double dt = ld_strong_f64(&a.sc->dt);  // formed by the CFL decision in this launch
    const double dtdx = fmul(dt, g.idx[0]);
    const int ex = g.n[0] + 1;
    for (long long id = t0; id < w; id += T) {
      const int i = (int)(id % ex), j = (int)(id / ex);
      if (i < g.n[0] && j < g.n[1]) {
        const int c = g.at(i, j, 0);
#pragma unroll
        for (int q = 0; q < 6; q++) a.L.q[q][c] = fmul(-dtdx, a.L.q[q][c]);
      }
      ct_rk_item<2, true>(g, a.U0, a.Us, a.Out, a.L, a.E, dt, a.mode, id, &a.D, &a.D);
      if (a.ghost_out && i < g.n[0] && j < g.n[1]) {
        // every ghost slot whose wrapped position is (i, j) takes its values
        // (the copies ghost_shell_item makes in the next stage's ghost phase)
        const int c = g.at(i, j, 0);
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) v[q] = a.Out.q[q][c];
        for (int jj = j - g.n[1] * ((j + g.G) / g.n[1]); jj <= g.n[1] + g.G; jj += g.n[1])
          for (int ii = i - g.n[0] * ((i + g.G) / g.n[0]); ii <= g.n[0] + g.G; ii += g.n[0]) {
            if (ii == i && jj == j) continue;
            const int d = g.at(ii, jj, 0);
#pragma unroll
            for (int q = 0; q < 8; q++) a.Out.q[q][d] = v[q];
          }
      }
    }
  }
  coop_exit(a.bar);
}

}  // namespace mhd
