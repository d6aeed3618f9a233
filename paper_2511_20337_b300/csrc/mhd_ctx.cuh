// The single-grid context behind mhd_ctx* and the launch helpers of one RK
// stage, shared by the entry points of mhd_api.cu and the adjoint of
// mhd_adjoint.cu.  Internal to the library.
#pragma once
#include "mhd.h"
#include "mhd_glm.cuh"
#include "mhd_kernels.cuh"

namespace mhd {
struct AdjointState;
struct CoopBar;
}

struct mhd_ctx {
  mhd_config cfg;
  mhd::Grid g;
  cudaStream_t stream;
  bool own_stream;
  size_t field_elems;  // words from one field's start to the next's: the used words, rounded up, + guard
  long long field_used;  // words a field uses (the grid's cells with ghost zones)
  int pool_fields;     // fields in the pool
  double* pool;        // every field lives in this one allocation, after kGuardWords guard words
  mhd::F8 U[3];        // RK registers (U[0] = U^n); each register's 8 fields are contiguous
  mhd::F8 P;           // primitives of the stage input
  mhd::L6 L;           // stage increment of the cell variables
  mhd::FaceIngr ING;   // UCT face ingredients
  mhd::E3 E;           // edge fields
  double* lam;         // near-IEEE CFL rate of every cell (the candidate pass of the CFL step)
  mhd::DevScalars* sc;
  bool has_state;
  int seglen;
  long long launches;
  int launches_per_step;
  cudaGraphExec_t graph;
  bool graph_ready;
  // profiling: an event after every launch, tagged with its kernel class
  bool prof_on;
  int prof_n;
  cudaEvent_t prof_ev[128];
  int prof_cls[128];
  mhd::AdjointState* adj;  // buffers of the adjoint, made by its first run
  // divergence cleaning (g.glm): 9-field registers; GU[r].q[0..7] alias U[r]
  // (cell B in slots 5..7), GU[r].q[8] is psi
  mhd::F9 GU[3], GP, GL;
  int reg_fields;          // fields per RK register: 8 (CT) or 9 (GLM); contiguous
  // grids too small to fill the device with one sweep (CT): the y (and z)
  // sweeps run beside the x sweep on streams aux[], joined by events, and
  // leave their raw flux differences in D[0] (D[1]); ct_rk completes the stage
  // increment in the sequential order, so the result is the same to the bit
  bool split;
  cudaStream_t aux[2];
  cudaEvent_t ev_fork, ev_join[2];
  mhd::L6 D[2];
  // div B monitor at the end of every step (CT): 0 = off, else the tolerance
  // on max |div B| h / max |B_c| above which a step reports MHD_ERR_DIVB
  double divb_tol;
  // fused stage (2D CT grids with the side-by-side sweep buffers): each RK
  // stage is one cooperative launch of coop_blocks blocks whose phases are
  // separated by grid barriers in *bar, every wait bounded by coop_limit_ns
  bool fused;
  int coop_blocks;
  unsigned long long coop_limit_ns;
  mhd::CoopBar* bar;
};

namespace mhd {

void prof_mark(mhd_ctx* c, int cls);
void ghost_fill(mhd_ctx* c, const F8& S);
// primitives of S into c->P (+ CFL dt); fast: c2p_fast (the stages after the
// first, whose primitives decide nothing that must match the oracle bitwise)
void prim(mhd_ctx* c, const F8& S, bool cfl, bool fast = false);
void sweeps(mhd_ctx* c, const F8& S);                // all directions: c->L and c->ING
void emf(mhd_ctx* c, const F8& S);                   // edge fields into c->E
void ct_rk(mhd_ctx* c, const F8& U0, const F8& Us, const F8& Out, int mode);
int stage_mode(int rk, int s);                       // COMB_* of stage s
// Stage s of a step with explicit registers: Out = combine(U0, Us, L(Us)).
void run_stage_regs(mhd_ctx* c, int s, const F8& U0, const F8& Us, const F8& Out, bool cfl);
void run_stage(mhd_ctx* c, int s, bool cfl);         // on the context's registers
void run_step(mhd_ctx* c, bool device_dt);
void divb_check(mhd_ctx* c, double tol);            // the div B monitor on U[0] (tol 0: measure only)
void adjoint_free(mhd_ctx* c);                       // defined in mhd_adjoint.cu
bool split_now(const mhd_ctx* c);                    // sweeps side by side in this launch sequence
int sweep_rs(const mhd_config* cfg);                 // the sweeps' Riemann-solver template value
// fused stage (mhd_coop.cu)
int coop_init(mhd_ctx* c);                           // eligibility, barrier, blocks; fused on where eligible
void coop_free(mhd_ctx* c);
bool fused_now(const mhd_ctx* c);                    // fused stages in this launch sequence
void coop_stage(mhd_ctx* c, int s, const F8& U0, const F8& Us, const F8& Out, bool cfl);
int coop_clear(mhd_ctx* c);                          // the barrier's initial state after a timeout

}  // namespace mhd
