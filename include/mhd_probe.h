/*
 * libmhd measurement entry points (not part of the method).
 *
 * The paper reports wall-clock throughput only (cell-updates per second, §4);
 * these calls give the per-kernel device times and the FP64 peak that the
 * benchmark needs to place a kernel on its roofline.  Same conventions as
 * mhd.h: int return codes, caller-owned pointers, work on the context stream.
 */
#ifndef MHD_PROBE_H
#define MHD_PROBE_H

#include "mhd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* kernel classes of one time step */
#define MHD_KCLASS_GHOST    0   /* ghost-zone fill */
#define MHD_KCLASS_PRIM     1   /* primitive recovery (+ CFL reduction) */
#define MHD_KCLASS_SWEEP_X  2   /* reconstruction + Riemann + flux difference, x */
#define MHD_KCLASS_SWEEP_Y  3
#define MHD_KCLASS_SWEEP_Z  4
#define MHD_KCLASS_EMF      5   /* UCT edge fields */
#define MHD_KCLASS_CT_RK    6   /* CT face update + RK combine */
#define MHD_KCLASS_OTHER    7   /* step-size bookkeeping */
#define MHD_NKCLASS         8

/* Advance nsteps CFL steps exactly as mhd_advance does, but launching each
 * kernel eagerly with a CUDA event recorded after it on the context stream.
 * ms_out[MHD_NKCLASS] receives the summed device time per kernel class
 * (milliseconds, event-to-event) and launches_out[MHD_NKCLASS] (may be NULL)
 * the launch counts.  Sync. */
int mhd_profile_steps(mhd_ctx* ctx, int nsteps, double* ms_out, int* launches_out);

/* As mhd_profile_steps, for a batched ensemble (mhd_batch_step's kernels). */
typedef struct mhd_batch mhd_batch;
int mhd_batch_profile_steps(mhd_batch* b, int nsteps, double* ms_out, int* launches_out);

/* kernel classes of the adjoint's reverse pass (0..7 above: forward kernels
 * re-run inside the stage transposes) */
#define MHD_AKCLASS_COMBINE 8   /* RK-combine and CT-curl transposes */
#define MHD_AKCLASS_EDGE    9   /* UCT edge-field transposes */
#define MHD_AKCLASS_RIEMANN 10  /* Riemann solver + flux difference transposes */
#define MHD_AKCLASS_RECON   11  /* PLM reconstruction transposes */
#define MHD_AKCLASS_C2P     12  /* primitive-recovery transposes */
#define MHD_AKCLASS_GHOST   13  /* ghost-fill transposes */
#define MHD_NAKCLASS        14

/* Run mhd_adjoint_run(ctx, nsteps, dts, ckpt_every, MHD_FUNC_MAGNETIC_ENERGY,
 * ...) with CUDA events on the context stream: phase_ms[3] = device time of
 * the forward pass, of the block recomputes and of the reverse pass;
 * class_ms[MHD_NAKCLASS] splits the reverse pass by kernel class (event to
 * event, so a memset counts with the kernel after it).  Syncs after every
 * reverse step.  Leaves the context as mhd_adjoint_run does. */
int mhd_adjoint_profile(mhd_ctx* ctx, int nsteps, const double* dts, int ckpt_every, double* phase_ms,
                        double* class_ms);

/* The adjoint's vector-Jacobian product of the Riemann solver
 * (MHD_RIEMANN_HLL / _HLLD) on n faces, by two independent routes: the
 * forward-mode multi-tangent evaluation of the solver (dual) and the
 * hand-written reverse the adjoint uses (hand).  Host arrays:
 * in[15 n] = (rho, u, v, w, b1, b2, p of the left state, the same of the
 * right state, b_n) per face in the sweep frame; cot[12 n] = (7 flux
 * cotangents, 5 UCT-ingredient cotangents a+, a-, d, u_L, u_R); dual and
 * hand [15 n] receive the cotangents of the 15 inputs.  Sync. */
int mhd_probe_riemann_vjp(int riemann, int n, double gamma, const double* in, const double* cot, double* dual,
                          double* hand);

/* The same with the edge-field form: emf = MHD_EMF_UCT_HLL, or
 * MHD_EMF_UCT_HLLD with riemann = MHD_RIEMANN_HLLD (the solver's own weights,
 * whose reverse runs through the fan regions' star ratios and speeds).
 * cot[13 n] = (7 flux cotangents, 6 ingredient cotangents in the order of
 * mhd_probe_riemann's ing: a^L, a^R, d^L, u_L, u_R, d^R; for UCT-HLL a+, a-,
 * d, u_L, u_R and a sixth that is ignored).  Sync. */
int mhd_probe_riemann_vjp_emf(int riemann, int emf, int n, double gamma, const double* in, const double* cot,
                              double* dual, double* hand);

/* The ghost fill of a CT context and its transpose, for the dot-product check
 * <fill(x), abar> = <x, fill^T(abar)>.  x, abar: host arrays [8][E] of whole
 * padded fields (E = ext_x ext_y ext_z, ext_d = n_d + 2G + 1 on active axes,
 * 1 otherwise, G = 2 for PLM and 3 for WENO-Z / PPM, x fastest), in the slot
 * order of the state (rho, m_x, m_y, m_z, E, B_x, B_y, B_z faces; 2D: cell
 * B_z in slot 7).  fx receives the filled x, xbar the transpose applied to
 * abar (what the adjoint does at the end of every stage).  MHD_ERR_ARG on a
 * GLM context.  Sync. */
int mhd_probe_ghost_vjp(mhd_ctx* ctx, const double* x, const double* abar, double* fx, double* xbar);

/* One first RK stage of a CT context, U* = U + L(U) with step dt, and its
 * transpose: grad = J^T w, J the Jacobian of U* with respect to U and w a
 * cotangent of U* on the evolved cells and faces (the combine transpose
 * reads w there only).  U, w, grad:
 * host arrays in the layout of mhd_set_conserved (rho, m_x, m_y, m_z, E, then
 * the three face fields; 2D: cell B_z in slot 7).  Allocates the adjoint's
 * buffers on first use and leaves the context's step size at dt (its state and
 * time are not changed).  MHD_ERR_ARG on a GLM context.  Sync. */
int mhd_probe_stage_vjp(mhd_ctx* ctx, const double* const* U, double dt, const double* const* w,
                        double* const* grad);

/* The sweeps' Riemann solver (MHD_RIEMANN_HLL / _HLLD) on n faces, with the
 * UCT-HLL or (emf = MHD_EMF_UCT_HLLD, HLLD only) UCT-HLLD face weights.
 * Host arrays: in[15 n] as for mhd_probe_riemann_vjp; F[7 n] receives the
 * sweep-frame flux (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) and ing[6 n] the
 * ingredients (a^L, a^R, d^L, u_L, u_R, d^R; UCT-HLL: a+, a-, d, u_L, u_R, d).
 * Sync. */
int mhd_probe_riemann(int riemann, int emf, int n, double gamma, const double* in, double* F, double* ing);

/* Both per-cell CFL rates of the single-grid step (the rate of the CFL
 * reading: sum over the ndim axes of (|v_d| + c_f,d) / dx_d, c_f,d the fast
 * speed with the cell field B_d) for n primitive states: near_out[n] gets the
 * candidate-pass rate (IEEE products and sums, approximate square roots and
 * reciprocal) and ieee_out[n] the IEEE rate that decides the step.  prim is
 * a host array [n][8] = (rho, vx, vy, vz, bx, by, bz, p); dx[3] the cell
 * widths (> 0); gamma > 1.  Sync. */
int mhd_probe_cfl_rate(int ndim, double gamma, const double* dx, int n, const double* prim, double* near_out,
                       double* ieee_out);

/* Measure the FP64 pipe's throughput on the current device: every SM runs
 * eight independent chains of dependent DFMA per thread (all operands in
 * registers, the addend shared by the chains) for about 20 ms;
 * *gflops_out = 2 * DFMA per second / 1e9.  Sync; allocates and frees a
 * small device buffer. */
int mhd_probe_fp64(double* gflops_out);

/* The issue rate of the FP64 pipe for the instruction forms below, each
 * measured as mhd_probe_fp64 is, reported as 2 * instructions per second / 1e9
 * (so directly comparable with a DFMA peak).  rates[MHD_FP64_NFORMS]; about
 * 0.1 s.  Sync. */
#define MHD_FP64_FORM_DFMA          0  /* DFMA, operands in registers, shared addend (= mhd_probe_fp64) */
#define MHD_FP64_FORM_DFMA_CONST    1  /* DFMA with literal (constant) multiplier and addend */
#define MHD_FP64_FORM_DFMA_DISTINCT 2  /* DFMA, register operands, a different addend register per chain */
#define MHD_FP64_FORM_DMUL          3  /* DMUL of two registers */
#define MHD_FP64_FORM_DADD          4  /* DADD of two registers */
#define MHD_FP64_NFORMS             5
int mhd_probe_fp64_forms(double* rates);

#ifdef __cplusplus
}
#endif
#endif /* MHD_PROBE_H */
