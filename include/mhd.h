/*
 * libmhd — FP64 finite-volume ideal-MHD time step on one B300 (sm_103a).
 *
 * The method (paper §2 "Numerical methods"): the conservation law of
 * Eq. cons_law with the ideal-MHD state and flux tensor of Eq. mhd and the
 * total energy of Eq. Energy, advanced by the semi-discrete finite-volume
 * update of Eq. FV with an SSP Runge-Kutta integrator (Eq. RK3, and the
 * two-stage SSP-RK2).  Each stage recovers primitives (§2.2, the inversion
 * below Eq. reconstruct), reconstructs interface states (Eq. reconstruct:
 * PLM-minmod, WENO-Z or PPM), evaluates the Riemann flux of §2.2 (HLL or
 * HLLD), and evolves the staggered face field by constrained transport with
 * upwind (UCT) edge electric fields so that the discrete div B stays at
 * round-off (§2.2, last paragraph before §3).
 *
 * Conventions for every entry point:
 *   - returns 0 (MHD_OK) or a negative MHD_ERR_* code; nothing is thrown;
 *   - the caller owns every pointer it passes; the library copies in and out
 *     and never keeps a caller pointer after the call returns;
 *   - all device work runs on the stream given in mhd_config.stream (NULL =
 *     the legacy default stream); calls marked "async" return before the work
 *     is done, calls marked "sync" wait for that stream.
 *
 * State layout at the boundary (no ghost zones, x fastest, float64):
 *   cell arrays rho, mx, my, mz, E (and, in 2D, the cell-centred Bz):
 *       [nz][ny][nx]                                   (2D: nz = 1)
 *   face fields, stored at the left face of each cell (x0 + i dx, ...):
 *       Bx [nz][ny][nx+1],  By [nz][ny+1][nx],  Bz [nz+1][ny][nx] (3D only).
 *   On a periodic axis the last face equals the first: it is ignored on
 *   input and written as a copy of the first on output.
 */
#ifndef MHD_H
#define MHD_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define MHD_OK              0
#define MHD_ERR_ARG        -1   /* invalid argument or configuration */
#define MHD_ERR_CUDA       -2   /* a CUDA runtime call failed */
#define MHD_ERR_OOM        -3   /* device allocation failed */
#define MHD_ERR_UNPHYSICAL -4   /* a non-positive (or non-finite) density or pressure met in a stage */
#define MHD_ERR_TIMEOUT    -5   /* a bounded device-side wait gave up */
#define MHD_ERR_STATE      -6   /* no state has been set on this context */
#define MHD_ERR_TOO_LARGE  -7   /* grid needs more scratch than mhd_step_noalloc's fixed array */
#define MHD_ERR_DIVB       -8   /* the div B monitor (mhd_set_divb_check) found max |div B| h / max |B_c|
                                   above its tolerance */
#define MHD_ERR_GUARD      -9   /* a guard word after (or before) a device array was overwritten */

/* ---- options ---- */
#define MHD_RECON_PLM     0     /* piecewise linear, minmod limiter */
#define MHD_RECON_WENOZ   1     /* fifth-order WENO-Z (Borges et al. 2008) */
#define MHD_RECON_PPM     2     /* piecewise parabolic (Colella & Woodward 1984) */
#define MHD_RIEMANN_HLL   0
#define MHD_RIEMANN_HLLD  1     /* Miyoshi & Kusano 2005 */
#define MHD_BC_PERIODIC   0
#define MHD_BC_OUTFLOW    1     /* zero-gradient; normal ghost face field from div B = 0 */
#define MHD_MEM_HOST      0
#define MHD_MEM_DEVICE    1

typedef struct {
  int ndim;             /* 2 or 3 */
  int nx, ny, nz;       /* interior cells per axis (nz ignored in 2D) */
  double x0[3], x1[3];  /* domain bounds; dx = (x1 - x0) / n */
  double gamma;         /* adiabatic index of the ideal equation of state (Eq. Energy) */
  int recon;            /* MHD_RECON_* */
  int riemann;          /* MHD_RIEMANN_* */
  int rk;               /* 2 (SSP-RK2) or 3 (SSP-RK3, Eq. RK3) */
  double cfl;           /* Courant number of mhd_cfl_dt / mhd_advance */
  int bc[6];            /* x-, x+, y-, y+, z-, z+: MHD_BC_*; periodic needs both sides periodic */
  double p_floor;       /* floor on the recovered pressure (0 = none): a recovered pressure below
                           it is raised to it in the primitives only; the conserved energy is not
                           changed (the paper is silent on floors; see mhd_counters) */
  void* stream;         /* cudaStream_t for all device work; NULL = default stream */
  int divb;             /* MHD_DIVB_CT (0, constrained transport on staggered faces) or
                           MHD_DIVB_GLM (cell-centred B with GLM divergence cleaning) */
  double glm_alpha;     /* GLM damping constant alpha >= 0: after each step
                           psi <- psi exp(-alpha c_h dt / min dx); ignored for CT */
  int emf;              /* CT edge fields (§4.1 "UCT HLLD average"):
                           MHD_EMF_UCT_HLL (0): the UCT form with the HLL weights
                             a+ = S_R+/(S_R+ - S_L-), a- = -S_L-/(..), d = -S_R+ S_L-/(..);
                           MHD_EMF_UCT_HLLD (1, needs MHD_RIEMANN_HLLD and CT): the same form
                             with the HLLD solver's own weights, which write its flux of a
                             transverse field component as a^L F_L + a^R F_R + d^L B_L - d^R B_R
                             (three more face fields); not supported by mhd_adjoint */
} mhd_config;

#define MHD_DIVB_CT  0
#define MHD_DIVB_GLM 1
#define MHD_EMF_UCT_HLL  0
#define MHD_EMF_UCT_HLLD 1

typedef struct mhd_ctx mhd_ctx;   /* opaque; owns all device state of one grid */

/* Create a context on the current CUDA device: validates cfg, allocates the
 * device state (three RK registers, primitives, stage increment, face
 * ingredients and edge fields; about 55 doubles per padded cell in 3D).
 * The grid is the uniform Cartesian mesh of the finite-volume method of
 * paper §2.2: cell averages of rho, m, E at cell centres x0 + (i + 1/2) dx
 * and the staggered face field of constrained transport at the cell faces,
 * with the ghost layers a stencil of cfg->recon needs (2, or 3 for
 * WENO-Z / PPM).
 * *out receives the handle.  MHD_ERR_ARG on a bad configuration,
 * MHD_ERR_OOM if the device allocation fails.  Sync. */
int mhd_create(const mhd_config* cfg, mhd_ctx** out);

/* Release every device allocation of ctx.  Sync.  ctx may be NULL. */
int mhd_destroy(mhd_ctx* ctx);

/* Set the conserved state.  U[0..4] = rho, mx, my, mz, E (cell arrays);
 * B[0], B[1] = face Bx, By; B[2] = face Bz (3D) or cell Bz (2D); layout as in
 * the file header.  mem = MHD_MEM_HOST or MHD_MEM_DEVICE says where the
 * caller's arrays live (host arrays should be pinned for async copies).
 * Resets the simulation time to 0.  Async: the copies may still be running
 * when the call returns (pageable host arrays are staged before it returns,
 * pinned ones and device arrays are read later), so keep pinned or device
 * arrays unchanged until the stream has passed the copies. */
int mhd_set_conserved(mhd_ctx* ctx, int mem, const double* const* U, const double* const* B);

/* Set the state from primitives: rho, v[0..2], p (cell arrays) and the field
 * B[0..2] as in mhd_set_conserved.  The conserved variables follow from
 * m = rho v and Eq. Energy with the cell-centred field (mean of the two
 * bounding faces; 2D Bz is the cell value).  Async. */
int mhd_set_prim(mhd_ctx* ctx, int mem, const double* rho, const double* const* v, const double* p,
                 const double* const* B);

/* Copy the current conserved state out (same layout as mhd_set_conserved).
 * Sync.  Returns the device status of the last steps (MHD_ERR_UNPHYSICAL if a
 * non-positive density or pressure was met; see mhd_status). */
int mhd_get_conserved(mhd_ctx* ctx, int mem, double* const* U, double* const* B);

/* Change the boundary conditions (same encoding as mhd_config.bc).  Only
 * changes between periodic and outflow that keep the ghost width are allowed. */
int mhd_set_boundaries(mhd_ctx* ctx, const int bc[6]);

/* CFL time step of the current state (reading of the paper, which is silent):
 *   dt = cfl / max over interior cells of sum_d (|v_d| + cf_d) / dx_d,
 * cf_d the fast magnetosonic speed along d with the cell-centred B_d.
 * Computed on the device with IEEE operations in a fixed order.  Sync. */
int mhd_cfl_dt(mhd_ctx* ctx, double* dt_out);

/* Advance one time step of size dt: the RK stages of Eq. RK3 (SSP-RK3, or
 * the two-stage SSP-RK2), each stage U' = combine(U^n, U^s, L(U^s)) with L the
 * Delta t-scaled finite-volume increment of Eq. FV built from the
 * reconstruction of Eq. reconstruct and the Riemann flux of §2.2, and the face
 * field advanced by constrained transport with the UCT edge fields (§2.2, the
 * paragraph before §3; §4.1 "UCT HLLD average").  Async; a non-positive
 * density or pressure is reported by the next sync call. */
int mhd_step(mhd_ctx* ctx, double dt);

/* Advance nsteps steps as mhd_step does, each with its own CFL dt (the
 * reading of mhd_cfl_dt; the paper states no CFL condition) computed on the
 * device from the state at the start of that step, with no host round trip.
 * The launch sequence of a step is captured once in a CUDA graph and
 * replayed.  Async. */
int mhd_advance(mhd_ctx* ctx, int nsteps);

/* Simulation time (sum of the dt of all steps since the last set).  Sync. */
int mhd_get_time(mhd_ctx* ctx, double* t_out);

/* Set the simulation time (after mhd_set_conserved, which resets it to 0):
 * with mhd_get_conserved and mhd_get_time this checkpoints a run and resumes
 * it, the resumed steps equal to the bit to those of the uninterrupted run.
 * t must not be NaN.  Async. */
int mhd_set_time(mhd_ctx* ctx, double t);

/* dt of the last step taken by mhd_advance (or given to mhd_step).  Sync. */
int mhd_last_dt(mhd_ctx* ctx, double* dt_out);

/* Wait for the context's stream and report the first device-side error of the
 * steps since the last call: MHD_OK, or MHD_ERR_UNPHYSICAL with *bad_cell
 * (may be NULL) = the smallest flat interior index k*ny*nx + j*nx + i of a
 * cell whose recovered density or pressure was not positive, or
 * MHD_ERR_TIMEOUT (a grid barrier of the fused stage gave up; *bad_cell = -1;
 * see mhd_set_fused), or MHD_ERR_DIVB.  Clears it. */
int mhd_status(mhd_ctx* ctx, long long* bad_cell);

/* div B monitor (CT only; MHD_ERR_ARG with GLM).  Constrained transport keeps
 * the discrete divergence of the staggered face field at round-off (paper
 * §2.2, the paragraph on the induction equation before §3):
 *   div_c = sum_d (B_d at the upper face - B_d at the lower face) / dx_d
 * per interior cell.  The monitor forms
 *   rel = max_c |div_c| h / max_c |B_c|,   h = min_d dx_d,
 * B_c the cell-centred field (mean of the two faces; 2D B_z the cell value).
 * mhd_set_divb_check(ctx, tol): tol > 0 checks rel at the end of every later
 * step (a few microseconds of device work per step, captured with the step);
 * a step with rel > tol sets the status MHD_ERR_DIVB, reported by the next
 * sync call with *bad_cell the flat index of the cell of largest |div| h
 * (compared in single precision; ties go to the larger index).  tol = 0
 * turns it off (the default).  Sync.
 * mhd_divb(ctx, &rel): rel of the current state, without setting a status.  Sync. */
int mhd_set_divb_check(mhd_ctx* ctx, double tol);
int mhd_divb(mhd_ctx* ctx, double* rel_out);

/* Event counters since the last state set (sync):
 *   *recon_fallbacks: cell reconstructions (per cell, direction and stage)
 *     that fell back to first order because a reconstructed density or
 *     pressure was not positive;
 *   *pressure_floors: interior-cell primitive recoveries (per cell and
 *     primitive pass) whose pressure was raised to p_floor.
 * Either pointer may be NULL. */
int mhd_counters(mhd_ctx* ctx, long long* recon_fallbacks, long long* pressure_floors);

/* Number of kernel launches the library issued on this context so far
 * (graph replays count the kernels inside the graph). */
long long mhd_launch_count(const mhd_ctx* ctx);

/* Sweep segment length: the number of faces one thread of a sweep marches
 * (default: the longest of 2..256 that leaves about eight waves of threads
 * on the device in the sweep with the fewest faces).  Shorter segments give
 * more threads, longer ones fewer repeated Riemann solves and reconstructions
 * at segment ends (one each per segment); the result does not depend on it.
 * >= 1.  Sync. */
int mhd_set_seglen(mhd_ctx* ctx, int seglen);

/* The segment length in use (the default, the last mhd_set_seglen or the
 * mhd_autotune choice). */
int mhd_get_seglen(const mhd_ctx* ctx, int* seglen_out);

/* Choose the segment length by timing two CFL steps for each of 2, 4, 8, 12,
 * 16, 20, 24, 28, 32, 40, 48, 64, 96, 128 and the lengths that split the longest
 * pencil's faces into 4..12 equal segments (up to twice the longest axis) on
 * the current state, which is restored
 * afterwards together with the time and counters; *seglen_out (may be NULL)
 * receives the choice.  Where the fused stage is available (see below) both
 * launch forms are timed and the faster is kept (mhd_get_fused reports it).
 * Sync; allocates a temporary copy of the state. */
int mhd_autotune(mhd_ctx* ctx, int* seglen_out);

/* ---- fused stage (2D, CT) ----
 *
 * On 2D constrained-transport grids small enough that the y sweep runs beside
 * the x sweep (below about 670^2 cells), each RK stage (Eq. RK3, or the
 * two-stage SSP-RK2) is one cooperative kernel launch instead of one launch
 * per phase.  Its phases -- ghost fill, primitive recovery with the CFL step
 * of mhd_cfl_dt, the two sweeps (Eq. FV), the UCT edge fields and the CT + RK
 * combine (§2.2) -- execute the same item arithmetic in the same order, separated by
 * grid-wide barriers, so the state equals the per-phase launches' to the bit.
 * It is on by default for grids of up to 256^2 cells (where it was measured
 * level with or faster than the per-phase launches) on devices with
 * cooperative launches; mhd_autotune picks the faster form for any eligible
 * grid.
 * Profiling (mhd_profile_steps) and the adjoint's recompute context use the
 * per-phase launches.
 *
 * Every barrier wait is bounded (default 1 s).  A wait that runs out sets
 * MHD_ERR_TIMEOUT in the device status; every block of the launch returns at
 * its next barrier, later stage launches return at once, and the next sync
 * call (mhd_status, mhd_get_conserved) reports it and re-arms the barrier.
 * The conserved state is then that of the last completed step (a stage writes
 * its output only after its last barrier); the time and counters may include
 * the failed step's.
 *
 * mhd_set_fused(ctx, on): 1 = fused stages (MHD_ERR_ARG where the context does
 *   not qualify: 3D, GLM, larger 2D grids, no cooperative launch), 0 = one
 *   launch per phase.  Sync.
 * mhd_get_fused(ctx, &on, &blocks): whether the fused stage is on, and the
 *   blocks of its launch (0 where the context does not qualify; blocks may be
 *   NULL).
 * mhd_set_wait_limit(ctx, seconds): the bound of every wait, 0 < seconds <= 60.
 *   Sync.
 * mhd_inject_skip_arrive(ctx, block, barrier): fault injection for tests:
 *   from the next launch on, block `block` does not arrive at barrier
 *   `barrier` (counted from 0 within each stage launch) of every stage, so
 *   that barrier's wait runs out; block = -1 turns it off.  A timeout report
 *   by mhd_status also turns it off.  Sync.
 * mhd_fused_waits(ctx, &n): the barriers of the last fused stage launch
 *   that completed its edge fields.  Sync. */
int mhd_set_fused(mhd_ctx* ctx, int on);
int mhd_get_fused(const mhd_ctx* ctx, int* on_out, int* blocks_out);
int mhd_set_wait_limit(mhd_ctx* ctx, double seconds);
int mhd_inject_skip_arrive(mhd_ctx* ctx, int block, int barrier);
int mhd_fused_waits(mhd_ctx* ctx, int* waits_out);

/* Static text for a return code. */
const char* mhd_strerror(int code);

/* ---- guard words ----
 *
 * Not an operation of the paper: a check of the library's own memory.  Every
 * device array of a context (each field of its pool: RK registers,
 * primitives, increments, face ingredients, edge fields, CFL rates) is
 * followed by at least 32 guard words, and the pool starts with 32 of them.
 * The words hold a signalling-NaN bit pattern that no arithmetic produces and
 * no memset writes.  They are written once, when the context is made; no
 * launch of a step reads or writes them, so they cost nothing per step (256
 * bytes per field).  A changed word means that some launch wrote outside the
 * array it was given.
 *
 * mhd_check_guards(ctx, &field, &word): sync; scans every guard word of the
 *   context's pool.  MHD_OK (field = -1, word = -1) when all are intact, else
 *   MHD_ERR_GUARD with the first damaged word in pool order: `field` is the
 *   array's index in the pool (0 .. nfields-1) and `word` counts from the
 *   array's end (0 = the first word past its last element), or is negative
 *   for the words before field 0 (-1 = the word just before it).  The guard
 *   stays damaged; later checks report it again.
 * mhd_guard_layout(ctx, &nfields, &used, &words_after): the pool's field
 *   count, the elements each field uses (the cells of the grid with its ghost
 *   zones), and the guard words after each field (>= 32).
 * mhd_inject_guard_write(ctx, field, word): for tests: writes 0.0 into guard
 *   word (field, word) from the host, as an out-of-bounds store would;
 *   MHD_ERR_ARG where (field, word) is not a guard word.  Sync.
 * The batched ensemble and the domain have the same check over every run's
 * block and every brick (mhd_batch_check_guards, mhd_domain_check_guards). */
#define MHD_GUARD_SEND -2   /* mhd_domain_check_guards: a brick's region of the halo send buffer */
#define MHD_GUARD_RECV -3   /* ... of the halo receive buffer */
int mhd_check_guards(mhd_ctx* ctx, int* field, long long* word);
int mhd_guard_layout(const mhd_ctx* ctx, int* nfields, long long* used, long long* words_after);
int mhd_inject_guard_write(mhd_ctx* ctx, int field, long long word);

/* ---- divergence cleaning (divb = MHD_DIVB_GLM) ----
 *
 * The div B control the paper uses for its strong-scaling runs (§2.1, citing
 * Dedner et al. 2002 and Mignone et al. 2010; §4.1, §4.2): cell-centred B and
 * a scalar psi.  At each face the (B_n, psi) system, linear with speeds
 * -+c_h, is solved exactly (B_m = (B_n^L + B_n^R)/2 - (psi^R - psi^L)/(2 c_h),
 * psi_m = (psi^L + psi^R)/2 - c_h (B_n^R - B_n^L)/2; fluxes psi_m for B_n and
 * c_h^2 B_m for psi) and the Riemann solver runs with normal field B_m.
 * c_h = cfl / (dt sum_d 1/dx_d); after each step psi is multiplied by
 * exp(-glm_alpha c_h dt / min dx).  In this mode the B arrays of
 * mhd_set_conserved, mhd_set_prim and mhd_get_conserved are cell arrays
 * [nz][ny][nx] (Bx, By, Bz), setting the state sets psi = 0, and there is no
 * pressure floor (p_floor must be 0).  The batched, adjoint and
 * allocation-free entry points are CT-only (MHD_ERR_ARG). */

/* psi in or out: one cell array [nz][ny][nx], host or device per mem.
 * MHD_ERR_ARG on a CT context.  set: async; get: sync. */
int mhd_set_psi(mhd_ctx* ctx, int mem, const double* psi);
int mhd_get_psi(mhd_ctx* ctx, int mem, double* psi);

/* ---- batched ensemble ----
 *
 * Many independent grids advanced together (the ensemble workload of the
 * benchmark: uneven 2D Orszag-Tang runs with their own plasma beta and Mach
 * number).  All runs share ndim, recon, riemann, rk and the boundary kinds;
 * each has its own size, domain, gamma, cfl, p_floor and CFL dt.  Every kernel
 * of a stage is one launch over all runs (each block serves one run, so every
 * run executes exactly the single-grid arithmetic), and a step is captured
 * once in a CUDA graph and replayed.  The stream is cfgs[0].stream. */
typedef struct mhd_batch mhd_batch;

/* Validate every cfgs[r] (same scheme and boundary kinds; MHD_ERR_ARG
 * otherwise) and allocate the device state of all runs.  Sync. */
int mhd_batch_create(int nruns, const mhd_config* cfgs, mhd_batch** out);
int mhd_batch_destroy(mhd_batch* b);

/* State of one run, layout and mem as in mhd_set_conserved / mhd_get_conserved.
 * Setting resets that run's time and counters.  set: async; get: sync. */
int mhd_batch_set_conserved(mhd_batch* b, int run, int mem, const double* const* U, const double* const* B);
int mhd_batch_get_conserved(mhd_batch* b, int run, int mem, double* const* U, double* const* B);

/* As mhd_batch_get_conserved, without waiting: the copies are queued in the
 * batch's stream order, so reading many runs costs one wait
 * (mhd_batch_synchronize) instead of one per run.  The destination arrays
 * must stay valid, and host ones pinned, until that wait returns.  Async. */
int mhd_batch_get_conserved_async(mhd_batch* b, int run, int mem, double* const* U, double* const* B);

/* Wait until the batch's queued work and copies are done.  Sync. */
int mhd_batch_synchronize(mhd_batch* b);

/* Packed state I/O: the states of all runs as one contiguous array of
 * mhd_batch_packed_size(b) doubles -- run 0's 8 slots (rho, mx, my, mz, E,
 * B[0], B[1], B[2], each in the layout of mhd_batch_set_conserved, x
 * fastest), then run 1's, and so on.  One copy and one scatter (gather)
 * kernel replace 8 copies per run.  A host array is staged through a device
 * buffer of that size, allocated on first use (the call then waits for it);
 * a device array is read or written in place.  Setting resets every run's
 * time and counters.  Both calls are async: keep the array unchanged (set)
 * or unread (get) until mhd_batch_synchronize returns; host arrays should be
 * pinned. */
long long mhd_batch_packed_size(const mhd_batch* b);
int mhd_batch_set_conserved_packed(mhd_batch* b, int mem, const double* packed);
int mhd_batch_get_conserved_packed(mhd_batch* b, int mem, double* packed);

/* Advance every run nsteps steps, each run with its own CFL dt computed on the
 * device.  Every run must have a state (MHD_ERR_STATE).  Async. */
int mhd_batch_step(mhd_batch* b, int nsteps);

/* Choose the sweep segment length (faces a thread marches; shorter segments
 * give more threads, longer ones fewer repeated Riemann solves) for the runs
 * of at most 128^2 cells and for the larger ones, by timing two steps of each
 * of 16 candidates on the current states, which are restored afterwards.
 * Writes the choice (either pointer may be NULL).  Sync; allocates a
 * temporary copy of the states. */
int mhd_batch_autotune(mhd_batch* b, int* seglen_small, int* seglen_large);

/* Set the two segment lengths directly (>= 1).  Sync. */
int mhd_batch_set_seglen(mhd_batch* b, int seglen_small, int seglen_large);

/* Simulation time of every run (t_out[nruns]).  Sync. */
int mhd_batch_get_times(mhd_batch* b, double* t_out);

/* First device-side error of any run (as mhd_status, with *bad_run the run's
 * index, -1 if none).  Sync; does not clear. */
int mhd_batch_status(mhd_batch* b, int* bad_run, long long* bad_cell);
/* Guard words of every run's block of fields (see "guard words"): MHD_OK, or
 * MHD_ERR_GUARD with the run, field and word of the first damaged word
 * (lowest run first).  Sync. */
int mhd_batch_check_guards(mhd_batch* b, int* run, int* field, long long* word);

/* Kernel launches issued by the batch so far (graph replays count their kernels). */
long long mhd_batch_launch_count(const mhd_batch* b);

/* ---- adjoint ----
 *
 * Gradient of a functional J of the final state with respect to the initial
 * state, by the transpose of every kernel of the step (the discrete adjoint:
 * exact up to rounding for the scheme as executed, with the limiter, wave-fan
 * and min/max branches the forward values take; where an argument of minmod
 * is exactly zero, minmod's derivative is taken as zero).  The step sizes are
 * treated as constants (frozen): the CFL maximum is not differentiated.
 *   MHD_FUNC_MAGNETIC_ENERGY  J = 1/2 sum_cells |B_c|^2 dV, B_c the mean of
 *                             the cell's two faces (2D B_z: the cell value);
 *   MHD_FUNC_MISFIT           J = 1/2 sum_cells sum_q (U_q - T_q)^2 dV over
 *                             rho, m_x, m_y, m_z, E (2D: and the cell B_z).
 * Supported: PLM, WENO-Z or PPM reconstruction (for WENO-Z the derivative of
 * the weights is taken, so the gradient is that of the nonlinear scheme; for
 * PPM the clip and steepening choices the forward values take), HLL or HLLD,
 * RK2 or RK3, UCT-HLL or UCT-HLLD edge fields (UCT-HLLD: through the
 * solver's fan-region weights and star ratios), periodic or outflow axes
 * (outflow: the transposes of the zero-gradient copies and of the ghost normal
 * field's div B = 0 march), at least 2G+1 cells per axis (5 for PLM, 7 for
 * WENO-Z and PPM; MHD_ERR_ARG otherwise).  On a periodic axis the face at n is
 * the ghost copy of face 0 and its gradient entry is 0; on an outflow axis it
 * is a face of its own. */
#define MHD_FUNC_MAGNETIC_ENERGY 0
#define MHD_FUNC_MISFIT          1

/* Run nsteps steps from the context's state, evaluate J and its gradient with
 * respect to that initial state, and keep the gradient in the context.
 *   dts:        host array of nsteps step sizes, or NULL for the CFL dt of
 *               every step (computed in the forward pass, then frozen);
 *   ckpt_every: k >= 1; the state is saved every k steps and each block of k
 *               steps recomputed once in the reverse pass (device memory:
 *               ceil(nsteps/k) + k*rk + 1 states plus ~128 scratch fields);
 *   target:     for MHD_FUNC_MISFIT, 5 (3D) or 6 (2D: + B_z) cell arrays in
 *               the layout of mhd_set_conserved, host or device per mem;
 *               ignored (may be NULL) otherwise;
 *   J_out, dts_out (nsteps): J and the step sizes used; may be NULL.
 * Afterwards the context holds the final state (as after the same steps with
 * mhd_step), its time advanced by the sum of the step sizes.  Sync;
 * allocates the adjoint's buffers on first use (freed by mhd_destroy).
 * MHD_ERR_UNPHYSICAL if the forward pass met a non-positive density or
 * pressure. */
int mhd_adjoint_run(mhd_ctx* ctx, int nsteps, const double* dts, int ckpt_every, int functional, int mem,
                    const double* const* target, double* J_out, double* dts_out);

/* The last mhd_adjoint_run's gradient with respect to the initial conserved
 * state: gU[5] cell arrays and gB[3] face arrays (2D: gB[2] the cell B_z), in
 * the layout of mhd_get_conserved.  The duplicate last face of a periodic axis
 * carries 0: the whole derivative of that face sits on face 0.  MHD_ERR_STATE
 * before a successful run.  Sync. */
int mhd_adjoint_grad_conserved(mhd_ctx* ctx, int mem, double* const* gU, double* const* gB);

/* The last mhd_adjoint_run's gradient with respect to the initial density and
 * velocity, holding the initial pressure and magnetic field fixed (cell
 * arrays: grad_rho, grad_v[3]).  MHD_ERR_STATE before a successful run.  Sync. */
int mhd_adjoint_grad_prim(mhd_ctx* ctx, int mem, double* grad_rho, double* const* grad_v);

/* ---- domain decomposition ----
 *
 * One grid split into px x py x pz bricks (paper §3.4 "Multi GPU
 * communication", Fig. par_ex: the domain is split between processes and, at
 * every stage, the data each neighbour needs -- 8 neighbours in 2D, 26 in 3D,
 * diagonal ones included -- is packed into device buffers, exchanged and
 * unpacked into the ghost zones).  Each brick is a single-grid context on the
 * current device; its ghost fill is replaced by
 *   pack     (one kernel per brick: the boxes of its interior its neighbours
 *             need, into its send buffer),
 *   exchange (one device-to-device copy per brick and neighbour, from the
 *             sender's send buffer into the receiver's receive buffer),
 *   unpack   (one kernel per brick: its receive buffer into its ghost shell),
 * followed by the outflow fill on the sides that lie on an outflow boundary
 * of the whole grid.  Every ghost slot then holds the undivided grid's value,
 * so the bricks advance exactly as the undivided grid does: the state after
 * any number of steps, the CFL step (the least of the bricks' steps) and the
 * time equal the undivided grid's to the bit.  All bricks run on the one
 * device and on cfg->stream; this is the decomposition and the exchange of a
 * multi-GPU run with the transfers made by local device copies.
 *
 * Brick layout: bricks are numbered x fastest over the brick grid; axis d of
 * N cells splits into parts[d] spans, the first N % parts[d] of them one cell
 * longer.  Constraints (MHD_ERR_ARG otherwise): constrained transport
 * (divb = MHD_DIVB_CT), parts[d] >= 1 (1 on inactive axes), at least G + 1
 * cells per brick on every active axis (G = 2 for PLM, 3 otherwise), at most
 * 4096 bricks. */
typedef struct mhd_domain mhd_domain;

/* One box of a brick's halo exchange, in the brick's padded coordinates
 * (cell index -G .. n+G per active axis, 0 on inactive ones):
 *   peer    the neighbouring brick;
 *   dir     its direction (-1, 0 or +1 per axis);
 *   lo, ext first slot and slots per axis (ext = 1 on inactive axes);
 *   offset  first slot of the box in the brick's send (receive) buffer; the
 *           buffer holds, box after box, the 8 state fields of the box
 *           field-major (field q of slot k at 8 offset + q slots_of_box + k),
 *           slots x fastest.
 * A send box (dir o) is the part of the brick's interior the neighbour in
 * direction o needs: per axis o = +1: [n-G, n-1]; o = -1: [0, G]; o = 0:
 * [0, n-1].  A receive box (dir o) is the ghost region in direction o:
 * o = -1: [-G, -1]; o = +1: [n, n+G]; o = 0: [0, n-1] (the slot n+G of the
 * upper layers is the last face of a face array).  The box a brick sends in
 * direction o lands in the box its peer receives from direction -o; the two
 * have the same extents.  Periodic axes wrap around the brick grid; across an
 * outflow boundary of the whole grid there is no neighbour and no box. */
typedef struct {
  int peer;
  int dir[3];
  int lo[3];
  int ext[3];
  long long offset;
} mhd_halo_box;

/* Host-only index maps (no device work; usable without a GPU):
 * mhd_domain_brick: the first global cell lo[3] and the cells n[3] of brick
 *   `brick` (inactive axes: lo 0, n 1);
 * mhd_domain_halo: the brick's send boxes (send != 0) or receive boxes
 *   (send == 0) in direction order (x fastest over dir, all-zero skipped),
 *   at most max_boxes of them (26 suffice), *nboxes their number. */
int mhd_domain_brick(const mhd_config* cfg, const int parts[3], int brick, int lo[3], int n[3]);
int mhd_domain_halo(const mhd_config* cfg, const int parts[3], int brick, int send, mhd_halo_box* boxes,
                    int max_boxes, int* nboxes);

/* Create the bricks (one context each, with the whole grid's dx) and the
 * exchange buffers on the current device.  Sync. */
int mhd_domain_create(const mhd_config* cfg, const int parts[3], mhd_domain** out);
int mhd_domain_destroy(mhd_domain* d);

/* The whole grid's state in the boundary layout of this file (host or device
 * per mem), scattered to the bricks; resets the time and counters.  Async as
 * mhd_set_conserved. */
int mhd_domain_set_conserved(mhd_domain* d, int mem, const double* const* U, const double* const* B);

/* Gather the whole grid's state (after an exchange, so a periodic axis's last
 * face is a copy of the first).  Sync; returns the device status as
 * mhd_domain_status. */
int mhd_domain_get_conserved(mhd_domain* d, int mem, double* const* U, double* const* B);

/* The CFL step of the whole grid (as mhd_cfl_dt), without advancing the time.  Sync. */
int mhd_domain_cfl_dt(mhd_domain* d, double* dt_out);

/* One step of size dt (async), or nsteps CFL steps with dt on the device,
 * captured once in a CUDA graph and replayed (async). */
int mhd_domain_step(mhd_domain* d, double dt);
int mhd_domain_advance(mhd_domain* d, int nsteps);

/* Simulation time of the whole grid.  Sync. */
int mhd_domain_get_time(mhd_domain* d, double* t_out);

/* First device-side error of any brick since the last call (as mhd_status),
 * *bad_cell (may be NULL) the smallest flat index of the whole grid,
 * k*ny*nx + j*nx + i, among the bricks' first bad cells.  Sync; clears. */
int mhd_domain_status(mhd_domain* d, long long* bad_cell);

/* Sums of the bricks' counters (as mhd_counters).  The pressure floors count
 * interior cells, as on the undivided grid; the reconstruction fallbacks count
 * every reconstruction a brick's sweeps made, and a brick also reconstructs
 * the cells next to it in its halo, so that count can exceed the undivided
 * grid's.  Sync. */
int mhd_domain_counters(mhd_domain* d, long long* recon_fallbacks, long long* pressure_floors);

/* Sweep segment length of every brick (as mhd_set_seglen).  Sync. */
int mhd_domain_set_seglen(mhd_domain* d, int seglen);

/* Kernel launches so far (graph replays count their kernels); bytes moved by
 * one exchange (all bricks, all boxes). */
long long mhd_domain_launch_count(const mhd_domain* d);
long long mhd_domain_halo_bytes(const mhd_domain* d);
/* Guard words of every brick's context and of every brick's region of the
 * halo send and receive buffers (each region has 32 guard words before it and
 * at least 32 after it): MHD_OK, or MHD_ERR_GUARD with the brick and either
 * the field of its pool or MHD_GUARD_SEND / MHD_GUARD_RECV, and the word as
 * in mhd_check_guards.  Bricks' pools are scanned first.  Sync. */
int mhd_domain_check_guards(mhd_domain* d, int* brick, int* field, long long* word);

/* ---- allocation-free variant ----
 *
 * For callers that must not allocate device memory: for example code whose
 * device memory is owned by another allocator or a fixed budget (a framework's
 * caching pool, a pre-reserved arena), or code that may not block on the
 * device-wide synchronisation that cudaMalloc and cudaFree can imply.  The
 * paper has no counterpart; this is a property of the library only.
 *
 * mhd_step_noalloc advances the caller's state, held in device memory in the
 * boundary layout of this file (U[0..4] cells, B[0..2] fields, as in
 * mhd_set_conserved), by one step of size dt, in place.  It creates no
 * context: every intermediate array (the padded RK registers, primitives,
 * stage increment, face ingredients, edge fields and the device scalars)
 * lives in one file-scope device array of MHD_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.  The call allocates
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine).
 *
 * Limit: the padded scratch -- 57 float64 fields with the UCT-HLL edge fields,
 * 60 with UCT-HLLD, each over the padded box (nx+2G+1)(ny+2G+1)(nz+2G+1)
 * rounded up to 32 elements (G = 2 for PLM, 3 otherwise; 2D: no z padding),
 * plus 256 bytes of device scalars -- must fit in the array.  Largest square
 * and cubic grids that fit:
 *                  2D PLM   2D WENO-Z/PPM   3D PLM   3D WENO-Z/PPM
 *     UCT-HLL       266^2       264^2        36^3        34^3
 *     UCT-HLLD      259^2       257^2        36^3        34^3
 * Larger grids are rejected with MHD_ERR_TOO_LARGE before any device work.
 *
 * The array is shared by every call and keeps the last call's contents: the
 * call clears the part it uses before the step.  Calls that overlap on the GPU
 * (from several host threads or streams at once) race on it and must not be
 * made.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; that may load the
 * library's device code on that device, which is when the driver reserves the
 * array -- make that first call before any stream capture and before any
 * phase that must not see device memory change.  Work runs on cfg->stream
 * (NULL = legacy default stream) and the call waits for it.  A step that met
 * a non-positive density or pressure returns MHD_ERR_UNPHYSICAL and leaves the
 * caller's arrays as they were.  Sync. */
#define MHD_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int mhd_step_noalloc(const mhd_config* cfg, double* const* U, double* const* B, double dt);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
