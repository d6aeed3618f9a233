// Kernels of one finite-volume CT stage of ideal MHD (paper §2.2) on the
// padded device layout.
//
// Device layout: every field (8 state slots, 8 primitives, the stage
// increment, 5 face ingredients per direction, 3 edge fields) is a separate
// float64 array over the padded box i in [-G, nx+G], j in [-G, ny+G],
// k in [-G, nz+G] (2D: k = 0 only), x fastest.  The extra outermost slot holds
// the last face of face-centred arrays; index i of a face array is the face at
// x0 + i dx (left face of cell i).  State slots: 0 rho, 1-3 m, 4 E, 5-7 the
// face fields Bx, By, Bz (2D: slot 7 is the cell-centred Bz).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "mhd_math.cuh"

namespace mhd {

enum { RECON_PLM = 0, RECON_WENOZ = 1, RECON_PPM = 2 };
// Riemann solver of the sweeps; RS_HLLD_UCT is the HLLD flux with the solver's
// own UCT weights (UCT-HLLD edge fields) in place of the HLL ones.
enum { RS_HLL = 0, RS_HLLD = 1, RS_HLLD_UCT = 2 };

struct Grid {
  int ndim;
  int n[3];        // interior cells (n[2] = 1 in 2D)
  int G;           // ghost width on active axes
  int ext[3];      // padded extents
  int sy, sz;      // strides in elements
  int origin;      // offset of cell (0,0,0)
  int periodic[3];
  double dx[3], idx[3];
  double gamma, gm1, igm1, cfl, p_floor;
  int glm;         // 1: cell-centred B and psi (divergence cleaning), 0: CT
  __host__ __device__ __forceinline__ int at(int i, int j, int k) const { return origin + i + j * sy + k * sz; }
  __host__ __device__ __forceinline__ int stride(int d) const { return d == 0 ? 1 : (d == 1 ? sy : sz); }
  __host__ __device__ __forceinline__ int lo(int d) const { return d < ndim ? -G : 0; }
  __host__ __device__ __forceinline__ int hi(int d) const { return d < ndim ? n[d] + G : 0; }  // inclusive
};

struct F8 { double* q[8]; };
// UCT face ingredients per direction: a^L, a^R, d^L, u_L, u_R and (UCT-HLLD
// only, else null) d^R at each face; the flux of a transverse field component
// at the face is a^L F_L + a^R F_R + d^L B_L - d^R B_R (UCT-HLL: d^R = d^L).
struct FaceIngr { double* a[3][6]; };
struct E3 { double* e[3]; };
struct L6 { double* q[6]; };            // stage increment of rho, mx, my, mz, E (2D: + Bz)

struct DevScalars {                     // small device-side scalars of one context
  unsigned long long lmax_bits;         // max CFL rate of this step (as bits of a positive double)
  unsigned int blocks_done;             // ticket counter of the CFL reduction
  int status;                           // 0 or MHD_ERR_UNPHYSICAL
  long long bad_cell;                   // smallest flat index of a bad cell
  double dt;                            // current step
  double time;                          // accumulated time
  unsigned long long fallbacks;         // first-order reconstruction fallbacks
  unsigned long long floors;            // interior pressures raised to the floor
  unsigned long long lapx_bits;         // max of the near-IEEE CFL rates (candidate search)
  unsigned long long divb_key;          // div B check: float bits of max |div B| h (high) and its cell (low)
  unsigned long long bmax_bits;         // div B check: max |B_c|^2 over interior cells (bits)
  double divb_rel;                      // div B check: the last max |div B| h / max |B_c|
};

// ---------------------------------------------------------------------------
// Ghost zones.  Periodic axes first (x, y, z), then outflow axes (x, y, z);
// each pass covers the full padded transverse range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap(int g, int n) {
  int r = g % n;
  return r < 0 ? r + n : r;
}

// Periodic pass along axis d: every slot at d-index in [-G,-1] U [n, n+G].
__host__ __device__ __forceinline__ long long ghost_layers_work(const Grid& g, int d) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  return (long long)(g.hi(t1) - g.lo(t1) + 1) * (g.hi(t2) - g.lo(t2) + 1) * (2 * g.G + 1);
}
__device__ __forceinline__ void ghost_periodic_item(const Grid& g, const F8& S, int d, long long id) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  int e1 = g.hi(t1) - g.lo(t1) + 1;
  int nl = 2 * g.G + 1;
  int l = (int)(id % nl);
  long long r = id / nl;
  int a = (int)(r % e1) + g.lo(t1);
  int b = (int)(r / e1) + g.lo(t2);
  int gi = l < g.G ? l - g.G : g.n[d] + (l - g.G);
  int x[3];
  x[d] = gi;
  x[t1] = a;
  x[t2] = b;
  int dst = g.at(x[0], x[1], x[2]);
  x[d] = wrap(gi, g.n[d]);
  int src = g.at(x[0], x[1], x[2]);
#pragma unroll
  for (int q = 0; q < 8; q++) S.q[q][dst] = S.q[q][src];
}
static __global__ void ghost_periodic_kernel(Grid g, F8 S, int d) {
  const long long total = ghost_layers_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ghost_periodic_item(g, S, d, id);
}

// All axes periodic: every ghost cell in one pass, copied from its interior
// cell with every index wrapped.  The same values as the passes above (there a
// corner takes a stale copy in the first pass and the wrapped one in a later
// pass).  The shell is enumerated as slabs, one per axis d: d-index in the
// ghost layers, the axes after d interior and the axes before d over the full
// padded range (so each ghost cell is in the slab of its highest ghost axis).
template <int NDIM>
__host__ __device__ __forceinline__ long long ghost_shell_slab(const Grid& g, int d) {
  long long w = 2 * g.G + 1;
  for (int t = 0; t < NDIM; t++)
    if (t < d) w *= g.n[t] + 2 * g.G + 1;
    else if (t > d) w *= g.n[t];
  return w;
}
template <int NDIM>
__host__ __device__ __forceinline__ long long ghost_shell_work(const Grid& g) {
  long long w = 0;
  for (int d = 0; d < NDIM; d++) w += ghost_shell_slab<NDIM>(g, d);
  return w;
}
template <int NDIM>
__device__ __forceinline__ void ghost_shell_item(const Grid& g, const F8& S, long long id) {
  int d = NDIM - 1;
  while (d > 0) {  // slabs of the outer axes come first
    const long long w = ghost_shell_slab<NDIM>(g, d);
    if (id < w) break;
    id -= w;
    d--;
  }
  const int nl = 2 * g.G + 1;
  int x[3] = {0, 0, 0};
  for (int t = 0; t < NDIM; t++) {  // axis t: full range (t < d), ghost layer (t == d), interior (t > d)
    const int e = t < d ? g.n[t] + nl : (t == d ? nl : g.n[t]);
    const int v = (int)(id % e);
    id /= e;
    x[t] = t < d ? v - g.G : (t == d ? (v < g.G ? v - g.G : g.n[t] + (v - g.G)) : v);
  }
  const int dst = g.at(x[0], x[1], x[2]);
  const int src = g.at(wrap(x[0], g.n[0]), NDIM > 1 ? wrap(x[1], g.n[1]) : 0, NDIM > 2 ? wrap(x[2], g.n[2]) : 0);
#pragma unroll
  for (int q = 0; q < 8; q++) S.q[q][dst] = S.q[q][src];
}
template <int NDIM>
static __global__ void ghost_shell_kernel(Grid g, F8 S) {
  const long long total = ghost_shell_work<NDIM>(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ghost_shell_item<NDIM>(g, S, id);
}

// Outflow pass along axis d, part 1: zero-gradient copies of every slot except
// the normal face field (d-index -1..-G from 0; n..n+G from n-1).  sides
// selects the low (bit 0) and high (bit 1) side; a brick of a decomposed grid
// has an outflow boundary on one side of an axis only.
__device__ __forceinline__ void ghost_outflow_copy_item(const Grid& g, const F8& S, int d, long long id,
                                                        int sides = 3) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  int e1 = g.hi(t1) - g.lo(t1) + 1;
  int nl = 2 * g.G + 1;
  int qn = (d < g.ndim) ? 5 + d : -1;
  int l = (int)(id % nl);
  long long r = id / nl;
  int a = (int)(r % e1) + g.lo(t1);
  int b = (int)(r / e1) + g.lo(t2);
  int gi = l < g.G ? l - g.G : g.n[d] + (l - g.G);
  if (!(sides & (gi < 0 ? 1 : 2))) return;
  int x[3];
  x[d] = gi;
  x[t1] = a;
  x[t2] = b;
  int dst = g.at(x[0], x[1], x[2]);
  x[d] = gi < 0 ? 0 : g.n[d] - 1;
  int src = g.at(x[0], x[1], x[2]);
#pragma unroll
  for (int q = 0; q < 8; q++)
    if (q != qn) S.q[q][dst] = S.q[q][src];
}
static __global__ void ghost_outflow_copy_kernel(Grid g, F8 S, int d) {
  const long long total = ghost_layers_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ghost_outflow_copy_item(g, S, d, id);
}

// Outflow pass along axis d, part 2: the normal face field of each ghost cell
// from a vanishing discrete div B, marching outward from the boundary face.
__host__ __device__ __forceinline__ long long ghost_rows_work(const Grid& g, int d) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  int e1 = g.hi(t1) - g.lo(t1) + (t1 < g.ndim ? 0 : 1);  // transverse range [-G, n+G-1]
  int e2 = g.hi(t2) - g.lo(t2) + (t2 < g.ndim ? 0 : 1);
  return (long long)e1 * e2;
}
__device__ __forceinline__ void ghost_outflow_normal_item(const Grid& g, const F8& S, int d, long long id,
                                                          int sides = 3) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  int e1 = g.hi(t1) - g.lo(t1) + (t1 < g.ndim ? 0 : 1);
  double* Bn = S.q[5 + d];
  int a = (int)(id % e1) + g.lo(t1);
  int b = (int)(id / e1) + g.lo(t2);
  auto divT = [&](int cell) {
    int x[3];
    x[d] = cell;
    x[t1] = a;
    x[t2] = b;
    int c = g.at(x[0], x[1], x[2]);
    double s = 0.0;
    bool first = true;
    int ts[2] = {t1, t2};
    for (int m = 0; m < 2; m++) {
      int t = ts[m];
      if (t >= g.ndim) continue;
      const double* Bt = S.q[5 + t];
      double term = d_(s_(Bt[c + g.stride(t)], Bt[c]), g.dx[t]);
      s = first ? term : a_(s, term);
      first = false;
    }
    return s;
  };
  int x[3];
  x[t1] = a;
  x[t2] = b;
  for (int m = 1; m <= g.G && (sides & 1); m++) {
    x[d] = -m;
    int c = g.at(x[0], x[1], x[2]);
    Bn[c] = a_(Bn[c + g.stride(d)], m_(g.dx[d], divT(-m)));
  }
  for (int m = 0; m < g.G && (sides & 2); m++) {
    int cell = g.n[d] + m;
    x[d] = cell;
    int c = g.at(x[0], x[1], x[2]);
    Bn[c + g.stride(d)] = s_(Bn[c], m_(g.dx[d], divT(cell)));
  }
}
static __global__ void ghost_outflow_normal_kernel(Grid g, F8 S, int d) {
  const long long total = ghost_rows_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ghost_outflow_normal_item(g, S, d, id);
}

// ---------------------------------------------------------------------------
// Primitive recovery on every padded cell that has both faces; optional CFL
// rate over interior cells reduced to a device dt (the last block to finish
// forms dt = cfl / max rate and adds it to the time).  Also flags interior
// cells with a non-positive (or NaN) density or pressure.
// ---------------------------------------------------------------------------
template <int NDIM>
__host__ __device__ __forceinline__ long long prim_work(const Grid& g) {
  return (long long)(g.n[0] + 2 * g.G) * (g.n[1] + 2 * g.G) * (NDIM == 3 ? g.n[2] + 2 * g.G : 1);
}
// One padded cell: primitives, floor, status; returns its CFL rate (interior
// cells, CFL pass) or 0.  FAST: c2p_fast, with c2p_ieee's pressure wherever
// the floor or positivity test is within c2p_fast's error bound (the passes
// after the CFL pass; the CFL pass keeps c2p_ieee, whose primitives the exact
// CFL decision reads).
template <int NDIM, bool CFL, bool FAST = false>
__device__ __forceinline__ double prim_item(const Grid& g, const F8& S, const F8& P, DevScalars* sc, long long id) {
  const int nxp = g.n[0] + 2 * g.G, nyp = g.n[1] + 2 * g.G;
  int i = (int)(id % nxp) - g.G;
  long long r = id / nxp;
  int j = (int)(r % nyp) - g.G;
  int k = NDIM == 3 ? (int)(r / nyp) - g.G : 0;
  int c = g.at(i, j, k);
  double bx = m_(0.5, a_(S.q[5][c], S.q[5][c + 1]));
  double by = m_(0.5, a_(S.q[6][c], S.q[6][c + g.sy]));
  double bz = NDIM == 3 ? m_(0.5, a_(S.q[7][c], S.q[7][c + g.sz])) : S.q[7][c];
  Prim8 V;
  if (FAST) {
    double pb;
    V = c2p_fast(S.q[0][c], S.q[1][c], S.q[2][c], S.q[3][c], S.q[4][c], bx, by, bz, g.gm1, pb);
    if (lt_abs(fsub(V.p, g.p_floor), pb) || lt_abs(V.p, pb))
      V.p = c2p_ieee(S.q[0][c], S.q[1][c], S.q[2][c], S.q[3][c], S.q[4][c], bx, by, bz, g.gm1).p;
  } else {
    V = c2p_ieee(S.q[0][c], S.q[1][c], S.q[2][c], S.q[3][c], S.q[4][c], bx, by, bz, g.gm1);
  }
  bool interior = i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && k >= 0 && k < g.n[2];
  if (V.p < g.p_floor) {  // primitives only; the conserved energy is not changed
    V.p = g.p_floor;
    if (interior) atomicAdd(&sc->floors, 1ull);
  }
  P.q[0][c] = V.rho;
  P.q[1][c] = V.vx;
  P.q[2][c] = V.vy;
  P.q[3][c] = V.vz;
  P.q[4][c] = V.bx;
  P.q[5][c] = V.by;
  P.q[6][c] = V.bz;
  P.q[7][c] = V.p;
  double lam = 0.0;
  if (interior) {
    if (!(V.rho > 0.0) || !(V.p > 0.0)) {
      long long flat = ((long long)k * g.n[1] + j) * g.n[0] + i;
      atomicExch(&sc->status, -4);
      atomicMin((unsigned long long*)&sc->bad_cell, (unsigned long long)flat);
    }
    if (CFL) {
      double B2 = a_(a_(m_(V.bx, V.bx), m_(V.by, V.by)), m_(V.bz, V.bz));
      lam = m_(a_(dabs(V.vx), fast_speed_ieee(V.rho, V.p, B2, V.bx, g.gamma)), g.idx[0]);
      lam = a_(lam, m_(a_(dabs(V.vy), fast_speed_ieee(V.rho, V.p, B2, V.by, g.gamma)), g.idx[1]));
      if (NDIM == 3) lam = a_(lam, m_(a_(dabs(V.vz), fast_speed_ieee(V.rho, V.p, B2, V.bz, g.gamma)), g.idx[2]));
    }
  }
  return lam;
}
// Block maximum of rates (positive doubles: their bits order like unsigned
// integers), folded into *dst.  Every thread of the block must call this.
__device__ __forceinline__ void block_max_into(double lam_max, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam_max = fmax(lam_max, __shfl_xor_sync(0xffffffffu, lam_max, o));
  __shared__ double wm[8];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wm[wid] = lam_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmax(m, wm[w]);
    atomicMax(dst, (unsigned long long)__double_as_longlong(m));
  }
}

// Block maximum of the CFL rates, folded into the grid's maximum; the last of
// the grid's nblocks blocks forms dt = cfl / max rate and adds it to the time.
// Every thread of the block must call this.
__device__ __forceinline__ void cfl_block_finish(double lam_max, DevScalars* sc, double cfl, unsigned int nblocks) {
  // rates are positive: their bit patterns order like unsigned integers
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam_max = fmax(lam_max, __shfl_xor_sync(0xffffffffu, lam_max, o));
  __shared__ double wmax[8];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wmax[wid] = lam_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmax(m, wmax[w]);
    atomicMax(&sc->lmax_bits, (unsigned long long)__double_as_longlong(m));
    __threadfence();
    unsigned int ticket = atomicAdd(&sc->blocks_done, 1u);
    if (ticket == nblocks - 1) {
      __threadfence();
      double lmax = __longlong_as_double((long long)atomicAdd(&sc->lmax_bits, 0ull));
      double dt = d_(cfl, lmax);
      sc->dt = dt;
      sc->time = sc->time + dt;
      sc->lmax_bits = 0ull;
      sc->lapx_bits = 0ull;
      sc->blocks_done = 0u;
    }
  }
}

// CFL rate of one interior cell from its primitives: with IEEE operations
// throughout (prim_item's rate), or with the square roots and division
// replaced by refined seeds (fast_speed_near_ieee, within ~1e-14 of it).
template <int NDIM>
__device__ __forceinline__ double cfl_rate_near_ieee(const Grid& g, const Prim8& V) {
  double B2 = a_(a_(m_(V.bx, V.bx), m_(V.by, V.by)), m_(V.bz, V.bz));
  double lam = m_(a_(dabs(V.vx), fast_speed_near_ieee(V.rho, V.p, B2, V.bx, g.gamma)), g.idx[0]);
  lam = a_(lam, m_(a_(dabs(V.vy), fast_speed_near_ieee(V.rho, V.p, B2, V.by, g.gamma)), g.idx[1]));
  if (NDIM == 3) lam = a_(lam, m_(a_(dabs(V.vz), fast_speed_near_ieee(V.rho, V.p, B2, V.bz, g.gamma)), g.idx[2]));
  return lam;
}
template <int NDIM>
__device__ __forceinline__ double cfl_rate_ieee(const Grid& g, const Prim8& V) {
  double B2 = a_(a_(m_(V.bx, V.bx), m_(V.by, V.by)), m_(V.bz, V.bz));
  double lam = m_(a_(dabs(V.vx), fast_speed_ieee(V.rho, V.p, B2, V.bx, g.gamma)), g.idx[0]);
  lam = a_(lam, m_(a_(dabs(V.vy), fast_speed_ieee(V.rho, V.p, B2, V.by, g.gamma)), g.idx[1]));
  if (NDIM == 3) lam = a_(lam, m_(a_(dabs(V.vz), fast_speed_ieee(V.rho, V.p, B2, V.bz, g.gamma)), g.idx[2]));
  return lam;
}
// Primitive pass of the single grid (FAST: c2p_fast, for the stages after the
// first); with CFL, the near-IEEE rate of every
// interior cell goes to lam_near and its maximum to sc->lapx_bits (the
// IEEE decision follows in cfl_exact_kernel).
template <int NDIM, bool CFL, bool FAST>
static __global__ void __launch_bounds__(256) prim_kernel(Grid g, F8 S, F8 P, DevScalars* sc, double* lam_near) {
  const long long total = prim_work<NDIM>(g);
  double lam_max = 0.0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    prim_item<NDIM, false, FAST>(g, S, P, sc, id);
    if (CFL) {
      const int nxp = g.n[0] + 2 * g.G, nyp = g.n[1] + 2 * g.G;
      int i = (int)(id % nxp) - g.G;
      long long r = id / nxp;
      int j = (int)(r % nyp) - g.G;
      int k = NDIM == 3 ? (int)(r / nyp) - g.G : 0;
      if (i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && k >= 0 && k < g.n[2]) {
        const int c = g.at(i, j, k);
        Prim8 V;
        V.rho = P.q[0][c]; V.vx = P.q[1][c]; V.vy = P.q[2][c]; V.vz = P.q[3][c];
        V.bx = P.q[4][c]; V.by = P.q[5][c]; V.bz = P.q[6][c]; V.p = P.q[7][c];
        const double lam = cfl_rate_near_ieee<NDIM>(g, V);
        lam_near[c] = lam;
        lam_max = (lam > lam_max) ? lam : lam_max;
      }
    }
  }
  if (CFL) block_max_into(lam_max, &sc->lapx_bits);
}

// CFL step in two passes (single-grid path): the primitive pass stores, per
// interior cell, the rate computed with fast_speed_near_ieee (within ~1e-14
// of the IEEE rate) and its maximum M; this pass recomputes the IEEE rate of
// prim_item only where the stored rate is within 4e-13 of M -- the cell of
// the largest IEEE rate is among them -- and forms dt from their maximum:
// the same dt, to the bit, as the IEEE rate of every cell.
template <int NDIM>
static __global__ void __launch_bounds__(256) cfl_exact_kernel(Grid g, F8 P, const double* __restrict__ lam_near,
                                                               DevScalars* sc) {
  const double M = __longlong_as_double((long long)sc->lapx_bits);
  const double T = M * (1.0 - 4e-13);
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  double lam_max = 0.0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int i = (int)(id % g.n[0]);
    long long r = id / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    int c = g.at(i, j, k);
    if (lam_near[c] >= T) {
      Prim8 V;
      V.rho = P.q[0][c]; V.vx = P.q[1][c]; V.vy = P.q[2][c]; V.vz = P.q[3][c];
      V.bx = P.q[4][c]; V.by = P.q[5][c]; V.bz = P.q[6][c]; V.p = P.q[7][c];
      const double lam = cfl_rate_ieee<NDIM>(g, V);
      lam_max = (lam > lam_max) ? lam : lam_max;
    }
  }
  cfl_block_finish(lam_max, sc, g.cfl, gridDim.x);
}

// ---------------------------------------------------------------------------
// div B monitor (constrained transport keeps the discrete divergence of the
// face field at round-off, paper §2.2): per interior cell
//   div = sum_d (B_d(face +) - B_d(face -)) / dx_d,
// the largest |div| h (h = min dx) with its cell, and the largest |B_c|^2 of
// the cell-centred field (2D: B_z the cell value).  divb_finish_kernel forms
// rel = max |div| h / max |B_c| and, when rel > tol (tol > 0), reports
// MHD_ERR_DIVB with the cell of the largest |div| h (its value taken in
// single precision for the key; ties go to the larger index).
// ---------------------------------------------------------------------------
template <int NDIM>
static __global__ void __launch_bounds__(256) divb_kernel(Grid g, F8 S, DevScalars* sc) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  const double h = NDIM == 3 ? fmin(g.dx[0], fmin(g.dx[1], g.dx[2])) : fmin(g.dx[0], g.dx[1]);
  unsigned long long key = 0ull, b2max = 0ull;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % g.n[0]);
    const long long r = id / g.n[0];
    const int j = (int)(r % g.n[1]);
    const int k = (int)(r / g.n[1]);
    const int c = g.at(i, j, k);
    // the upper face of the last cell of a periodic axis is face 0 (its ghost
    // copy is refreshed only by the next stage's fill)
    const int ux = (i + 1 == g.n[0] && g.periodic[0]) ? c - i : c + 1;
    const int uy = (j + 1 == g.n[1] && g.periodic[1]) ? c - j * g.sy : c + g.sy;
    const double bxl = S.q[5][c], bxr = S.q[5][ux], byl = S.q[6][c], byr = S.q[6][uy];
    double div = (bxr - bxl) * g.idx[0] + (byr - byl) * g.idx[1];
    double bz = S.q[7][c];
    if (NDIM == 3) {
      const int uz = (k + 1 == g.n[2] && g.periodic[2]) ? c - k * g.sz : c + g.sz;
      const double bzr = S.q[7][uz];
      div += (bzr - bz) * g.idx[2];
      bz = 0.5 * (bz + bzr);
    }
    const double bx = 0.5 * (bxl + bxr), by = 0.5 * (byl + byr);
    const double b2 = bx * bx + by * by + bz * bz;
    const float v = (float)(fabs(div) * h);
    const unsigned long long kk = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)id;
    key = kk > key ? kk : key;
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b2);
    b2max = bb > b2max ? bb : b2max;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, b2max, o);
    key = k2 > key ? k2 : key;
    b2max = b2 > b2max ? b2 : b2max;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&sc->divb_key, key);
    atomicMax(&sc->bmax_bits, b2max);
  }
}
static __global__ void divb_finish_kernel(DevScalars* sc, double tol) {
  const unsigned long long key = sc->divb_key;
  const double b2 = __longlong_as_double((long long)sc->bmax_bits);
  const double v = (double)__uint_as_float((unsigned int)(key >> 32));
  const double rel = b2 > 0.0 ? v / sqrt(b2) : v;
  sc->divb_rel = rel;
  if (tol > 0.0 && rel > tol && sc->status == 0) {
    sc->status = -8;  // MHD_ERR_DIVB
    sc->bad_cell = (long long)(key & 0xffffffffull);
  }
  sc->divb_key = 0ull;
  sc->bmax_bits = 0ull;
}

// Set the step size from the host value (mhd_step) and add it to the time.
static __global__ void set_dt_kernel(DevScalars* sc, double dt) {
  sc->dt = dt;
  sc->time = sc->time + dt;
}

// ---------------------------------------------------------------------------
// Sweeps (see sweep_item below)
// ---------------------------------------------------------------------------
template <int RECON> struct Stencil { static constexpr int R = RECON == RECON_PLM ? 1 : 2; };

// Launch bounds of the sweep kernels (128 threads).  Defining
// MHD_SWEEP_MIN_BLOCKS asks the compiler to allow that many resident blocks
// per SM (registers capped at 65536 / (128 * it)); by default the compiler
// chooses (an explicit minimum of 1 changes its register choice).
#ifdef MHD_SWEEP_MIN_BLOCKS
#define MHD_SWEEP_BOUNDS __launch_bounds__(128, MHD_SWEEP_MIN_BLOCKS)
#else
#define MHD_SWEEP_BOUNDS __launch_bounds__(128)
#endif

// The x sweep marches its pencils along the contiguous axis: a warp's 32
// lanes hold 32 rows, so a direct load of one cell per lane touches 32
// sectors.  Instead the warp stages its rows' cells in shared memory, kXChunk
// cells at a time, with loads that cover 8 rows x 32 contiguous bytes each.
// All lanes of a warp then march the same segment in lockstep: the x sweep
// pads its row count to a multiple of 32 (padding lanes load, never store).
constexpr int kXChunk = 4;
constexpr int kXStride = kXChunk + 1;               // row pitch in the stage: no bank conflicts
constexpr int kXStageBuf = 7 * 32 * kXStride;       // doubles per chunk buffer of one warp
constexpr int kXStageWarp = 2 * kXStageBuf;         // double-buffered: the next chunk is in flight
constexpr int kSweepThreads = 128;
constexpr int kXStageBytes = kSweepThreads / 32 * kXStageWarp * (int)sizeof(double);  // per block (dynamic)

// Asynchronous 8-byte global -> shared copies (cp.async, committed in groups).
__device__ __forceinline__ void cp_async8(double* smem_dst, const double* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int DIR, int NDIM>
__host__ __device__ __forceinline__ long long sweep_rows(const Grid& g) {
  constexpr int U = (DIR == 0) ? 1 : 0;
  constexpr int V = (DIR == 0) ? 2 : (DIR == 1 ? 2 : 1);
  long long eu = (U < NDIM) ? g.n[U] + 2 : 1, ev = (V < NDIM) ? g.n[V] + 2 : 1;
  return eu * ev;
}
// The x sweep stages through shared memory when its pencils number at least
// this many (large 3D grids: the padding to whole warps costs < 2 %, and the
// data no longer fits in L2); smaller grids load directly.
constexpr long long kXStageMinRows = 2048;
template <int DIR, int NDIM>
__host__ __device__ __forceinline__ bool sweep_staged(const Grid& g) {
  return DIR == 0 && sweep_rows<DIR, NDIM>(g) >= kXStageMinRows;
}
template <int DIR, int NDIM>
__host__ __device__ __forceinline__ long long sweep_work(const Grid& g, int seglen) {
  long long rows = sweep_rows<DIR, NDIM>(g);
  if (sweep_staged<DIR, NDIM>(g)) rows = (rows + 31) / 32 * 32;
  return rows * ((g.n[DIR] + 1 + seglen - 1) / seglen);
}

// One segment of one pencil.  FETCH(x, v7) delivers the 7 sweep-order
// primitives of cell x of this pencil; it is called with x increasing by one
// from f0 - 1 - R (and identically on every lane of a warp when staged).
template <int DIR, int NDIM, int RECON, int RS, class FETCH>
__device__ __forceinline__ void sweep_body(const Grid& g, const double* __restrict__ Bface, const L6& L,
                                           const FaceIngr& ING, DevScalars* sc, int seglen, int accumulate, int base,
                                           int seg, bool active, bool row_interior, FETCH&& fetch) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int R = Stencil<RECON>::R;
  constexpr int W = 2 * R + 1;  // window of cells
  const int st = g.stride(DIR);
  const int nd = g.n[DIR];
  const int f0 = seg * seglen;
  const int f1 = min(f0 + seglen, nd + 1);  // owned faces [f0, f1)
  const int fend = min(f1, nd);             // last face computed
  const double dt = sc->dt;
  const double dtdx = fmul(dt, g.idx[DIR]);
  double win[7][W];
  // load window centred on cell f0 - 1
#pragma unroll
  for (int m = 0; m < W; m++) {
    double v7[7];
    fetch(f0 - 1 - R + m, v7);
#pragma unroll
    for (int v = 0; v < 7; v++) win[v][m] = v7[v];
  }
  // PLM: the left difference of the window's centre cell, carried along the pencil
  double dl[7];
  if (RECON == RECON_PLM) {
#pragma unroll
    for (int v = 0; v < 7; v++) dl[v] = fsub(win[v][1], win[v][0]);
  }
  // WENO-Z: what consecutive cells share of the indicators (WzCarry)
  WzCarry cv[7];
  if (RECON == RECON_WENOZ) {
#pragma unroll
    for (int v = 0; v < 7; v++) cv[v] = wenoz_start(win[v][0], win[v][1], win[v][2], win[v][3]);
  }
  auto reconstruct = [&](double plus[7], double minus[7], bool count) {
#pragma unroll
    for (int v = 0; v < 7; v++) {
      if (RECON == RECON_PLM) {
        const double dr = fsub(win[v][2], win[v][1]);
        recon_plm_d(win[v][1], dl[v], dr, plus[v], minus[v]);
        dl[v] = dr;
      }
      else if (RECON == RECON_WENOZ) {
        recon_wenoz_m(win[v][0], win[v][1], win[v][2], win[v][3], win[v][4], cv[v], plus[v], minus[v]);
      }
      else recon_ppm(win[v][0], win[v][1], win[v][2], win[v][3], win[v][4], plus[v], minus[v]);
    }
    // positivity fallback: first order in this cell
    if (!gt0(plus[0]) || !gt0(minus[0]) || !gt0(plus[6]) || !gt0(minus[6])) {
#pragma unroll
      for (int v = 0; v < 7; v++) plus[v] = minus[v] = win[v][R];
      if (count) atomicAdd(&sc->fallbacks, 1ull);
    }
  };
  double wl[7], wr[7], dummy[7];
  // cells are counted once: cell -1 by the first segment, cell f by the
  // segment that owns face f
  reconstruct(wl, dummy, active && seg == 0);  // V^L at face f0 (plus state of cell f0-1)
  double Fprev[7];
  for (int f = f0; f <= fend; f++) {
    // shift the window to be centred on cell f
#pragma unroll
    for (int v = 0; v < 7; v++) {
#pragma unroll
      for (int m = 0; m < W - 1; m++) win[v][m] = win[v][m + 1];
    }
    {
      double v7[7];
      fetch(f + R, v7);
#pragma unroll
      for (int v = 0; v < 7; v++) win[v][W - 1] = v7[v];
    }
    double plusN[7];
    reconstruct(plusN, wr, active && f < f1);  // cell f: V^L at f+1, V^R at f
    W7 L7 = {wl[0], wl[1], wl[2], wl[3], wl[4], wl[5], wl[6]};
    W7 R7 = {wr[0], wr[1], wr[2], wr[3], wr[4], wr[5], wr[6]};
    int cf = base + f * st;
    double bn = Bface[cf];
    Flux7 F;
    Ingr ing;
    if (RS != RS_HLL) riemann_hlld<double, RS == RS_HLLD_UCT>(L7, R7, bn, g.gamma, g.igm1, F, ing);
    else riemann_hll(L7, R7, bn, g.gamma, g.igm1, F, ing);
    if (active && f < f1) {
      ING.a[DIR][0][cf] = ing.ap;
      ING.a[DIR][1][cf] = ing.am;
      ING.a[DIR][2][cf] = ing.dd;
      ING.a[DIR][3][cf] = ing.uL;
      ING.a[DIR][4][cf] = ing.uR;
      if (RS == RS_HLLD_UCT) ING.a[DIR][5][cf] = ing.dr;
    }
    if (f > f0 && row_interior) {
      int cc = cf - st;  // cell f-1
      double dv[6];
      dv[0] = fsub(F.f[0], Fprev[0]);
      double dm[3];
      dm[DIR] = fsub(F.f[1], Fprev[1]);
      dm[T1] = fsub(F.f[2], Fprev[2]);
      dm[T2] = fsub(F.f[3], Fprev[3]);
      dv[1] = dm[0];
      dv[2] = dm[1];
      dv[3] = dm[2];
      dv[4] = fsub(F.f[6], Fprev[6]);
      constexpr int NV = NDIM == 2 ? 6 : 5;
      if (NDIM == 2) dv[5] = (DIR == 0) ? fsub(F.f[5], Fprev[5]) : fsub(F.f[4], Fprev[4]);
#pragma unroll
      for (int q = 0; q < NV; q++)  // explicit roundings: the same in every kernel that inlines this
        L.q[q][cc] = accumulate == 2 ? dv[q] : (accumulate ? fma(-dtdx, dv[q], L.q[q][cc]) : fmul(-dtdx, dv[q]));
    }
#pragma unroll
    for (int v = 0; v < 7; v++) {
      Fprev[v] = F.f[v];
      wl[v] = plusN[v];
    }
  }
}

// Direct-load sweep item: every direction, and the x sweep of smaller grids
// (see sweep_item below for what a sweep item does).
template <int DIR, int NDIM, int RECON, int RS>
__device__ __forceinline__ void sweep_item_direct(const Grid& g, const F8& P, const double* __restrict__ Bface, const L6& L,
                                           const FaceIngr& ING, DevScalars* sc, int seglen, int accumulate,
                                           long long id) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  // transverse ranges: fast index u, slow index w
  constexpr int U = (DIR == 0) ? 1 : 0;           // x is the fast index unless sweeping x
  constexpr int V = (DIR == 0) ? 2 : (DIR == 1 ? 2 : 1);
  const int lu = (U < NDIM) ? -1 : 0, hu = (U < NDIM) ? g.n[U] : 0;
  const int lv = (V < NDIM) ? -1 : 0, hv = (V < NDIM) ? g.n[V] : 0;
  const int eu = hu - lu + 1, ev = hv - lv + 1;
  const int nseg = (g.n[DIR] + 1 + seglen - 1) / seglen;
  const long long total = (long long)eu * ev * nseg;
  if (id >= total) return;
  const int iu = (int)(id % eu) + lu;
  const long long r = id / eu;
  const int iv = (int)(r % ev) + lv;
  const int seg = (int)(r / ev);
  int x[3];
  x[DIR] = 0;
  x[U] = iu;
  x[V] = iv;
  const bool row_interior = (U >= NDIM || (iu >= 0 && iu < g.n[U])) && (V >= NDIM || (iv >= 0 && iv < g.n[V]));
  const int base = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  // primitive slots in sweep order: rho, v_n, v_t1, v_t2, B_t1, B_t2, p
  const double* pr[7] = {P.q[0], P.q[1 + DIR], P.q[1 + T1], P.q[1 + T2], P.q[4 + T1], P.q[4 + T2], P.q[7]};
  auto fetch = [&](int xi, double v7[7]) {
    const int c = base + xi * st;
#pragma unroll
    for (int v = 0; v < 7; v++) v7[v] = pr[v][c];
  };
  sweep_body<DIR, NDIM, RECON, RS>(g, Bface, L, ING, sc, seglen, accumulate, base, seg, true, row_interior, fetch);
}

// Staged x-sweep item (grids for which sweep_staged holds): the warp's 32
// lanes march 32 pencils of one segment in lockstep; `stage` is this warp's
// shared-memory stage of kXStageWarp doubles (two chunk buffers).
template <int NDIM, int RECON, int RS>
__device__ __forceinline__ void sweep_item_staged(const Grid& g, const F8& P, const double* __restrict__ Bface,
                                                  const L6& L, const FaceIngr& ING, DevScalars* sc, int seglen,
                                                  int accumulate, long long id, double* stage) {
  constexpr int DIR = 0, T1 = 1, T2 = 2;
  const int lu = -1, lv = NDIM == 3 ? -1 : 0;
  const int eu = g.n[1] + 2;
  const long long rows = sweep_rows<DIR, NDIM>(g);
  const long long prow = (rows + 31) / 32 * 32;  // whole warps per segment
  if (id >= prow * ((g.n[DIR] + 1 + seglen - 1) / seglen)) return;  // whole warps
  long long row = id % prow;
  const int seg = (int)(id / prow);
  const bool active = row < rows;  // padding lanes load and march but never store
  if (!active) row = 0;
  const int iu = (int)(row % eu) + lu;
  const int iv = (int)(row / eu) + lv;
  const bool row_interior = active && iu >= 0 && iu < g.n[1] && (NDIM == 2 || (iv >= 0 && iv < g.n[2]));
  const int base = g.at(0, iu, iv);
  const double* pr[7] = {P.q[0], P.q[1 + DIR], P.q[1 + T1], P.q[1 + T2], P.q[4 + T1], P.q[4 + T2], P.q[7]};
  const int lane = threadIdx.x & 31;
  // lane's share of a chunk copy: element k*32 + lane is row (k*32+lane)/kXChunk, cell (k*32+lane)%kXChunk
  int rbase[kXChunk];
#pragma unroll
  for (int k = 0; k < kXChunk; k++) rbase[k] = __shfl_sync(0xffffffffu, base, (k * 32 + lane) / kXChunk);
  const int cix = lane % kXChunk;
  auto issue = [&](int x0, double* buf) {  // the warp's rows, cells [x0, x0 + kXChunk), all 7 primitives
#pragma unroll
    for (int k = 0; k < kXChunk; k++) {
      const int r = (k * 32 + lane) / kXChunk;
#pragma unroll
      for (int v = 0; v < 7; v++) cp_async8(buf + (v * 32 + r) * kXStride + cix, pr[v] + rbase[k] + x0 + cix);
    }
    cp_async_commit();
  };
  // Cells are requested in increasing order from f0 - 1 - R (the same on every
  // lane, so every branch below is warp-uniform).  Two chunks are in flight
  // ahead of the one being read; reads past the pencil end land in the next
  // padded row of the same field.
  int xc = (seg * seglen) - 1 - Stencil<RECON>::R;
  int cur = 0;
  issue(xc, stage);
  issue(xc + kXChunk, stage + kXStageBuf);
  cp_async_wait_all_but_one();
  __syncwarp();
  auto fetch = [&](int xi, double v7[7]) {
    if (xi >= xc + kXChunk) {
      __syncwarp();                                    // every lane is done with buffer cur
      issue(xc + 2 * kXChunk, stage + cur * kXStageBuf);
      xc += kXChunk;
      cur ^= 1;
      cp_async_wait_all_but_one();                     // the chunk at xc has landed
      __syncwarp();
    }
    const double* buf = stage + cur * kXStageBuf;
#pragma unroll
    for (int v = 0; v < 7; v++) v7[v] = buf[(v * 32 + lane) * kXStride + (xi - xc)];
  };
  sweep_body<DIR, NDIM, RECON, RS>(g, Bface, L, ING, sc, seglen, accumulate, base, seg, active, row_interior, fetch);
  cp_async_wait_all();  // no copy may still target this block's shared memory when it exits
}

// ---------------------------------------------------------------------------
// Sweep along DIR: each thread marches a segment of faces of one pencil,
// reconstructing each cell once, solving each face's Riemann problem once per
// segment, writing the face's UCT ingredients and accumulating the flux
// difference of Eq. FV into the stage increment of the cells it owns.
// Pencils cover transverse indices [-1, n_t] on active axes (the outer layer
// feeds the edge fields only).  The direct and staged items execute the
// same arithmetic (sweep_body repeats sweep_item_direct's), so their results
// agree to the bit.
// ---------------------------------------------------------------------------
template <int DIR, int NDIM, int RECON, int RS, bool STAGED = false>
static __global__ void MHD_SWEEP_BOUNDS
    sweep_kernel(Grid g, F8 P, const double* __restrict__ Bface, L6 L, FaceIngr ING, DevScalars* sc, int seglen,
                 int accumulate) {
  if constexpr (STAGED) {
    static_assert(DIR == 0, "only the x sweep stages");
    extern __shared__ double stage[];  // kXStageBytes, dynamic
    sweep_item_staged<NDIM, RECON, RS>(g, P, Bface, L, ING, sc, seglen, accumulate,
                                       blockIdx.x * (long long)blockDim.x + threadIdx.x,
                                       stage + (threadIdx.x >> 5) * kXStageWarp);
  } else {
    sweep_item_direct<DIR, NDIM, RECON, RS>(g, P, Bface, L, ING, sc, seglen, accumulate,
                                            blockIdx.x * (long long)blockDim.x + threadIdx.x);
  }
}

// ---------------------------------------------------------------------------
// UCT edge fields (reading of the UCT-HLL average):
//   E_c = -(a+_a u^W B_b^W + a-_a u^E B_b^E) + d_a (B_b^E - B_b^W)
//         + (a+_b u^S B_a^S + a-_b u^N B_a^N) - d_b (B_a^N - B_a^S)
// with the a-face ingredients averaged over the two a-faces touching the edge
// and minmod reconstructions of the face fields to the edge.  UCT-HLLD
// (HLLD = true): the same form with the HLLD weights a^L, a^R and separate
// d^L, d^R, i.e. the dissipation terms (d^R_a B_b^E - d^L_a B_b^W) and
// -(d^R_b B_a^N - d^L_b B_a^S).
// ---------------------------------------------------------------------------
// The averages of two face values carry a factor 1/2 each; it is folded into
// the sums as exact power-of-two scalings: a+ u^W = (1/4)(a1 + a2)(u1 + u2).
template <int C, bool HLLD = false>
__device__ __forceinline__ double uct_edge(const Grid& g, const F8& S, const FaceIngr& ING, int c) {
  constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
  const int sa = g.stride(A), sb = g.stride(B);
  const int cb = c - sb, ca = c - sa;
  const double* Ia[5] = {ING.a[A][0], ING.a[A][1], ING.a[A][2], ING.a[A][3], ING.a[A][4]};
  const double* Ib[5] = {ING.a[B][0], ING.a[B][1], ING.a[B][2], ING.a[B][3], ING.a[B][4]};
  auto add = [](double x, double y) { return fadd(x, y); };
  auto sub = [](double x, double y) { return fsub(x, y); };
  auto mul = [](double x, double y) { return fmul(x, y); };
  // sums over the two a-faces (b-faces) touching the edge
  double apa = add(Ia[0][cb], Ia[0][c]), ama = add(Ia[1][cb], Ia[1][c]), dda = add(Ia[2][cb], Ia[2][c]);
  double uW = add(Ia[3][cb], Ia[3][c]), uE = add(Ia[4][cb], Ia[4][c]);
  double apb = add(Ib[0][ca], Ib[0][c]), amb = add(Ib[1][ca], Ib[1][c]), ddb = add(Ib[2][ca], Ib[2][c]);
  double vS = add(Ib[3][ca], Ib[3][c]), vN = add(Ib[4][ca], Ib[4][c]);
  const double* Bb = S.q[5 + B];
  const double* Ba = S.q[5 + A];
  // B_b along a: values at a-cells -2, -1, 0, +1 relative to the edge
  double bm2 = Bb[c - 2 * sa], bm1 = Bb[c - sa], b0 = Bb[c], bp1 = Bb[c + sa];
  double dbm = sub(bm1, bm2), db0 = sub(b0, bm1), dbp = sub(bp1, b0);
  double BbW = fma(rk(RK_HALF), minmod(dbm, db0), bm1);
  double BbE = fma(rk(RK_MHALF), minmod(db0, dbp), b0);
  double am2 = Ba[c - 2 * sb], am1 = Ba[c - sb], a0 = Ba[c], ap1 = Ba[c + sb];
  double dam = sub(am1, am2), da0 = sub(a0, am1), dap = sub(ap1, a0);
  double BaS = fma(rk(RK_HALF), minmod(dam, da0), am1);
  double BaN = fma(rk(RK_MHALF), minmod(da0, dap), a0);
  // 4 E = -(A+a uW BbW + A-a uE BbE) + (A+b vS BaS + A-b vN BaN) + 2 (Da (BbE-BbW) - Db (BaN-BaS))
  double up = sub(fma(mul(apb, vS), BaS, mul(mul(amb, vN), BaN)), fma(mul(apa, uW), BbW, mul(mul(ama, uE), BbE)));
  double diss;
  if (HLLD) {
    const double dra = add(ING.a[A][5][cb], ING.a[A][5][c]), drb = add(ING.a[B][5][ca], ING.a[B][5][c]);
    diss = sub(fma(dra, BbE, -mul(dda, BbW)), fma(drb, BaN, -mul(ddb, BaS)));
  } else {
    diss = fma(dda, sub(BbE, BbW), -mul(ddb, sub(BaN, BaS)));
  }
  return fma(rk(RK_QUARTER), up, mul(rk(RK_HALF), diss));
}

template <int NDIM>
__host__ __device__ __forceinline__ long long edge_work(const Grid& g) {
  return (long long)(g.n[0] + 1) * (g.n[1] + 1) * (NDIM == 3 ? g.n[2] + 1 : 1);
}
template <int NDIM, bool HLLD = false>
__device__ __forceinline__ void emf_item(const Grid& g, const F8& S, const FaceIngr& ING, const E3& E, long long id) {
  const int ex = g.n[0] + 1, ey = g.n[1] + 1;
  int i = (int)(id % ex);
  long long r = id / ex;
  int j = (int)(r % ey);
  int k = (int)(r / ey);
  int c = g.at(i, j, k);
  if (NDIM == 2) {
    E.e[2][c] = uct_edge<2, HLLD>(g, S, ING, c);
  } else {
    if (k < g.n[2]) E.e[2][c] = uct_edge<2, HLLD>(g, S, ING, c);  // E_z at (x-face i, y-face j, cell k)
    if (i < g.n[0]) E.e[0][c] = uct_edge<0, HLLD>(g, S, ING, c);  // E_x at (cell i, y-face j, z-face k)
    if (j < g.n[1]) E.e[1][c] = uct_edge<1, HLLD>(g, S, ING, c);  // E_y at (x-face i, cell j, z-face k)
  }
}
template <int NDIM, bool HLLD>
static __global__ void __launch_bounds__(256) emf_kernel(Grid g, F8 S, FaceIngr ING, E3 E) {
  const long long total = edge_work<NDIM>(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    emf_item<NDIM, HLLD>(g, S, ING, E, id);
}

// ---------------------------------------------------------------------------
// CT face increment L_B = -dt curl E and the RK stage combine of every
// evolved cell and face:  out = a0*U0 + a1*Us + aL*L  in the fixed forms
//   stage "first":   Us + L
//   RK2 final:       (U0 + Us + L) / 2
//   RK3 second:      (3 U0 + Us + L) / 4
//   RK3 final:       (U0 + 2 Us + 2 L) / 3
// ---------------------------------------------------------------------------
enum { COMB_FIRST = 0, COMB_RK2_FINAL = 1, COMB_RK3_SECOND = 2, COMB_RK3_FINAL = 3 };

// Plain arithmetic here: the CT + RK kernel is bound by memory, where loading
// the register constants of the DFMA forms would cost more than it saves.
__device__ __forceinline__ double combine(int mode, double u0, double us, double l) {
  switch (mode) {
    case COMB_FIRST: return us + l;
    case COMB_RK2_FINAL: return 0.5 * ((u0 + us) + l);
    case COMB_RK3_SECOND: return 0.25 * (fma(3.0, u0, us) + l);
    default: return fma(2.0, l, fma(2.0, us, u0)) * (1.0 / 3.0);
  }
}

// SPLIT: the y (and z) sweeps ran beside the x sweep and left their raw flux
// differences in Dy (Dz); the stage increment is completed here exactly as the
// sequential sweeps accumulate it, L = fma(-dt/dz, Dz, fma(-dt/dy, Dy, L_x)).
template <int NDIM, bool SPLIT = false>
__device__ __forceinline__ void ct_rk_item(const Grid& g, const F8& U0, const F8& Us, const F8& Out, const L6& L,
                                           const E3& E, double dt, int mode, long long id, const L6* Dy = nullptr,
                                           const L6* Dz = nullptr) {
  const int ex = g.n[0] + 1, ey = g.n[1] + 1;
  int i = (int)(id % ex);
  long long r = id / ex;
  int j = (int)(r % ey);
  int k = (int)(r / ey);
  int c = g.at(i, j, k);
  const bool in_x = i < g.n[0], in_y = j < g.n[1], in_z = k < g.n[2];
  if (in_x && in_y && in_z) {
    constexpr int NV = NDIM == 2 ? 6 : 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
      int slot = q < 5 ? q : 7;
      double l = L.q[q][c];
      if (SPLIT) {
        l = fma(-(dt * g.idx[1]), Dy->q[q][c], l);
        if (NDIM == 3) l = fma(-(dt * g.idx[2]), Dz->q[q][c], l);
      }
      Out.q[slot][c] = combine(mode, U0.q[slot][c], Us.q[slot][c], l);
    }
  }
  // faces with normal d: evolved for d-index < n_d, or == n_d on an outflow axis
#pragma unroll
  for (int d = 0; d < NDIM; d++) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    int idx3[3] = {i, j, k};
    bool ok = true;
#pragma unroll
    for (int e = 0; e < NDIM; e++) {
      if (e == d) ok = ok && (idx3[e] < g.n[e] || !g.periodic[e]);
      else ok = ok && idx3[e] < g.n[e];
    }
    if (NDIM == 2) ok = ok && k == 0;
    if (!ok) continue;
    const bool has1 = d1 < NDIM, has2 = d2 < NDIM;
    double t1 = 0.0, t2 = 0.0;
    if (has1) t1 = __dmul_rn(E.e[d2][c + g.stride(d1)] - E.e[d2][c], dt * g.idx[d1]);
    if (has2) t2 = __dmul_rn(E.e[d1][c + g.stride(d2)] - E.e[d1][c], dt * g.idx[d2]);
    double lb = (has1 && has2) ? t2 - t1 : (has1 ? -t1 : t2);
    Out.q[5 + d][c] = combine(mode, U0.q[5 + d][c], Us.q[5 + d][c], lb);
  }
}
template <int NDIM>
static __global__ void __launch_bounds__(256) ct_rk_kernel(Grid g, F8 U0, F8 Us, F8 Out, L6 L, E3 E,
                                                    const DevScalars* sc, int mode) {
  const long long total = edge_work<NDIM>(g);
  const double dt = sc->dt;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ct_rk_item<NDIM>(g, U0, Us, Out, L, E, dt, mode, id);
}
template <int NDIM>
static __global__ void __launch_bounds__(256) ct_rk_split_kernel(Grid g, F8 U0, F8 Us, F8 Out, L6 L, L6 Dy, L6 Dz,
                                                          E3 E, const DevScalars* sc, int mode) {
  const long long total = edge_work<NDIM>(g);
  const double dt = sc->dt;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ct_rk_item<NDIM, true>(g, U0, Us, Out, L, E, dt, mode, id, &Dy, &Dz);
}

// ---------------------------------------------------------------------------
// State import / export helpers
// ---------------------------------------------------------------------------
// Primitive -> conserved in place on interior cells (slots 0..4 hold
// rho, vx, vy, vz, p on entry); faces (and 2D cell Bz) already set.
template <int NDIM>
static __global__ void prim_to_cons_kernel(Grid g, F8 S) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int i = (int)(id % g.n[0]);
    long long r = id / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    int c = g.at(i, j, k);
    double bx = 0.5 * (S.q[5][c] + S.q[5][c + 1]);
    double by = 0.5 * (S.q[6][c] + S.q[6][c + g.sy]);
    double bz = NDIM == 3 ? 0.5 * (S.q[7][c] + S.q[7][c + g.sz]) : S.q[7][c];
    double rho = S.q[0][c], vx = S.q[1][c], vy = S.q[2][c], vz = S.q[3][c], p = S.q[4][c];
    S.q[1][c] = rho * vx;
    S.q[2][c] = rho * vy;
    S.q[3][c] = rho * vz;
    S.q[4][c] = p * g.igm1 + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz);
  }
}

// ---------------------------------------------------------------------------
// Batched kernels: one launch advances a stage piece of many independent
// grids (an ensemble).  Each block belongs to exactly one run: run r owns the
// blocks [blk0[r], blk0[r+1]) of the launch, so a run's CFL reduction stays in
// its own blocks and no warp mixes runs.  Every run executes the same item
// bodies as the single-grid kernels, hence the same arithmetic.
// ---------------------------------------------------------------------------
struct RunDev {
  Grid g;
  F8 U[3];        // RK registers
  F8 P;           // primitives
  L6 L;           // stage increment
  FaceIngr ING;    // UCT face ingredients
  E3 E;           // edge fields
  DevScalars* sc;
  int seglen;     // sweep segment length of this run
};

// largest r with blk0[r] <= blockIdx.x
__device__ __forceinline__ int block_run(const int* __restrict__ blk0, int nruns) {
  int lo = 0, hi = nruns - 1;
  const int b = (int)blockIdx.x;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(blk0 + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ long long block_local_id(const int* __restrict__ blk0, int r) {
  return (long long)((int)blockIdx.x - __ldg(blk0 + r)) * blockDim.x + threadIdx.x;
}

static __global__ void __launch_bounds__(256) batch_ghost_periodic_kernel(const RunDev* __restrict__ runs,
                                                                   const int* __restrict__ blk0, int nruns, int d,
                                                                   int reg) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  const long long id = block_local_id(blk0, r);
  if (id < ghost_layers_work(R.g, d)) ghost_periodic_item(R.g, R.U[reg], d, id);
}
static __global__ void __launch_bounds__(256) batch_ghost_outflow_copy_kernel(const RunDev* __restrict__ runs,
                                                                       const int* __restrict__ blk0, int nruns, int d,
                                                                       int reg) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  const long long id = block_local_id(blk0, r);
  if (id < ghost_layers_work(R.g, d)) ghost_outflow_copy_item(R.g, R.U[reg], d, id);
}
static __global__ void __launch_bounds__(256) batch_ghost_outflow_normal_kernel(const RunDev* __restrict__ runs,
                                                                         const int* __restrict__ blk0, int nruns,
                                                                         int d, int reg) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  const long long id = block_local_id(blk0, r);
  if (id < ghost_rows_work(R.g, d)) ghost_outflow_normal_item(R.g, R.U[reg], d, id);
}
template <int NDIM, bool CFL>
static __global__ void __launch_bounds__(256) batch_prim_kernel(const RunDev* __restrict__ runs,
                                                         const int* __restrict__ blk0, int nruns, int reg) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  const long long id = block_local_id(blk0, r);
  double lam = 0.0;
  if (id < prim_work<NDIM>(R.g)) lam = prim_item<NDIM, CFL, !CFL>(R.g, R.U[reg], R.P, R.sc, id);
  if (CFL) cfl_block_finish(lam, R.sc, R.g.cfl, (unsigned int)(__ldg(blk0 + r + 1) - __ldg(blk0 + r)));
}
// Batched sweeps load directly (the ensemble's grids are small); a run whose
// x sweep would be staged is served by the same direct path here.
template <int DIR, int NDIM, int RECON, int RS>
static __global__ void MHD_SWEEP_BOUNDS
    batch_sweep_kernel(const RunDev* __restrict__ runs, const int* __restrict__ blk0, int nruns, int reg,
                       int accumulate) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  sweep_item_direct<DIR, NDIM, RECON, RS>(R.g, R.P, R.U[reg].q[5 + DIR], R.L, R.ING, R.sc, R.seglen, accumulate,
                                          block_local_id(blk0, r));
}
template <int NDIM, bool HLLD>
static __global__ void __launch_bounds__(256) batch_emf_kernel(const RunDev* __restrict__ runs,
                                                        const int* __restrict__ blk0, int nruns, int reg) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  const long long id = block_local_id(blk0, r);
  if (id < edge_work<NDIM>(R.g)) emf_item<NDIM, HLLD>(R.g, R.U[reg], R.ING, R.E, id);
}
template <int NDIM>
static __global__ void __launch_bounds__(256) batch_ct_rk_kernel(const RunDev* __restrict__ runs,
                                                          const int* __restrict__ blk0, int nruns, int reg_s,
                                                          int reg_out, int mode) {
  const int r = block_run(blk0, nruns);
  const RunDev& R = runs[r];
  const long long id = block_local_id(blk0, r);
  if (id < edge_work<NDIM>(R.g)) ct_rk_item<NDIM>(R.g, R.U[0], R.U[reg_s], R.U[reg_out], R.L, R.E, R.sc->dt, mode, id);
}

}  // namespace mhd
