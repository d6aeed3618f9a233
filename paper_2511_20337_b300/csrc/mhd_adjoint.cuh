// Reverse-mode (adjoint) kernels of one CT stage (paper §2.2) for PLM
// reconstruction on periodic grids.  Given the cotangent of a stage's output,
// they form the cotangent of its input state, transposing each forward kernel
// of mhd_kernels.cuh in turn:
//
//   combine (RK weights)  ->  curl of the edge fields (CT face update)
//   ->  UCT edge fields   ->  Riemann solver + flux difference (per face)
//   ->  PLM reconstruction (per cell)  ->  primitive recovery  ->  ghost fill
//
// Every transpose is written in gather form (each output element is summed by
// one thread in a fixed order), so no atomics are needed and the adjoint is
// deterministic.  Branches (minmod choices, positivity fallbacks, wave-fan
// regions, min/max) are those the forward values take; where an argument of
// minmod is exactly zero the derivative of minmod is taken as zero.  The
// Riemann solver's vector-Jacobian product comes from the templated solvers
// of mhd_math.cuh instantiated with the multi-tangent number D3: the exact
// derivative of the same operations the forward executes.
#pragma once
#include "mhd_kernels.cuh"
#include "mhd_dual.cuh"
#include "mhd_riemann_adj.cuh"

namespace mhd {

struct L3 { double* q[3]; };              // face arrays, one per normal direction
struct GE20 { double* q[3][20]; };        // per edge component: 20 edge-local cotangents

// Edge component C exists in the forward step: all three in 3D, E_z in 2D.
template <int NDIM> __device__ __forceinline__ bool has_edge(int C) { return NDIM == 3 || C == 2; }

// (i,j,k) is an edge of component C computed by the forward step (emf_item).
template <int NDIM>
__device__ __forceinline__ bool edge_valid(const Grid& g, int C, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i > g.n[0] || j > g.n[1]) return false;
  if (NDIM == 2) return C == 2 && k == 0;
  if (k > g.n[2]) return false;
  return C == 0 ? i < g.n[0] : (C == 1 ? j < g.n[1] : k < g.n[2]);
}

// Which argument minmod(a, b) passes on, for its derivative: 1 = a, 2 = b,
// 0 = neither (opposite signs or a zero argument, where the value is 0).
__device__ __forceinline__ int minmod_pick(double a, double b) {
  if (!((gt0(a) && gt0(b)) || (lt0(a) && lt0(b)))) return 0;
  return bits(b) < bits(a) ? 2 : 1;  // same signs: the bits order like the magnitudes (see minmod)
}

__device__ __forceinline__ void box_index(long long id, const int lo[3], const int ext[3], int x[3]) {
  x[0] = (int)(id % ext[0]) + lo[0];
  long long r = id / ext[0];
  x[1] = (int)(r % ext[1]) + lo[1];
  x[2] = (int)(r / ext[1]) + lo[2];
}

// ---------------------------------------------------------------------------
// Seed: cotangent of J with respect to the final state (ghost-filled S) and
// the per-cell terms of J.
//   magnetic energy: J = 1/2 dV sum_c |B_c|^2, B_c the mean of the two faces
//   misfit:          J = 1/2 dV sum_c sum_q (U_q - T_q)^2 over rho, m, E
//                    (2D: and the cell B_z)
// Written over the box of faces [0, n_d] (cells [0, n_d - 1]); the face at
// n_d of a periodic axis is the ghost copy of face 0 and is folded back by
// the ghost transpose.
// ---------------------------------------------------------------------------
enum { FUNC_MAGNETIC_ENERGY = 0, FUNC_MISFIT = 1 };

template <int NDIM>
__device__ __forceinline__ double cell_b(const Grid& g, const F8& S, int d, int c) {
  if (NDIM == 2 && d == 2) return S.q[7][c];
  return 0.5 * (S.q[5 + d][c] + S.q[5 + d][c + g.stride(d)]);
}

template <int NDIM>
static __global__ void adj_seed_kernel(Grid g, F8 S, F8 A, int which, L6 T, double dV, double* Jcell) {
  const long long total = edge_work<NDIM>(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int ex = g.n[0] + 1, ey = g.n[1] + 1;
    int i = (int)(id % ex);
    long long r = id / ex;
    int j = (int)(r % ey);
    int k = (int)(r / ey);
    const int x[3] = {i, j, k};
    const int c = g.at(i, j, k);
    const bool cell = i < g.n[0] && j < g.n[1] && k < g.n[2];
    if (cell) {
      double sum = 0.0;
      if (which == FUNC_MAGNETIC_ENERGY) {
        double bx = cell_b<NDIM>(g, S, 0, c), by = cell_b<NDIM>(g, S, 1, c), bz = cell_b<NDIM>(g, S, 2, c);
        sum = (bx * bx + by * by) + bz * bz;
        if (NDIM == 2) A.q[7][c] = dV * bz;
      } else {
        constexpr int NQ = NDIM == 2 ? 6 : 5;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
          int slot = q < 5 ? q : 7;
          double dq = S.q[slot][c] - T.q[q][c];
          sum = q == 0 ? dq * dq : sum + dq * dq;
          A.q[slot][c] = dV * dq;
        }
      }
      Jcell[((long long)k * g.n[1] + j) * g.n[0] + i] = sum;
    }
    if (which == FUNC_MAGNETIC_ENERGY) {
#pragma unroll
      for (int d = 0; d < NDIM; d++) {
        bool ok = true;
#pragma unroll
        for (int e = 0; e < NDIM; e++)
          if (e != d && x[e] >= g.n[e]) ok = false;
        if (!ok) continue;
        double acc = 0.0;
        if (x[d] < g.n[d]) acc += cell_b<NDIM>(g, S, d, c);
        if (x[d] > 0) acc += cell_b<NDIM>(g, S, d, c - g.stride(d));
        A.q[5 + d][c] = 0.5 * dV * acc;
      }
    }
  }
}

// Fixed-order sum of n values by one block (deterministic).
static __global__ void adj_sum_kernel(const double* __restrict__ v, long long n, double scale, double* out) {
  __shared__ double part[1024];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * part[0];
}

// ---------------------------------------------------------------------------
// Transpose of the periodic ghost fill: every ghost slot's cotangent is added
// to the interior slot it was copied from, then cleared.  The forward fills
// x, y, z in turn (each pass over the full padded transverse range), so the
// transposes run z, y, x.
// ---------------------------------------------------------------------------

// All axes' transposes in one pass: every ghost slot of a periodic axis wraps
// to exactly one interior cell, so the thread of that cell gathers its images
// and clears them.  The sums keep the order of the axis-by-axis passes (z, y,
// x): with Z = A + A(z image), Y = Z + Z(y image), the cell gets
// Y + Y(x image), each term present only where the image exists (for
// n_d >= 2G + 1 a cell has at most one image per axis).
template <int NDIM>
__device__ __forceinline__ void adj_ghost_shell_item(const Grid& g, const F8& A, long long id) {
  {
    const int i = (int)(id % g.n[0]);
    const long long r = id / g.n[0];
    const int j = (int)(r % g.n[1]);
    const int k = (int)(r / g.n[1]);
    // the image along axis d of interior index x (or the index itself when there is none)
    auto image = [&](int d, int x) {
      if (d >= NDIM) return x;
      if (x <= g.G) return x + g.n[d];            // upper ghost layer n_d + x (up to the extra slot n_d + G)
      if (x >= g.n[d] - g.G) return x - g.n[d];   // lower ghost layer
      return x;
    };
    const int ix = image(0, i), jy = image(1, j), kz = image(2, k);
    const bool hx = ix != i, hy = jy != j, hz = kz != k;
    if (!hx && !hy && !hz) return;
    const int ci[2] = {i, ix}, cj[2] = {j, jy}, ck[2] = {k, kz};
    // every value first, then the sums and stores: each slot is read once and
    // written after all reads, so the loads of all fields are in flight
    // together instead of one field's chain after another's
    double val[8][4][2];
#pragma unroll
    for (int q = 0; q < 8; q++)
#pragma unroll
      for (int u = 0; u < 2; u++)
#pragma unroll
        for (int v = 0; v < 2; v++) {
          if ((u == 1 && !hx) || (v == 1 && !hy)) continue;
          val[q][2 * u + v][0] = A.q[q][g.at(ci[u], cj[v], k)];
          if (hz) val[q][2 * u + v][1] = A.q[q][g.at(ci[u], cj[v], ck[1])];
        }
#pragma unroll
    for (int q = 0; q < 8; q++) {
      double* a = A.q[q];
      double xs[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {  // the cell's column and its x image
        if (u == 1 && !hx) continue;
        double ys[2];
#pragma unroll
        for (int v = 0; v < 2; v++) {  // the row and its y image
          if (v == 1 && !hy) continue;
          double z = val[q][2 * u + v][0];
          if (hz) {
            z += val[q][2 * u + v][1];
            a[g.at(ci[u], cj[v], ck[1])] = 0.0;
          }
          if (u == 1 || v == 1) a[g.at(ci[u], cj[v], k)] = 0.0;
          ys[v] = z;
        }
        xs[u] = hy ? ys[0] + ys[1] : ys[0];
      }
      a[g.at(i, j, k)] = hx ? xs[0] + xs[1] : xs[0];
    }
  }
}
template <int NDIM>
static __global__ void adj_ghost_shell_kernel(Grid g, F8 A) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    adj_ghost_shell_item<NDIM>(g, A, id);
}

// ---------------------------------------------------------------------------
// Transposes of the per-axis ghost passes (grids with an outflow axis).  The
// forward fills the periodic axes first, then each outflow axis with its copy
// pass and its normal-field pass, every pass over the full padded transverse
// range; the transposes run in the reverse order.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ long long pass_rows(const Grid& g, int d) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  return (long long)(g.hi(t1) - g.lo(t1) + 1) * (g.hi(t2) - g.lo(t2) + 1);
}
__device__ __forceinline__ void pass_row(const Grid& g, int d, long long r, int x[3]) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const int e1 = g.hi(t1) - g.lo(t1) + 1;
  x[t1] = (int)(r % e1) + g.lo(t1);
  x[t2] = (int)(r / e1) + g.lo(t2);
}

// Periodic pass along d: each interior slot x gathers its image x - n
// (x >= n - G) or x + n (x <= G) and clears it (n >= 2G + 1: one image at most).
static __global__ void adj_ghost_periodic_kernel(Grid g, F8 A, int d) {
  const int n = g.n[d];
  const long long total = pass_rows(g, d) * n;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int y[3];
    y[d] = (int)(id % n);
    pass_row(g, d, id / n, y);
    const int x = y[d];
    int img;
    if (x >= n - g.G) img = x - n;
    else if (x <= g.G) img = x + n;
    else continue;
    const int c = g.at(y[0], y[1], y[2]);
    y[d] = img;
    const int ci = g.at(y[0], y[1], y[2]);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      A.q[q][c] += A.q[q][ci];
      A.q[q][ci] = 0.0;
    }
  }
}

// Outflow copy pass along d: the boundary cell gathers the G copies on its
// side (G + 1 slots on the high side, the last one the extra face slot) of
// every slot but the normal face field, and clears them.
static __global__ void adj_ghost_outflow_copy_kernel(Grid g, F8 A, int d) {
  const int n = g.n[d];
  const long long total = pass_rows(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int y[3];
    pass_row(g, d, id, y);
    auto at = [&](int x) {
      y[d] = x;
      return g.at(y[0], y[1], y[2]);
    };
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (q == 5 + d) continue;
      double* a = A.q[q];
      double s = a[at(0)];
      for (int x = -g.G; x < 0; x++) {
        s += a[at(x)];
        a[at(x)] = 0.0;
      }
      a[at(0)] = s;
      s = a[at(n - 1)];
      for (int x = n; x <= n + g.G; x++) {
        s += a[at(x)];
        a[at(x)] = 0.0;
      }
      a[at(n - 1)] = s;
    }
  }
}

// Outflow normal-field pass along d, part 1, per row of the pass: the forward
// marches B_n[-m] = B_n[-m + 1] + dx_d divT(-m) (m = 1..G) and
// B_n[n + m + 1] = B_n[n + m] - dx_d divT(n + m) (m = 0..G-1), divT the
// tangential divergence of the ghost cell.  Walking each march back, the
// cotangent of a ghost face, with those of the faces beyond it, passes to the
// face inside it; H keeps each ghost face's total (the factor of its divT)
// and the ghost faces' own cotangents are cleared.
static __global__ void adj_ghost_outflow_chain_kernel(Grid g, F8 A, int d, double* H) {
  const int n = g.n[d];
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const int e1 = g.hi(t1) - g.lo(t1) + (t1 < g.ndim ? 0 : 1);
  const long long total = ghost_rows_work(g, d);
  double* An = A.q[5 + d];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int y[3];
    y[t1] = (int)(id % e1) + g.lo(t1);
    y[t2] = (int)(id / e1) + g.lo(t2);
    auto at = [&](int x) {
      y[d] = x;
      return g.at(y[0], y[1], y[2]);
    };
    double s = 0.0;
    for (int m = g.G; m >= 1; m--) {
      const int f = at(-m);
      s += An[f];
      An[f] = 0.0;
      H[f] = s;
    }
    An[at(0)] += s;
    s = 0.0;
    for (int m = g.G - 1; m >= 0; m--) {
      const int f = at(n + m + 1);
      s += An[f];
      An[f] = 0.0;
      H[f] = s;
    }
    An[at(n)] += s;
  }
}

// Part 2, per tangential face of the ghost cells (layer l: cells -1..-G, then
// n..n+G-1): divT(cell) of row r holds (B_t[r + 1] - B_t[r]) / dx_t, so face f
// of axis t gets +k H from row f - 1 and -k H from row f, k = +-dx_d / dx_t
// (minus on the high side), H the row's factor from part 1.
__host__ __device__ __forceinline__ long long adj_outflow_faces_work(const Grid& g, int d) {
  return 2LL * g.G * pass_rows(g, d);
}
static __global__ void adj_ghost_outflow_faces_kernel(Grid g, F8 A, int d, const double* __restrict__ H) {
  const int n = g.n[d];
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const long long total = adj_outflow_faces_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(id % (2 * g.G));
    int p[3];
    pass_row(g, d, id / (2 * g.G), p);
    const bool low = l < g.G;
    const int cell = low ? -(l + 1) : n + (l - g.G);
    const int hslot = low ? cell : cell + 1;  // the row's ghost face: B_n[-m] or B_n[n + m + 1]
    const int ts[2] = {t1, t2};
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const int t = ts[k], u = ts[1 - k];
      if (t >= g.ndim) continue;
      if (u < g.ndim && p[u] > g.hi(u) - 1) continue;  // not a row of the pass across u
      const int f = p[t];
      const double coef = (low ? g.dx[d] : -g.dx[d]) / g.dx[t];
      int y[3];
      y[d] = hslot;
      y[u] = p[u];
      double acc = 0.0;
      if (f - 1 >= g.lo(t)) {
        y[t] = f - 1;
        acc += coef * H[g.at(y[0], y[1], y[2])];
      }
      if (f <= g.hi(t) - 1) {
        y[t] = f;
        acc -= coef * H[g.at(y[0], y[1], y[2])];
      }
      y[d] = cell;
      y[t] = f;
      A.q[5 + t][g.at(y[0], y[1], y[2])] += acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Transpose of the stage combine  out = c0 U0 + c1 Us + cL L  (cells), and
// out_B = c0 B0 + c1 Bs + cL L_B (evolved faces): the cotangents of the stage
// increment (Lb on cells, LB on faces) and the accumulation into U0 and Us.
// ---------------------------------------------------------------------------
// Face (normal d) at index x evolved by the CT update on a periodic grid: the
// faces the combine transpose writes LB on (every other LB is zero).
template <int NDIM>
__device__ __forceinline__ bool face_evolved(const Grid& g, int d, const int x[3]) {
  bool ok = NDIM == 3 || x[2] == 0;
#pragma unroll
  for (int e = 0; e < NDIM; e++) {
    ok = ok && x[e] >= 0;
    if (e == d) ok = ok && (x[e] < g.n[e] || !g.periodic[e]);
    else ok = ok && x[e] < g.n[e];
  }
  return ok;
}

// The combine transpose fused with that of the CT curl: Eb is formed
// from LB = cL Aout on the evolved faces (zero elsewhere), read from Aout,
// which no thread of this kernel writes.
template <int NDIM>
__device__ __forceinline__ void adj_combine_item(const Grid& g, const F8& Aout, const F8& A0, const F8& As,
                                                 const L6& Lb, const E3& Eb, double c0, double c1, double cL,
                                                 double dt, long long id) {
  {
    const int ex = g.n[0] + 1, ey = g.n[1] + 1;
    int i = (int)(id % ex);
    long long r = id / ex;
    int j = (int)(r % ey);
    int k = (int)(r / ey);
    int c = g.at(i, j, k);
    if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
      constexpr int NV = NDIM == 2 ? 6 : 5;
#pragma unroll
      for (int q = 0; q < NV; q++) {
        int slot = q < 5 ? q : 7;
        double x = Aout.q[slot][c];
        Lb.q[q][c] = cL * x;
        A0.q[slot][c] += c0 * x;
        As.q[slot][c] += c1 * x;
      }
    }
    const int idx3[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < NDIM; d++) {
      bool ok = true;
#pragma unroll
      for (int e = 0; e < NDIM; e++) {
        if (e == d) ok = ok && (idx3[e] < g.n[e] || !g.periodic[e]);
        else ok = ok && idx3[e] < g.n[e];
      }
      if (NDIM == 2) ok = ok && k == 0;
      if (!ok) continue;
      double x = Aout.q[5 + d][c];
      A0.q[5 + d][c] += c0 * x;
      As.q[5 + d][c] += c1 * x;
    }
    // transpose of the CT face increment L_B,d = -dt (curl E)_d at the edges
    // (i, j, k): E_C enters the faces of normal (C+1)%3 through their
    // (C+2)-difference and the faces of normal (C+2)%3 through their
    // (C+1)-difference
    auto lb = [&](int d, int di, int dj, int dk) {
      const int x[3] = {i + di, j + dj, k + dk};
      return face_evolved<NDIM>(g, d, x) ? cL * Aout.q[5 + d][g.at(x[0], x[1], x[2])] : 0.0;
    };
#pragma unroll
    for (int C = 0; C < 3; C++) {
      if (!edge_valid<NDIM>(g, C, i, j, k)) continue;
      double acc = 0.0;
      const int d = (C + 1) % 3, d1 = (C + 2) % 3;
      if (d < NDIM && d1 < NDIM)
        acc += (dt * g.idx[d1]) * (lb(d, 0, 0, 0) - lb(d, -(d1 == 0), -(d1 == 1), -(d1 == 2)));
      const int e = (C + 2) % 3, e2 = (C + 1) % 3;
      if (e < NDIM && e2 < NDIM)
        acc += (dt * g.idx[e2]) * (lb(e, -(e2 == 0), -(e2 == 1), -(e2 == 2)) - lb(e, 0, 0, 0));
      Eb.e[C][c] = acc;
    }
  }
}
template <int NDIM>
static __global__ void adj_combine_kernel(Grid g, F8 Aout, F8 A0, F8 As, L6 Lb, E3 Eb, double c0, double c1,
                                          double cL, double dt) {
  const long long total = edge_work<NDIM>(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    adj_combine_item<NDIM>(g, Aout, A0, As, Lb, Eb, c0, c1, cL, dt, id);
}


// ---------------------------------------------------------------------------
// Transpose of one UCT edge field (uct_edge<C, HLLD>): the edge-local
// cotangents
//   0-4   a-face ingredient sums (a+, a-, d, u^W, u^E; UCT-HLLD: a^L, a^R,
//         d^L, u^W, u^E), each shared by the two a-faces touching the edge,
//   5-9   the same for the b-faces,
//   10-13 the face field B_b at a-offsets -2, -1, 0, +1,
//   14-17 the face field B_a at b-offsets -2, -1, 0, +1,
//   18-19 UCT-HLLD only: d^R of the a-faces and of the b-faces.
// ---------------------------------------------------------------------------
// Cotangents of (v_-2, v_-1, v_0, v_+1) from the cotangents gw, ge of the two
// minmod-limited edge values  w = v_-1 + m(v_-1 - v_-2, v_0 - v_-1)/2  and
// e = v_0 - m(v_0 - v_-1, v_+1 - v_0)/2.
__device__ __forceinline__ void edge_recon_vjp(double vm2, double vm1, double v0, double vp1, double gw, double gev,
                                               double w[4]) {
  w[0] = w[1] = w[2] = w[3] = 0.0;
  int pw = minmod_pick(fsub(vm1, vm2), fsub(v0, vm1));
  if (pw == 1) { w[0] = fsub(w[0], kmul(RK_HALF, gw)); w[1] = fadd(w[1], fmul(1.5, gw)); }
  else if (pw == 2) { w[1] = fadd(w[1], kmul(RK_HALF, gw)); w[2] = fadd(w[2], kmul(RK_HALF, gw)); }
  else w[1] = fadd(w[1], gw);
  int pe = minmod_pick(fsub(v0, vm1), fsub(vp1, v0));
  if (pe == 1) { w[1] = fadd(w[1], kmul(RK_HALF, gev)); w[2] = fadd(w[2], kmul(RK_HALF, gev)); }
  else if (pe == 2) { w[2] = fadd(w[2], fmul(1.5, gev)); w[3] = fsub(w[3], kmul(RK_HALF, gev)); }
  else w[2] = fadd(w[2], gev);
}

template <int C, bool HLLD = false>
__device__ __forceinline__ void uct_edge_vjp(const Grid& g, const F8& S, const FaceIngr& ING, int c, double eb,
                                             double* const* ge) {
  constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
  const int sa = g.stride(A), sb = g.stride(B);
  const int cb = c - sb, ca = c - sa;
  const double* Ia[5] = {ING.a[A][0], ING.a[A][1], ING.a[A][2], ING.a[A][3], ING.a[A][4]};
  const double* Ib[5] = {ING.a[B][0], ING.a[B][1], ING.a[B][2], ING.a[B][3], ING.a[B][4]};
  double apa = fadd(Ia[0][cb], Ia[0][c]), ama = fadd(Ia[1][cb], Ia[1][c]), dda = fadd(Ia[2][cb], Ia[2][c]);
  double uW = fadd(Ia[3][cb], Ia[3][c]), uE = fadd(Ia[4][cb], Ia[4][c]);
  double apb = fadd(Ib[0][ca], Ib[0][c]), amb = fadd(Ib[1][ca], Ib[1][c]), ddb = fadd(Ib[2][ca], Ib[2][c]);
  double vS = fadd(Ib[3][ca], Ib[3][c]), vN = fadd(Ib[4][ca], Ib[4][c]);
  const double* Bb = S.q[5 + B];
  const double* Ba = S.q[5 + A];
  double bm2 = Bb[c - 2 * sa], bm1 = Bb[c - sa], b0 = Bb[c], bp1 = Bb[c + sa];
  double BbW = fma(rk(RK_HALF), minmod(fsub(bm1, bm2), fsub(b0, bm1)), bm1);
  double BbE = fma(rk(RK_MHALF), minmod(fsub(b0, bm1), fsub(bp1, b0)), b0);
  double am2 = Ba[c - 2 * sb], am1 = Ba[c - sb], a0 = Ba[c], ap1 = Ba[c + sb];
  double BaS = fma(rk(RK_HALF), minmod(fsub(am1, am2), fsub(a0, am1)), am1);
  double BaN = fma(rk(RK_MHALF), minmod(fsub(a0, am1), fsub(ap1, a0)), a0);
  // E = (1/4) [(apb vS BaS + amb vN BaN) - (apa uW BbW + ama uE BbE)]
  //   + (1/2) [dda (BbE - BbW) - ddb (BaN - BaS)]
  // UCT-HLLD: the dissipation (1/2) [(dra BbE - dda BbW) - (drb BaN - ddb BaS)]
  // with the d^R sums dra, drb
  const double gu = kmul(RK_QUARTER, eb), gd = kmul(RK_HALF, eb);
  double dra = dda, drb = ddb;
  if (HLLD) {
    dra = fadd(ING.a[A][5][cb], ING.a[A][5][c]);
    drb = fadd(ING.a[B][5][ca], ING.a[B][5][c]);
  }
  ge[0][c] = fmul(fmul(-gu, uW), BbW);
  ge[1][c] = fmul(fmul(-gu, uE), BbE);
  ge[2][c] = HLLD ? fmul(-gd, BbW) : fmul(gd, (fsub(BbE, BbW)));
  ge[3][c] = fmul(fmul(-gu, apa), BbW);
  ge[4][c] = fmul(fmul(-gu, ama), BbE);
  ge[5][c] = fmul(fmul(gu, vS), BaS);
  ge[6][c] = fmul(fmul(gu, vN), BaN);
  ge[7][c] = HLLD ? fmul(gd, BaS) : fmul(-gd, (fsub(BaN, BaS)));
  ge[8][c] = fmul(fmul(gu, apb), BaS);
  ge[9][c] = fmul(fmul(gu, amb), BaN);
  if (HLLD) {
    ge[18][c] = fmul(gd, BbE);
    ge[19][c] = fmul(-gd, BaN);
  }
  double w[4];
  edge_recon_vjp(bm2, bm1, b0, bp1, fsub(fmul(fmul(-gu, apa), uW), fmul(gd, dda)),
                 fadd(fmul(fmul(-gu, ama), uE), fmul(gd, dra)), w);
  ge[10][c] = w[0];
  ge[11][c] = w[1];
  ge[12][c] = w[2];
  ge[13][c] = w[3];
  edge_recon_vjp(am2, am1, a0, ap1, fadd(fmul(fmul(gu, apb), vS), fmul(gd, ddb)),
                 fsub(fmul(fmul(gu, amb), vN), fmul(gd, drb)), w);
  ge[14][c] = w[0];
  ge[15][c] = w[1];
  ge[16][c] = w[2];
  ge[17][c] = w[3];
}

template <int NDIM, bool HLLD = false>
__device__ __forceinline__ void adj_edge_item(const Grid& g, const F8& S, const FaceIngr& ING, const E3& Eb,
                                              const GE20& GE, long long id) {
  const int ex = g.n[0] + 1, ey = g.n[1] + 1;
  int i = (int)(id % ex);
  long long r = id / ex;
  int j = (int)(r % ey);
  int k = (int)(r / ey);
  int c = g.at(i, j, k);
  if (edge_valid<NDIM>(g, 2, i, j, k)) uct_edge_vjp<2, HLLD>(g, S, ING, c, Eb.e[2][c], GE.q[2]);
  if (NDIM == 3) {
    if (edge_valid<NDIM>(g, 0, i, j, k)) uct_edge_vjp<0, HLLD>(g, S, ING, c, Eb.e[0][c], GE.q[0]);
    if (edge_valid<NDIM>(g, 1, i, j, k)) uct_edge_vjp<1, HLLD>(g, S, ING, c, Eb.e[1][c], GE.q[1]);
  }
}
template <int NDIM, bool HLLD = false>
static __global__ void adj_edge_kernel(Grid g, F8 S, FaceIngr ING, E3 Eb, GE20 GE) {
  const long long total = edge_work<NDIM>(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    adj_edge_item<NDIM, HLLD>(g, S, ING, Eb, GE, id);
}
// The combine / CT-curl transpose and the UCT edge transpose of the same
// edge index in one thread (the edge item reads only the edge cotangents the
// combine item of its own index wrote), with the primitive cotangents of the
// reconstruction transposes cleared in the same launch: one launch for what
// adj_combine_kernel, adj_edge_kernel and a memset do, the same operations on
// every element.
template <int NDIM, bool HLLD = false>
static __global__ void adj_combine_edge_kernel(Grid g, F8 Aout, F8 A0, F8 As, L6 Lb, E3 Eb, double c0, double c1,
                                               double cL, double dt, F8 S, FaceIngr ING, GE20 GE, double* pb,
                                               long long pb_count) {
  const long long total = edge_work<NDIM>(g);
  const long long T = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long id = t0; id < total; id += T) {
    adj_combine_item<NDIM>(g, Aout, A0, As, Lb, Eb, c0, c1, cL, dt, id);
    adj_edge_item<NDIM, HLLD>(g, S, ING, Eb, GE, id);
  }
  for (long long id = t0; id < pb_count; id += T) pb[id] = 0.0;
}

// Face-field cotangents from the edge reconstructions: the face field of
// normal D is B_b of E_C for C = (D+1)%3 (reconstructed along a = (D+2)%3)
// and B_a of E_C for C = (D+2)%3 (along b = (D+1)%3).  Box: [-2, n+1] on
// every active axis.
// The cells and faces of the box [-2, n + 1] on every active axis.
template <int NDIM>
__host__ __device__ __forceinline__ long long adj_box_work(const Grid& g) {
  return (long long)(g.n[0] + 4) * (g.n[1] + 4) * (NDIM == 3 ? g.n[2] + 4 : 1);
}
template <int NDIM>
__device__ __forceinline__ void adj_edge_faces_item(const Grid& g, const GE20& GE, const F8& A, long long id) {
  int lo[3] = {-2, -2, NDIM == 3 ? -2 : 0};
  int ext[3] = {g.n[0] + 4, g.n[1] + 4, NDIM == 3 ? g.n[2] + 4 : 1};
  {
    int x[3];
    box_index(id, lo, ext, x);
    const int f = g.at(x[0], x[1], x[2]);
#pragma unroll
    for (int D = 0; D < NDIM; D++) {
      double acc = 0.0;
      bool any = false;
#pragma unroll
      for (int role = 0; role < 2; role++) {
        const int C = role == 0 ? (D + 1) % 3 : (D + 2) % 3;
        if (!has_edge<NDIM>(C)) continue;
        const int ax = role == 0 ? (D + 2) % 3 : (D + 1) % 3;  // reconstruction axis
        const int base = role == 0 ? 10 : 14;
#pragma unroll
        for (int m = 0; m < 4; m++) {  // this face is offset (m - 2) from edge e = f + (2 - m) along ax
          int y[3] = {x[0], x[1], x[2]};
          y[ax] += 2 - m;
          if (!edge_valid<NDIM>(g, C, y[0], y[1], y[2])) continue;
          acc += GE.q[C][base + m][g.at(y[0], y[1], y[2])];
          any = true;
        }
      }
      if (any) A.q[5 + D][f] += acc;
    }
  }
}
template <int NDIM>
static __global__ void adj_edge_faces_kernel(Grid g, GE20 GE, F8 A) {
  const long long total = adj_box_work<NDIM>(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    adj_edge_faces_item<NDIM>(g, GE, A, id);
}

// ---------------------------------------------------------------------------
// Riemann solver and flux difference, per face of direction DIR (faces
// [0, n_DIR], transverse [-1, n_t] as in the sweep): recompute the face's PLM
// states, take the flux cotangent from the stage-increment cotangents of its
// two cells, the UCT-ingredient cotangents from the edges that use the face,
// and push both through the solver.  Writes the cotangents of the left and
// right states, adds that of the normal face field, and records the PLM
// decisions of cell f (and of cell -1 at face 0) for the reconstruction
// reverse.
// ---------------------------------------------------------------------------
// PLM states of one cell from its 3-cell window with the positivity fallback.
__device__ __forceinline__ bool plm_cell(const double w[7][3], double plus[7], double minus[7]) {
#pragma unroll
  for (int v = 0; v < 7; v++) recon_plm(w[v][0], w[v][1], w[v][2], plus[v], minus[v]);
  if (!gt0(plus[0]) || !gt0(minus[0]) || !gt0(plus[6]) || !gt0(minus[6])) {
#pragma unroll
    for (int v = 0; v < 7; v++) plus[v] = minus[v] = w[v][1];
    return true;
  }
  return false;
}

// The PLM decisions of one cell for its reverse: the minmod pick of every
// primitive (2 bits each: 0 none, 1 the left difference, 2 the right one) and
// the positivity fallback (bit 14).
constexpr unsigned kPlmFallbackBit = 1u << 14;
__device__ __forceinline__ unsigned plm_code(const double w[7][3], bool fallback) {
  unsigned code = fallback ? kPlmFallbackBit : 0u;
#pragma unroll
  for (int v = 0; v < 7; v++) code |= (unsigned)minmod_pick(w[v][1] - w[v][0], w[v][2] - w[v][1]) << (2 * v);
  return code;
}

// WENO-Z or PPM states of one cell from its 5-cell window, with the positivity
// fallback of the forward sweep (recon_wenoz gives the marching sweep's bits).
template <int RECON>
__device__ __forceinline__ void recon_one5(const double w[5], double& plus, double& minus) {
  if constexpr (RECON == RECON_WENOZ) recon_wenoz(w[0], w[1], w[2], w[3], w[4], plus, minus);
  else recon_ppm(w[0], w[1], w[2], w[3], w[4], plus, minus);
}
template <int RECON>
__device__ __forceinline__ bool recon_cell5(const double w[7][5], double plus[7], double minus[7]) {
#pragma unroll
  for (int v = 0; v < 7; v++) recon_one5<RECON>(w[v], plus[v], minus[v]);
  if (!gt0(plus[0]) || !gt0(minus[0]) || !gt0(plus[6]) || !gt0(minus[6])) {
#pragma unroll
    for (int v = 0; v < 7; v++) plus[v] = minus[v] = w[v][2];
    return true;
  }
  return false;
}

template <int DIR, int NDIM>
__device__ __forceinline__ void sweep_box(const Grid& g, int lo[3], int ext[3], int dir_lo, int dir_hi) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a == DIR) { lo[a] = dir_lo; ext[a] = dir_hi - dir_lo + 1; }
    else if (a < NDIM) { lo[a] = -1; ext[a] = g.n[a] + 2; }
    else { lo[a] = 0; ext[a] = 1; }
  }
}

// Vector-Jacobian product of the Riemann solver by forward-mode numbers: five
// passes of three tangents over the 15 inputs (W_L, W_R, b_n).  Kept as the
// cross-check of the hand-written reverse below.
template <int RS>
__device__ __forceinline__ void riemann_vjp_dual(const double xin[15], double gamma, double igm1, const double Fb[7],
                                                 const double Ib[6], double xb[15]) {
#pragma unroll
  for (int p = 0; p < 5; p++) {
    D3 in[15];
#pragma unroll
    for (int i = 0; i < 15; i++) {
      in[i] = D3(xin[i]);
      if (i / 3 == p) in[i].d[i % 3] = 1.0;
    }
    W7T<D3> L = {in[0], in[1], in[2], in[3], in[4], in[5], in[6]};
    W7T<D3> R = {in[7], in[8], in[9], in[10], in[11], in[12], in[13]};
    Flux7T<D3> F;
    IngrT<D3> ing;
    if (RS == RS_HLLD_UCT) riemann_hlld<D3, true>(L, R, in[14], gamma, igm1, F, ing);
    else if (RS == RS_HLLD) riemann_hlld(L, R, in[14], gamma, igm1, F, ing);
    else riemann_hll(L, R, in[14], gamma, igm1, F, ing);
#pragma unroll
    for (int t = 0; t < 3; t++) {
      double acc = Ib[0] * ing.ap.d[t];
      if (RS == RS_HLLD_UCT) acc = fma(Ib[5], ing.dr.d[t], acc);
      acc = fma(Ib[1], ing.am.d[t], acc);
      acc = fma(Ib[2], ing.dd.d[t], acc);
      acc = fma(Ib[3], ing.uL.d[t], acc);
      acc = fma(Ib[4], ing.uR.d[t], acc);
#pragma unroll
      for (int q = 0; q < 7; q++) acc = fma(Fb[q], F.f[q].d[t], acc);
      xb[3 * p + t] = acc;
    }
  }
}

// Vector-Jacobian product of the Riemann solver by its hand-written reverse.
// Ib: the ingredient cotangents (a+, a-, d, u_L, u_R; RS_HLLD_UCT: a^L, a^R,
// d^L, u_L, u_R, d^R).
template <int RS>
__device__ __forceinline__ void riemann_vjp(const double xin[15], double gamma, double igm1, const double Fb[7],
                                            const double Ib[6], double xb[15]) {
  const W7 L = {xin[0], xin[1], xin[2], xin[3], xin[4], xin[5], xin[6]};
  const W7 R = {xin[7], xin[8], xin[9], xin[10], xin[11], xin[12], xin[13]};
  W7b Lb, Rb;
  double bnb = 0.0;
  if (RS == RS_HLLD_UCT) riemann_hlld_vjp<true>(L, R, xin[14], gamma, igm1, Fb, Ib, Lb, Rb, bnb);
  else if (RS == RS_HLLD) riemann_hlld_vjp(L, R, xin[14], gamma, igm1, Fb, Ib, Lb, Rb, bnb);
  else riemann_hll_vjp(L, R, xin[14], gamma, igm1, Fb, Ib, Lb, Rb, bnb);
  const double out[15] = {Lb.rho, Lb.u, Lb.v, Lb.w, Lb.b1, Lb.b2, Lb.p,
                          Rb.rho, Rb.u, Rb.v, Rb.w, Rb.b1, Rb.b2, Rb.p, bnb};
#pragma unroll
  for (int i = 0; i < 15; i++) xb[i] = out[i];
}

// Both products on n faces: in[15 n] = (W_L, W_R, b_n) per face, cot[NC n] =
// (flux cotangent 7, ingredient cotangents NC - 7: 5, or 6 with d^R);
// dual / hand [15 n].
template <int RS, int NC = 12>
static __global__ void riemann_vjp_probe_kernel(int n, double gamma, const double* __restrict__ in,
                                                const double* __restrict__ cot, double* dual, double* hand) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  double x[15], Fb[7], Ib[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, xb[15];
#pragma unroll
  for (int i = 0; i < 15; i++) x[i] = in[15 * f + i];
#pragma unroll
  for (int i = 0; i < 7; i++) Fb[i] = cot[NC * f + i];
#pragma unroll
  for (int i = 0; i < NC - 7; i++) Ib[i] = cot[NC * f + 7 + i];
  const double igm1 = 1.0 / (gamma - 1.0);
  riemann_vjp_dual<RS>(x, gamma, igm1, Fb, Ib, xb);
#pragma unroll
  for (int i = 0; i < 15; i++) dual[15 * f + i] = xb[i];
  riemann_vjp<RS>(x, gamma, igm1, Fb, Ib, xb);
#pragma unroll
  for (int i = 0; i < 15; i++) hand[15 * f + i] = xb[i];
}

// WENO-Z / PPM: the face states of direction DIR, each cell's reconstruction
// formed once (cells [-1, n] along DIR, [-1, n] across): its plus state into
// WbL at face x+1, its minus state into WbR at face x -- the slots where the
// Riemann transpose of that face reads them and then stores their cotangents.
template <int DIR, int NDIM>
__host__ __device__ __forceinline__ long long adj_face_states_work(const Grid& g) {
  long long w = 1;
  for (int d = 0; d < 3; d++) w *= d == DIR ? g.n[d] + 2 : (d < NDIM ? g.n[d] + 2 : 1);
  return w;
}
template <int DIR, int NDIM, int RECON>
static __global__ void __launch_bounds__(128) adj_face_states_kernel(Grid g, F8 P, F8 WbL, F8 WbR,
                                                                     unsigned* fallback) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= adj_face_states_work<DIR, NDIM>(g)) return;
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  int lo[3], ext[3];
  sweep_box<DIR, NDIM>(g, lo, ext, -1, g.n[DIR]);
  int x[3];
  box_index(id, lo, ext, x);
  const int co = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  const double* pr[7] = {P.q[0], P.q[1 + DIR], P.q[1 + T1], P.q[1 + T2], P.q[4 + T1], P.q[4 + T2], P.q[7]};
  double w[7][5], plus[7], minus[7];
#pragma unroll
  for (int v = 0; v < 7; v++)
#pragma unroll
    for (int m = 0; m < 5; m++) w[v][m] = pr[v][co + (m - 2) * st];
  fallback[co] = recon_cell5<RECON>(w, plus, minus) ? 1u : 0u;  // for the reconstruction transpose
  const bool up = x[DIR] + 1 <= g.n[DIR], down = x[DIR] >= 0;
#pragma unroll
  for (int v = 0; v < 7; v++) {
    if (up) WbL.q[v][co + st] = plus[v];
    if (down) WbR.q[v][co] = minus[v];
  }
}

template <int DIR, int NDIM>
__host__ __device__ __forceinline__ long long adj_riemann_work(const Grid& g) {
  long long faces = 1;
  for (int d = 0; d < 3; d++) faces *= d == DIR ? g.n[d] + 1 : (d < NDIM ? g.n[d] + 2 : 1);
  return faces;
}
template <int DIR, int NDIM, int RS, int RECON = RECON_PLM>
__device__ __forceinline__ void adj_riemann_item(const Grid& g, const F8& P, const double* Bn, const L6& Lb,
                                                 const GE20& GE, double dt, const F8& WbL, const F8& WbR,
                                                 double* Bnb, unsigned* plm_codes, long long id) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  int lo[3], ext[3];
  sweep_box<DIR, NDIM>(g, lo, ext, 0, g.n[DIR]);
  int x[3];
  box_index(id, lo, ext, x);
  const int cf = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  const double* pr[7] = {P.q[0], P.q[1 + DIR], P.q[1 + T1], P.q[1 + T2], P.q[4 + T1], P.q[4 + T2], P.q[7]};
  // the face's states: plus of cell f-1 and minus of cell f
  double xin[15];
  if constexpr (RECON != RECON_PLM) {  // the states adj_face_states_kernel left in the cotangent slots
#pragma unroll
    for (int v = 0; v < 7; v++) {
      xin[v] = WbL.q[v][cf];
      xin[7 + v] = WbR.q[v][cf];
    }
  } else {
    double w[7][3], plus[7], minus[7];
#pragma unroll
    for (int v = 0; v < 7; v++)
#pragma unroll
      for (int m = 0; m < 3; m++) w[v][m] = pr[v][cf + (m - 2) * st];
    bool fb = plm_cell(w, plus, minus);
    if (x[DIR] == 0) plm_codes[cf - st] = plm_code(w, fb);  // cell -1
#pragma unroll
    for (int v = 0; v < 7; v++) xin[v] = plus[v];
#pragma unroll
    for (int v = 0; v < 7; v++)
#pragma unroll
      for (int m = 0; m < 3; m++) w[v][m] = pr[v][cf + (m - 1) * st];
    fb = plm_cell(w, plus, minus);
    plm_codes[cf] = plm_code(w, fb);  // cell f
#pragma unroll
    for (int v = 0; v < 7; v++) xin[7 + v] = minus[v];
  }
  xin[14] = Bn[cf];
  // flux cotangent: L(cell f-1) gets -dtdx F_f, L(cell f) gets +dtdx F_f
  const double dtdx = dt * g.idx[DIR];
  auto lbar = [&](int q) { return dtdx * (Lb.q[q][cf] - Lb.q[q][cf - st]); };
  double Fb[7];
  Fb[0] = lbar(0);
  Fb[1] = lbar(1 + DIR);
  Fb[2] = lbar(1 + T1);
  Fb[3] = lbar(1 + T2);
  Fb[4] = 0.0;
  Fb[5] = 0.0;
  Fb[6] = lbar(4);
  if (NDIM == 2) {
    if (DIR == 0) Fb[5] = lbar(5);
    else Fb[4] = lbar(5);
  }
  // UCT-ingredient cotangent from the edges that use this face
  double Ib[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int role = 0; role < 2; role++) {
    const int C = role == 0 ? (DIR + 2) % 3 : (DIR + 1) % 3;  // this face is an a-face / a b-face of E_C
    if (!has_edge<NDIM>(C)) continue;
    const int ax = role == 0 ? (DIR + 1) % 3 : (DIR + 2) % 3;  // the edges at this face and one step up ax
    const int base = role == 0 ? 0 : 5;
#pragma unroll
    for (int m = 0; m < 2; m++) {
      int y[3] = {x[0], x[1], x[2]};
      y[ax] += m;
      if (!edge_valid<NDIM>(g, C, y[0], y[1], y[2])) continue;
      const int e = g.at(y[0], y[1], y[2]);
#pragma unroll
      for (int q = 0; q < 5; q++) Ib[q] += GE.q[C][base + q][e];
      if (RS == RS_HLLD_UCT) Ib[5] += GE.q[C][18 + role][e];
    }
  }
  double xb[15];
  riemann_vjp<RS>(xin, g.gamma, g.igm1, Fb, Ib, xb);
#pragma unroll
  for (int v = 0; v < 7; v++) {
    WbL.q[v][cf] = xb[v];
    WbR.q[v][cf] = xb[7 + v];
  }
  Bnb[cf] += xb[14];
}
template <int DIR, int NDIM, int RS, int RECON = RECON_PLM>
static __global__ void __launch_bounds__(128) adj_riemann_kernel(Grid g, F8 P, const double* __restrict__ Bn,
                                                                 L6 Lb, GE20 GE, double dt, F8 WbL, F8 WbR,
                                                                 double* Bnb, unsigned* plm_codes) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= adj_riemann_work<DIR, NDIM>(g)) return;
  adj_riemann_item<DIR, NDIM, RS, RECON>(g, P, Bn, Lb, GE, dt, WbL, WbR, Bnb, plm_codes, id);
}

// ---------------------------------------------------------------------------
// PLM reconstruction, per cell of the sweep box along DIR ([-2, n_DIR + 1]):
// gather the state cotangents of the three cells whose reconstruction reads
// this cell and add their contribution to the primitive cotangents, with the
// PLM decisions adj_riemann_kernel recorded for those cells.
// ---------------------------------------------------------------------------
// Primitive slot of the v-th sweep-order variable of direction d.
__device__ __forceinline__ int recon_slot(int d, int v) {
  return v == 0 ? 0 : (v < 4 ? 1 + (d + v - 1) % 3 : (v < 6 ? 4 + (d + v - 3) % 3 : 7));
}
template <int DIR, int NDIM>
__device__ __forceinline__ void adj_recon_item(const Grid& g, const unsigned* plm_codes, const F8& WbL,
                                               const F8& WbR, const int x[3], double acc[7]) {
  // acc[v]: the cotangent this cell's primitive recon_slot(DIR, v) receives
  const int c = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  const int n = g.n[DIR];
#pragma unroll
  for (int v = 0; v < 7; v++) acc[v] = 0.0;
#pragma unroll
  for (int o = -1; o <= 1; o++) {  // reconstruction of cell x + o reads this cell at window slot 1 - o
    const int xo = x[DIR] + o;
    if (xo < -1 || xo > n) continue;
    const int co = c + o * st;
    const unsigned code = plm_codes[co];
    const bool fb = (code & kPlmFallbackBit) != 0u;
#pragma unroll
    for (int v = 0; v < 7; v++) {
      const double pb = xo + 1 <= n ? WbL.q[v][co + st] : 0.0;  // plus state: left state of face xo+1
      const double mb = xo >= 0 ? WbR.q[v][co] : 0.0;           // minus state: right state of face xo
      if (fb) {
        if (o == 0) acc[v] += pb + mb;
        continue;
      }
      double ws[3] = {0.0, 0.0, 0.0};  // cotangents of the window cells
      ws[1] = pb + mb;
      const double db = 0.5 * (pb - mb);
      const int pick = (int)((code >> (2 * v)) & 3u);
      if (pick == 1) { ws[1] += db; ws[0] -= db; }
      else if (pick == 2) { ws[2] += db; ws[1] -= db; }
      acc[v] += ws[1 - o];
    }
  }
}
// Every direction's reconstruction transpose in one launch, over the union of
// the directions' sweep boxes ([-2, n + 1] along the direction, the sweep's
// pencils [-1, n] across it): each cell adds the directions' contributions to
// its primitive cotangents in direction order, the same additions in the
// same order as one launch per direction.
template <int NDIM>
__device__ __forceinline__ void adj_recon_all_item(const Grid& g, const unsigned* codes0, const unsigned* codes1,
                                                   const unsigned* codes2, const F8& WbL0, const F8& WbR0,
                                                   const F8& WbL1, const F8& WbR1, const F8& WbL2, const F8& WbR2,
                                                   const F8& Pb, long long id) {
  int lo[3] = {-2, -2, NDIM == 3 ? -2 : 0};
  int ext[3] = {g.n[0] + 4, g.n[1] + 4, NDIM == 3 ? g.n[2] + 4 : 1};
  int x[3];
  box_index(id, lo, ext, x);
  // in the DIR box: [-2, n + 1] along DIR, [-1, n] along the other active axes
  auto in_box = [&](int dir) {
    for (int e = 0; e < NDIM; e++)
      if (e != dir && (x[e] < -1 || x[e] > g.n[e])) return false;
    return true;
  };
  const bool in[3] = {in_box(0), in_box(1), NDIM == 3 && in_box(2)};
  double acc[3][7];
  if (in[0]) adj_recon_item<0, NDIM>(g, codes0, WbL0, WbR0, x, acc[0]);
  if (in[1]) adj_recon_item<1, NDIM>(g, codes1, WbL1, WbR1, x, acc[1]);
  if (in[2]) adj_recon_item<NDIM == 3 ? 2 : 0, NDIM>(g, codes2, WbL2, WbR2, x, acc[2]);
  // the primitive cotangents the directions add to, all loaded before any
  // store; then each direction's terms in direction order, as separate
  // launches per direction would add them
  const int c = g.at(x[0], x[1], x[2]);
  bool t[8] = {false, false, false, false, false, false, false, false};
#pragma unroll
  for (int d = 0; d < NDIM; d++)
    if (in[d])
#pragma unroll
      for (int v = 0; v < 7; v++) t[recon_slot(d, v)] = true;
  double pv[8];
#pragma unroll
  for (int q = 0; q < 8; q++)
    if (t[q]) pv[q] = Pb.q[q][c];
#pragma unroll
  for (int d = 0; d < NDIM; d++)
    if (in[d])
#pragma unroll
      for (int v = 0; v < 7; v++) pv[recon_slot(d, v)] += acc[d][v];
#pragma unroll
  for (int q = 0; q < 8; q++)
    if (t[q]) Pb.q[q][c] = pv[q];
}
template <int NDIM>
static __global__ void __launch_bounds__(128) adj_recon_all_kernel(Grid g, const unsigned* __restrict__ codes0,
                                                                   const unsigned* __restrict__ codes1,
                                                                   const unsigned* __restrict__ codes2, F8 WbL0,
                                                                   F8 WbR0, F8 WbL1, F8 WbR1, F8 WbL2, F8 WbR2,
                                                                   F8 Pb) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= adj_box_work<NDIM>(g)) return;
  adj_recon_all_item<NDIM>(g, codes0, codes1, codes2, WbL0, WbR0, WbL1, WbR1, WbL2, WbR2, Pb, id);
}

// ---------------------------------------------------------------------------
// WENO-Z and PPM reconstruction transposes.  A cell's reconstruction reads
// five cells, so a cell's cotangent gathers from the reconstructions of five
// cells; re-deriving each of them in every reader would cost five times the
// work.  Instead two launches per direction:
//   cell pass    per owner cell x ([-1, n] along DIR, [-1, n] across): redo
//                its reconstruction and form the cotangents of its five
//                window cells from those of its plus state (left state of
//                face x+1) and minus state (right state of face x);
//                window slot m of variable v goes to T.q[7 m + v];
//   gather pass  per cell ([-3, n + 2] along DIR): add the slots the five
//                owners x-2..x+2 left for it (slot 2 - o of owner x+o), in
//                owner order, to its primitive cotangents.
// T lives in the edge-local cotangent fields, free once the Riemann
// transposes of every direction have read them.
// ---------------------------------------------------------------------------
struct T35 { double* q[35]; };

// Constants of the WENO-Z reverse that the shared register table lacks, read
// into registers the same way (a DFMA with a register operand issues faster
// than one with a constant-bank operand).
__device__ double kWzAdjK[2] = {-0.6, -6.0};
__device__ __forceinline__ double wk(int i) { return __ldg(&kWzAdjK[i]); }

// Reverse of recon_wenoz (both faces of the middle cell of a[0..4]): ab[]
// receives the window cotangents for pb = dJ/d(plus), mb = dJ/d(minus).  The
// values to linearise at are formed without divisions, within a few ulps of
// the forward's, in scaled forms that the FMAs take for free: the indicators
// as BE_k = 4 (beta_k + eps) = (13/3) t_k^2 + u_k^2 + 4 eps (the factor
// cancels in r_k = tau5 / (beta_k + eps)), the candidates as Q_k = 6 q_k with
// d_0 folded into Q_0' = 6 d_0 q_0, so that with g_k = 1 + r_k^2
//   plus = num / den,  num = g_0 Q_0' + 0.6 g_1 Q_1 + 0.3 g_2 Q_2,
//   den = 0.6 g_0 + 3.6 g_1 + 1.8 g_2  (= 6 sum_k d_k g_k),
// and the mirrored weights for minus.  Reverse, with P = pb / den:
//   dJ/dQ_0' = P g_0, dJ/dQ_1 = 0.6 P g_1, dJ/dQ_2 = 0.3 P g_2,
//   dJ/dg_0 = P (Q_0' - 0.6 plus), dJ/dg_1 = 0.6 P (Q_1 - 6 plus),
//   dJ/dg_2 = 0.3 P (Q_2 - 6 plus)  (and the mirror for minus);
//   g_k = 1 + r_k^2, r_k = tau ib_k, ib_k = 1 / BE_k: with S_k = r_k gb_k ib_k,
//   dJ/dtau = 2 sum_k S_k, dJ/dBE_k = -2 S_k r_k, plus dJ/dtau for k = 0 and
//   minus it for k = 2; E_k = 2 dJ/dBE_k carries the factor 2 of
//   dBE_k/dt_k = 2 (13/3) t_k and dBE_k/du_k = 2 u_k;
// then the transposes of the linear stencils t_k, u_k and Q.
__device__ __forceinline__ void wenoz_vjp(const double a[5], double pb, double mb, double ab[5]) {
  // forward
  const double t0 = fadd(fma(rk(RK_M2), a[1], a[0]), a[2]);
  const double t1 = fadd(fma(rk(RK_M2), a[2], a[1]), a[3]);
  const double t2 = fadd(fma(rk(RK_M2), a[3], a[2]), a[4]);
  const double u0 = fma(rk(RK_3), a[2], fma(rk(RK_M4), a[1], a[0]));
  const double u1 = fsub(a[1], a[3]);
  const double u2 = fma(rk(RK_3), a[2], fma(rk(RK_M4), a[3], a[4]));
  const double K0 = kmul(RK_13_3, t0), K1 = kmul(RK_13_3, t1), K2 = kmul(RK_13_3, t2);
  const double be0 = fma(K0, t0, fma(u0, u0, rk(RK_4WEPS)));
  const double be1 = fma(K1, t1, fma(u1, u1, rk(RK_4WEPS)));
  const double be2 = fma(K2, t2, fma(u2, u2, rk(RK_4WEPS)));
  const double tau = fsub(be0, be2);
  const double ib0 = rcp(be0), ib1 = rcp(be1), ib2 = rcp(be2);
  const double r0 = fmul(tau, ib0), r1 = fmul(tau, ib1), r2 = fmul(tau, ib2);
  const double g0 = fma(r0, r0, rk(RK_ONE)), g1 = fma(r1, r1, rk(RK_ONE)), g2 = fma(r2, r2, rk(RK_ONE));
  const double c11 = kmul(RK_1_1, a[2]);
  const double Qp0 = fma(rk(RK_0_2), a[0], fma(rk(RK_M0_7), a[1], c11));
  const double Qp1 = fma(rk(RK_5), a[2], fma(rk(RK_2), a[3], -a[1]));
  const double Qp2 = fma(rk(RK_2), a[2], fma(rk(RK_5), a[3], -a[4]));
  const double Qm0 = fma(rk(RK_0_2), a[4], fma(rk(RK_M0_7), a[3], c11));
  const double Qm1 = fma(rk(RK_5), a[2], fma(rk(RK_2), a[1], -a[3]));
  const double Qm2 = fma(rk(RK_2), a[2], fma(rk(RK_5), a[1], -a[0]));
  const double w1 = kmul(RK_0_6, g1), K61 = kmul(RK_3_6, g1);
  const double w2p = kmul(RK_0_3, g2), w0m = kmul(RK_0_3, g0);
  const double ip = rcp(fma(rk(RK_0_6), g0, fma(rk(RK_1_8), g2, K61)));
  const double im = rcp(fma(rk(RK_0_6), g2, fma(rk(RK_1_8), g0, K61)));
  const double vp = fmul(fma(g0, Qp0, fma(w1, Qp1, fmul(w2p, Qp2))), ip);
  const double vm = fmul(fma(g2, Qm0, fma(w1, Qm1, fmul(w0m, Qm2))), im);
  // reverse
  const double P = fmul(pb, ip), M = fmul(mb, im);
  const double QBp0 = fmul(P, g0), QBp1 = fmul(P, w1), QBp2 = fmul(P, w2p);
  const double QBm0 = fmul(M, g2), QBm1 = fmul(M, w1), QBm2 = fmul(M, w0m);
  const double P3 = kmul(RK_0_3, P), M3 = kmul(RK_0_3, M);
  const double gb0 = fma(P, fma(wk(0), vp, Qp0), fmul(M3, fma(wk(1), vm, Qm2)));
  const double gb1 = kmul(RK_0_6, fma(P, fma(wk(1), vp, Qp1), fmul(M, fma(wk(1), vm, Qm1))));
  const double gb2 = fma(M, fma(wk(0), vm, Qm0), fmul(P3, fma(wk(1), vp, Qp2)));
  const double S0 = fmul(fmul(r0, gb0), ib0), S1 = fmul(fmul(r1, gb1), ib1), S2 = fmul(fmul(r2, gb2), ib2);
  const double T4 = kmul(RK_FOUR, fadd(fadd(S0, S1), S2));  // 2 dJ/dtau
  const double E0 = fma(S0, kmul(RK_M4, r0), T4);
  const double E1 = fmul(S1, kmul(RK_M4, r1));
  const double E2 = fma(S2, kmul(RK_M4, r2), -T4);
  const double tb0 = fmul(E0, K0), tb1 = fmul(E1, K1), tb2 = fmul(E2, K2);
  const double ub0 = fmul(E0, u0), ub1 = fmul(E1, u1), ub2 = fmul(E2, u2);
  ab[0] = fma(rk(RK_0_2), QBp0, fsub(fadd(tb0, ub0), QBm2));
  ab[1] = fma(rk(RK_M0_7), QBp0,
              fma(rk(RK_2), QBm1,
                  fma(rk(RK_5), QBm2, fma(rk(RK_M2), tb0, fma(rk(RK_M4), ub0, fsub(fadd(tb1, ub1), QBp1))))));
  ab[2] = fma(rk(RK_1_1), fadd(QBp0, QBm0),
              fma(rk(RK_5), fadd(QBp1, QBm1),
                  fma(rk(RK_2), fadd(QBp2, QBm2), fma(rk(RK_3), fadd(ub0, ub2), fma(rk(RK_M2), tb1, fadd(tb0, tb2))))));
  ab[3] = fma(rk(RK_2), QBp1,
              fma(rk(RK_5), QBp2,
                  fma(rk(RK_M0_7), QBm0, fma(rk(RK_M2), tb2, fma(rk(RK_M4), ub2, fsub(fsub(tb1, ub1), QBm1))))));
  ab[4] = fma(rk(RK_0_2), QBm0, fsub(fadd(tb2, ub2), QBp2));
}

// Reverse of ppm_face(a, b, c, d): the clipped fourth-order value passes its
// cotangent fb to (a, b, c, d) with weights (-1/12, 7/12, 7/12, -1/12), or all
// of it to the neighbour it was clipped to (the choices ppm_face takes).
__device__ __forceinline__ void ppm_face_vjp(double a, double b, double c, double d, double fb, double ab[4]) {
  const double f = fma(rk(RK_7_12), fadd(b, c), -kmul(RK_1_12, fadd(a, d)));
  const double lo = imin(b, c), hi = imax(b, c);
  const bool lo_wins = order_key(f) < order_key(lo);  // imax(f, lo) took lo
  const bool hi_wins = order_key(hi) < order_key(lo_wins ? lo : f);  // imin(., hi) took hi
  ab[0] = ab[1] = ab[2] = ab[3] = 0.0;
  if (hi_wins) {
    if (order_key(b) < order_key(c)) ab[2] = fb;  // imax(b, c) = c
    else ab[1] = fb;
  } else if (lo_wins) {
    if (order_key(c) < order_key(b)) ab[2] = fb;  // imin(b, c) = c
    else ab[1] = fb;
  } else {
    ab[0] = (-1.0 / 12.0) * fb;
    ab[1] = (7.0 / 12.0) * fb;
    ab[2] = ab[1];
    ab[3] = ab[0];
  }
}
// Reverse of recon_ppm: the branch the forward values take (flattened,
// minus side steepened, plus side steepened, or neither), then the two face
// values' transposes.
__device__ __forceinline__ void ppm_vjp(const double s[5], double pb, double mb, double ab[5]) {
  const double vp = ppm_face(s[1], s[2], s[3], s[4]);
  const double vm = ppm_face(s[0], s[1], s[2], s[3]);
  double vpb = 0.0, vmb = 0.0;
  ab[0] = ab[1] = ab[2] = ab[3] = ab[4] = 0.0;
  if (!gt0(fmul(fsub(vp, s[2]), fsub(s[2], vm)))) {
    ab[2] = pb + mb;
  } else {
    const double dv = fsub(vp, vm);
    const double v6 = kmul(RK_6, fma(rk(RK_MHALF), fadd(vm, vp), s[2]));
    const double x = fmul(dv, v6), y = fmul(dv, dv);
    if (order_key(y) < order_key(x)) {         // vm = 3 s2 - 2 vp
      ab[2] = 3.0 * mb;
      vpb = pb - 2.0 * mb;
    } else if (order_key(x) < ~bits(y)) {      // vp = 3 s2 - 2 vm
      ab[2] = 3.0 * pb;
      vmb = mb - 2.0 * pb;
    } else {
      vpb = pb;
      vmb = mb;
    }
  }
  double fbv[4];
  ppm_face_vjp(s[1], s[2], s[3], s[4], vpb, fbv);
#pragma unroll
  for (int m = 0; m < 4; m++) ab[1 + m] += fbv[m];
  ppm_face_vjp(s[0], s[1], s[2], s[3], vmb, fbv);
#pragma unroll
  for (int m = 0; m < 4; m++) ab[m] += fbv[m];
}

template <int DIR, int NDIM>
__host__ __device__ __forceinline__ long long adj_recon5_cells(const Grid& g, int along) {
  long long w = 1;
  for (int d = 0; d < 3; d++) w *= d == DIR ? along : (d < NDIM ? g.n[d] + 2 : 1);
  return w;
}
template <int DIR, int NDIM, int RECON>
__device__ __forceinline__ void adj_recon5_cell_item(const Grid& g, const F8& P, const F8& WbL, const F8& WbR,
                                                     const unsigned* fallback, const T35& T, long long id) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  int lo[3], ext[3];
  sweep_box<DIR, NDIM>(g, lo, ext, -1, g.n[DIR]);
  int x[3];
  box_index(id, lo, ext, x);
  const int co = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  const int n = g.n[DIR];
  const double* pr[7] = {P.q[0], P.q[1 + DIR], P.q[1 + T1], P.q[1 + T2], P.q[4 + T1], P.q[4 + T2], P.q[7]};
  double w[7][5];
#pragma unroll
  for (int v = 0; v < 7; v++)
#pragma unroll
    for (int m = 0; m < 5; m++) w[v][m] = pr[v][co + (m - 2) * st];
  const bool fb = fallback[co] != 0u;  // the positivity fallback adj_face_states_kernel recorded
#pragma unroll
  for (int v = 0; v < 7; v++) {
    const double pb = x[DIR] + 1 <= n ? WbL.q[v][co + st] : 0.0;
    const double mb = x[DIR] >= 0 ? WbR.q[v][co] : 0.0;
    double ab[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (fb) ab[2] = pb + mb;
    else if constexpr (RECON == RECON_WENOZ) wenoz_vjp(w[v], pb, mb, ab);
    else ppm_vjp(w[v], pb, mb, ab);
#pragma unroll
    for (int m = 0; m < 5; m++) T.q[7 * m + v][co] = ab[m];
  }
}
template <int DIR, int NDIM, int RECON>
static __global__ void __launch_bounds__(128) adj_recon5_cell_kernel(Grid g, F8 P, F8 WbL, F8 WbR,
                                                                     const unsigned* __restrict__ fallback, T35 T) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= adj_recon5_cells<DIR, NDIM>(g, g.n[DIR] + 2)) return;
  adj_recon5_cell_item<DIR, NDIM, RECON>(g, P, WbL, WbR, fallback, T, id);
}
template <int DIR, int NDIM>
static __global__ void __launch_bounds__(128) adj_recon5_gather_kernel(Grid g, T35 T, F8 Pb) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= adj_recon5_cells<DIR, NDIM>(g, g.n[DIR] + 6)) return;
  int lo[3], ext[3];
  sweep_box<DIR, NDIM>(g, lo, ext, -3, g.n[DIR] + 2);
  int x[3];
  box_index(id, lo, ext, x);
  const int c = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  const int n = g.n[DIR];
  double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int o = -2; o <= 2; o++) {  // owner x + o reads this cell at window slot 2 - o
    const int xo = x[DIR] + o;
    if (xo < -1 || xo > n) continue;
#pragma unroll
    for (int v = 0; v < 7; v++) acc[v] += T.q[7 * (2 - o) + v][c + o * st];
  }
#pragma unroll
  for (int v = 0; v < 7; v++) Pb.q[recon_slot(DIR, v)][c] += acc[v];
}

// ---------------------------------------------------------------------------
// Primitive recovery, v = m/rho, p = (G-1)(E - m.v/2 - B^2/2) with the cell
// field B = the mean of its two faces, transposed in one launch: thread id
// serves the padded cell and the faces with the same index.
//   cell: the cotangents of rho, m, E (2D: and of the cell B_z) from the
//         primitive cotangents Pb; a pressure raised to the floor passes none;
//   face: half of each adjacent padded cell's field cotangent
//         Pb.q[4 + d] - (G-1) pb B_d, formed by the face itself.
template <int NDIM>
__device__ __forceinline__ double adj_c2p_gp(const Grid& g, const F8& S, const F8& P, const F8& Pb, int c) {
  // The forward raises a recovered pressure below the floor to it in every
  // padded cell, a floor of 0 included (outflow ghost cells can recover a
  // negative pressure: their normal field is extrapolated, their energy
  // copied); such a cell passes no pressure cotangent.  A stored pressure
  // above the floor was not raised; one at the floor is decided as the
  // forward decided it, on the IEEE pressure.
  double pb = Pb.q[7][c];
  if (!(P.q[7][c] > g.p_floor)) {
    Prim8 V = c2p_ieee(S.q[0][c], S.q[1][c], S.q[2][c], S.q[3][c], S.q[4][c], P.q[4][c], P.q[5][c], P.q[6][c], g.gm1);
    if (V.p < g.p_floor) pb = 0.0;
  }
  return g.gm1 * pb;
}
template <int NDIM>
__device__ __forceinline__ void adj_c2p_item(const Grid& g, const F8& S, const F8& P, const F8& Pb, const F8& A,
                                             long long id) {
  int lo[3] = {-g.G, -g.G, NDIM == 3 ? -g.G : 0};
  int ext[3] = {g.n[0] + 2 * g.G + 1, g.n[1] + 2 * g.G + 1, NDIM == 3 ? g.n[2] + 2 * g.G + 1 : 1};
  {
    int x[3];
    box_index(id, lo, ext, x);
    const int c = g.at(x[0], x[1], x[2]);
    bool cell = true;  // a padded cell: every index within [-G, n + G - 1]
#pragma unroll
    for (int e = 0; e < NDIM; e++)
      if (x[e] > g.n[e] + g.G - 1) cell = false;
    // the increments first, then the cotangents they add to, then the stores,
    // so that all loads are in flight together
    double cv[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (cell) {
      const double rho = P.q[0][c], vx = P.q[1][c], vy = P.q[2][c], vz = P.q[3][c];
      const double gp = adj_c2p_gp<NDIM>(g, S, P, Pb, c);
      const double ir = 1.0 / rho;
      const double vbx = Pb.q[1][c], vby = Pb.q[2][c], vbz = Pb.q[3][c];
      const double v2 = (vx * vx + vy * vy) + vz * vz;
      cv[0] = (Pb.q[0][c] - ((vbx * vx + vby * vy) + vbz * vz) * ir) + 0.5 * gp * v2;
      cv[1] = vbx * ir - gp * vx;
      cv[2] = vby * ir - gp * vy;
      cv[3] = vbz * ir - gp * vz;
      cv[4] = gp;
      if (NDIM == 2) cv[5] = Pb.q[6][c] - gp * P.q[6][c];
    }
    bool fok[3] = {false, false, false};
    double fv[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < NDIM; d++) {
      bool ok = true;  // the transverse indices must be those of padded cells
#pragma unroll
      for (int e = 0; e < NDIM; e++)
        if (e != d && x[e] > g.n[e] + g.G - 1) ok = false;
      if (!ok) continue;
      double acc = 0.0;
      if (x[d] <= g.n[d] + g.G - 1) acc += Pb.q[4 + d][c] - adj_c2p_gp<NDIM>(g, S, P, Pb, c) * P.q[4 + d][c];
      if (x[d] - 1 >= -g.G) {
        const int cm = c - g.stride(d);
        acc += Pb.q[4 + d][cm] - adj_c2p_gp<NDIM>(g, S, P, Pb, cm) * P.q[4 + d][cm];
      }
      fok[d] = true;
      fv[d] = 0.5 * acc;
    }
    constexpr int kCellSlot[6] = {0, 1, 2, 3, 4, 7};
    constexpr int NC = NDIM == 2 ? 6 : 5;
    double ao[6], fo[3];
    if (cell)
#pragma unroll
      for (int k = 0; k < NC; k++) ao[k] = A.q[kCellSlot[k]][c];
#pragma unroll
    for (int d = 0; d < NDIM; d++)
      if (fok[d]) fo[d] = A.q[5 + d][c];
    if (cell)
#pragma unroll
      for (int k = 0; k < NC; k++) A.q[kCellSlot[k]][c] = ao[k] + cv[k];
#pragma unroll
    for (int d = 0; d < NDIM; d++)
      if (fok[d]) A.q[5 + d][c] = fo[d] + fv[d];
  }
}
template <int NDIM>
static __global__ void adj_c2p_kernel(Grid g, F8 S, F8 P, F8 Pb, F8 A) {
  const long long total = (long long)g.ext[0] * g.ext[1] * g.ext[2];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    adj_c2p_item<NDIM>(g, S, P, Pb, A, id);
}


// Chain of the initial conserved cotangent to the initial primitives with p
// and B held: m = rho v, E = p/(G-1) + rho v^2/2 + B^2/2.
template <int NDIM>
static __global__ void adj_to_prim_kernel(Grid g, F8 A, F8 P, F8 out) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int i = (int)(id % g.n[0]);
    long long r = id / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    int c = g.at(i, j, k);
    const double rho = P.q[0][c], vx = P.q[1][c], vy = P.q[2][c], vz = P.q[3][c];
    const double ar = A.q[0][c], mx = A.q[1][c], my = A.q[2][c], mz = A.q[3][c], ae = A.q[4][c];
    const double v2 = (vx * vx + vy * vy) + vz * vz;
    out.q[0][c] = ((ar + ((mx * vx + my * vy) + mz * vz)) + 0.5 * ae * v2);
    out.q[1][c] = rho * (mx + ae * vx);
    out.q[2][c] = rho * (my + ae * vy);
    out.q[3][c] = rho * (mz + ae * vz);
  }
}

static __global__ void set_dt_only_kernel(DevScalars* sc, double dt) { sc->dt = dt; }
static __global__ void record_dt_kernel(const DevScalars* sc, double* dts, int n) { dts[n] = sc->dt; }

}  // namespace mhd
