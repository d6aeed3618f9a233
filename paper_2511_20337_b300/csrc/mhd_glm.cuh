// Kernels of the scheme with GLM divergence cleaning (the paper's
// alternative to constrained transport, §2.1 citing Dedner et al. 2002 and
// Mignone et al. 2010): cell-centred B and a scalar psi, the (B_n, psi)
// subsystem solved exactly at each face, the HLL/HLLD solver run with the
// resulting normal field B_m:
//   B_m   = (B_n^L + B_n^R)/2 - (psi^R - psi^L) / (2 c_h),
//   psi_m = (psi^L + psi^R)/2 - c_h (B_n^R - B_n^L) / 2,
//   fluxes: psi_m for B_n, c_h^2 B_m for psi.
// c_h = C / (dt sum_d 1/dx_d) (the largest speed the step's CFL condition
// allows); after each step psi <- psi exp(-alpha c_h dt / dh), dh = min dx.
// The energy equation carries no psi term.
//
// State: 9 cell-centred fields over the padded box (layout of
// mhd_kernels.cuh): rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi.
#pragma once
#include "mhd_kernels.cuh"

namespace mhd {

struct F9 { double* q[9]; };

// c_h of a step of size dt, in the order of the reading (IEEE operations).
__device__ __forceinline__ double glm_ch(const Grid& g, double dt) {
  double s = g.idx[0];
  for (int d = 1; d < g.ndim; d++) s = a_(s, g.idx[d]);
  return d_(g.cfl, m_(dt, s));
}

// Ghost cells along d: periodic wrap or zero-gradient copy of every field,
// over the full padded transverse range (periodic axes first, as in the CT
// scheme).
static __global__ void glm_ghost_kernel(Grid g, F9 S, int d) {
  const long long total = ghost_layers_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
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
    x[d] = g.periodic[d] ? wrap(gi, g.n[d]) : (gi < 0 ? 0 : g.n[d] - 1);
    int src = g.at(x[0], x[1], x[2]);
#pragma unroll
    for (int q = 0; q < 9; q++) S.q[q][dst] = S.q[q][src];
  }
}

// Primitives (rho, v, B, p, psi) of every padded cell; interior status and,
// with CFL, the rate reduced to dt as in the CT scheme.
template <int NDIM, bool CFL>
static __global__ void __launch_bounds__(256) glm_prim_kernel(Grid g, F9 S, F9 P, DevScalars* sc) {
  const long long total = prim_work<NDIM>(g);
  double lam_max = 0.0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int nxp = g.n[0] + 2 * g.G, nyp = g.n[1] + 2 * g.G;
    int i = (int)(id % nxp) - g.G;
    long long r = id / nxp;
    int j = (int)(r % nyp) - g.G;
    int k = NDIM == 3 ? (int)(r / nyp) - g.G : 0;
    int c = g.at(i, j, k);
    Prim8 V = c2p_ieee(S.q[0][c], S.q[1][c], S.q[2][c], S.q[3][c], S.q[4][c], S.q[5][c], S.q[6][c], S.q[7][c],
                       g.gm1);
    P.q[0][c] = V.rho;
    P.q[1][c] = V.vx;
    P.q[2][c] = V.vy;
    P.q[3][c] = V.vz;
    P.q[4][c] = V.bx;
    P.q[5][c] = V.by;
    P.q[6][c] = V.bz;
    P.q[7][c] = V.p;
    P.q[8][c] = S.q[8][c];
    const bool interior = i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && k >= 0 && k < g.n[2];
    if (interior) {
      if (!(V.rho > 0.0) || !(V.p > 0.0)) {
        long long flat = ((long long)k * g.n[1] + j) * g.n[0] + i;
        atomicExch(&sc->status, -4);
        atomicMin((unsigned long long*)&sc->bad_cell, (unsigned long long)flat);
      }
      if (CFL) {
        double B2 = a_(a_(m_(V.bx, V.bx), m_(V.by, V.by)), m_(V.bz, V.bz));
        double lam = m_(a_(dabs(V.vx), fast_speed_ieee(V.rho, V.p, B2, V.bx, g.gamma)), g.idx[0]);
        lam = a_(lam, m_(a_(dabs(V.vy), fast_speed_ieee(V.rho, V.p, B2, V.by, g.gamma)), g.idx[1]));
        if (NDIM == 3) lam = a_(lam, m_(a_(dabs(V.vz), fast_speed_ieee(V.rho, V.p, B2, V.bz, g.gamma)), g.idx[2]));
        lam_max = (lam > lam_max) ? lam : lam_max;
      }
    }
  }
  if (CFL) cfl_block_finish(lam_max, sc, g.cfl, gridDim.x);
}

// One sweep along DIR over the interior rows: each thread marches a segment
// of faces of one pencil (as the CT sweep), reconstructing the 9 sweep-frame
// primitives (rho, v_n, v_t1, v_t2, B_n, B_t1, B_t2, p, psi) of each cell
// once, solving each face once per segment and accumulating the flux
// difference of Eq. FV into the stage increment of all 9 variables.
template <int DIR, int NDIM>
__host__ __device__ __forceinline__ long long glm_sweep_work(const Grid& g, int seglen) {
  constexpr int U = (DIR == 0) ? 1 : 0;
  constexpr int V = (DIR == 0) ? 2 : (DIR == 1 ? 2 : 1);
  long long eu = (U < NDIM) ? g.n[U] : 1, ev = (V < NDIM) ? g.n[V] : 1;
  return eu * ev * ((g.n[DIR] + 1 + seglen - 1) / seglen);
}

template <int DIR, int NDIM, int RECON, int RS>
static __global__ void __launch_bounds__(128) glm_sweep_kernel(Grid g, F9 P, F9 L, DevScalars* sc, int seglen,
                                                                int accumulate) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int R = Stencil<RECON>::R;
  constexpr int W = 2 * R + 1;
  constexpr int U = (DIR == 0) ? 1 : 0;
  constexpr int V = (DIR == 0) ? 2 : (DIR == 1 ? 2 : 1);
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= glm_sweep_work<DIR, NDIM>(g, seglen)) return;
  const int eu = (U < NDIM) ? g.n[U] : 1, ev = (V < NDIM) ? g.n[V] : 1;
  const int iu = (int)(id % eu);
  const long long r = id / eu;
  const int iv = (int)(r % ev);
  const int seg = (int)(r / ev);
  int x[3];
  x[DIR] = 0;
  x[U] = iu;
  x[V] = iv;
  const int base = g.at(x[0], x[1], x[2]);
  const int st = g.stride(DIR);
  const int nd = g.n[DIR];
  const int f0 = seg * seglen;
  const int f1 = min(f0 + seglen, nd + 1);
  const int fend = min(f1, nd);
  const double dt = sc->dt;
  const double dtdx = fmul(dt, g.idx[DIR]);
  const double ch = glm_ch(g, dt);
  const double hich = kmul(RK_HALF, rcp(ch)), ch2 = fmul(ch, ch);
  const double* pr[9] = {P.q[0], P.q[1 + DIR], P.q[1 + T1], P.q[1 + T2], P.q[4 + DIR],
                         P.q[4 + T1], P.q[4 + T2], P.q[7], P.q[8]};
  double win[9][W];
#pragma unroll
  for (int m = 0; m < W; m++) {
    int c = base + (f0 - 1 - R + m) * st;
#pragma unroll
    for (int v = 0; v < 9; v++) win[v][m] = pr[v][c];
  }
  // PLM: the left difference of the window's centre cell, carried along the pencil
  double dl[9];
  if (RECON == RECON_PLM) {
#pragma unroll
    for (int v = 0; v < 9; v++) dl[v] = fsub(win[v][1], win[v][0]);
  }
  // WENO-Z: the curvatures of the stencils centred on the window's cells 1 and
  // 2 (their 13/12 multiples are formed again: nine variables' worth would not
  // fit in registers)
  double cv[9][2];
  if (RECON == RECON_WENOZ) {
#pragma unroll
    for (int v = 0; v < 9; v++) {
      cv[v][0] = curv(win[v][0], win[v][1], win[v][2]).t;
      cv[v][1] = curv(win[v][1], win[v][2], win[v][3]).t;
    }
  }
  auto reconstruct = [&](double plus[9], double minus[9], bool count) {
#pragma unroll
    for (int v = 0; v < 9; v++) {
      if (RECON == RECON_PLM) {
        const double dr = fsub(win[v][2], win[v][1]);
        recon_plm_d(win[v][1], dl[v], dr, plus[v], minus[v]);
        dl[v] = dr;
      }
      else if (RECON == RECON_WENOZ) {
        Curv c2;
        recon_wenoz_c(win[v][0], win[v][1], win[v][2], win[v][3], win[v][4], curv_of(cv[v][0]), curv_of(cv[v][1]), c2,
                      plus[v], minus[v]);
        cv[v][0] = cv[v][1];
        cv[v][1] = c2.t;
      }
      else recon_ppm(win[v][0], win[v][1], win[v][2], win[v][3], win[v][4], plus[v], minus[v]);
    }
    if (!gt0(plus[0]) || !gt0(minus[0]) || !gt0(plus[7]) || !gt0(minus[7])) {
#pragma unroll
      for (int v = 0; v < 9; v++) plus[v] = minus[v] = win[v][R];
      if (count) atomicAdd(&sc->fallbacks, 1ull);
    }
  };
  double wl[9], wr[9], dummy[9];
  reconstruct(wl, dummy, false);  // cell f0 - 1: a ghost or another segment's cell
  double Fprev[9];
  for (int f = f0; f <= fend; f++) {
#pragma unroll
    for (int v = 0; v < 9; v++) {
#pragma unroll
      for (int m = 0; m < W - 1; m++) win[v][m] = win[v][m + 1];
    }
    {
      int c = base + (f + R) * st;
#pragma unroll
      for (int v = 0; v < 9; v++) win[v][W - 1] = pr[v][c];
    }
    double plusN[9];
    reconstruct(plusN, wr, f < f1 && f < nd);  // cell f, counted once by the segment owning face f
    // the (B_n, psi) subsystem
    const double Bm = fma(rk(RK_HALF), fadd(wl[4], wr[4]), -fmul(fsub(wr[8], wl[8]), hich));
    const double psim = fma(rk(RK_HALF), fadd(wl[8], wr[8]), -fmul(kmul(RK_HALF, ch), fsub(wr[4], wl[4])));
    W7 L7 = {wl[0], wl[1], wl[2], wl[3], wl[5], wl[6], wl[7]};
    W7 R7 = {wr[0], wr[1], wr[2], wr[3], wr[5], wr[6], wr[7]};
    Flux7 F7;
    Ingr ing;
    if (RS == RS_HLLD) riemann_hlld(L7, R7, Bm, g.gamma, g.igm1, F7, ing);
    else riemann_hll(L7, R7, Bm, g.gamma, g.igm1, F7, ing);
    // fluxes of the 9 conserved variables in state order
    double F[9];
    F[0] = F7.f[0];
    F[1 + DIR] = F7.f[1];
    F[1 + T1] = F7.f[2];
    F[1 + T2] = F7.f[3];
    F[4] = F7.f[6];
    F[5 + DIR] = psim;
    F[5 + T1] = F7.f[4];
    F[5 + T2] = F7.f[5];
    F[8] = fmul(ch2, Bm);
    if (f > f0) {
      const int cc = base + (f - 1) * st;  // cell f - 1
#pragma unroll
      for (int q = 0; q < 9; q++) {
        const double dv = fsub(F[q], Fprev[q]);
        L.q[q][cc] = accumulate ? fma(-dtdx, dv, L.q[q][cc]) : -fmul(dtdx, dv);
      }
    }
#pragma unroll
    for (int q = 0; q < 9; q++) Fprev[q] = F[q];
#pragma unroll
    for (int v = 0; v < 9; v++) wl[v] = plusN[v];
  }
}

// RK combine of every interior cell and field (combine() of mhd_kernels.cuh);
// after the last stage psi is damped by exp(-alpha c_h dt / dh).
template <int NDIM>
static __global__ void __launch_bounds__(256) glm_combine_kernel(Grid g, F9 U0, F9 Us, F9 Out, F9 L,
                                                                  const DevScalars* sc, int mode, int last,
                                                                  double alpha, double dh) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  const double dt = sc->dt;
  const double decay = last ? exp(-alpha * glm_ch(g, dt) * dt / dh) : 1.0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int i = (int)(id % g.n[0]);
    long long r = id / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    int c = g.at(i, j, k);
#pragma unroll
    for (int q = 0; q < 9; q++) {
      double v = combine(mode, U0.q[q][c], Us.q[q][c], L.q[q][c]);
      Out.q[q][c] = (q == 8 && last) ? v * decay : v;
    }
  }
}

// Primitive -> conserved in place on interior cells (slots 0..4 hold rho, v,
// p on entry; slots 5..7 the cell field).
template <int NDIM>
static __global__ void glm_prim_to_cons_kernel(Grid g, F9 S) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int i = (int)(id % g.n[0]);
    long long r = id / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    int c = g.at(i, j, k);
    double bx = S.q[5][c], by = S.q[6][c], bz = S.q[7][c];
    double rho = S.q[0][c], vx = S.q[1][c], vy = S.q[2][c], vz = S.q[3][c], p = S.q[4][c];
    S.q[1][c] = rho * vx;
    S.q[2][c] = rho * vy;
    S.q[3][c] = rho * vz;
    S.q[4][c] = fma(p, g.igm1, fma(0.5 * rho, fma(vx, vx, fma(vy, vy, vz * vz)), 0.5 * fma(bx, bx, fma(by, by, bz * bz))));
  }
}

}  // namespace mhd
