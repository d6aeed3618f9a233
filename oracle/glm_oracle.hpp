// ORACLE — test infrastructure only (see oracle/mhd_oracle.hpp header).
//
// The scheme with hyperbolic-parabolic divergence cleaning (GLM) instead of
// constrained transport: the alternative div B control the paper uses for
// its strong-scaling runs (§2.1, citing Dedner et al. 2002 and Mignone et al.
// 2010; §4.1 and §4.2 "divergence cleaning").  The paper prints no formulas;
// this follows the mixed GLM formulation of those papers, with the readings
// stated where they are made:
//
//   dB/dt + div(v B - B v) + grad psi = 0,
//   dpsi/dt + c_h^2 div B = -(c_h^2 / c_p^2) psi,
//
// all variables cell-centred (9: rho, m, E, B, psi).  At each face the
// (B_n, psi) subsystem, linear with speeds -+c_h, is solved exactly:
//   B_m   = (B_n^L + B_n^R)/2 - (psi^R - psi^L) / (2 c_h),
//   psi_m = (psi^L + psi^R)/2 - c_h (B_n^R - B_n^L) / 2,
// its fluxes are psi_m (for B_n) and c_h^2 B_m (for psi), and the MHD
// Riemann solver (HLL / HLLD of mhd_oracle.hpp) runs with the normal field
// B_m on both sides.  The energy equation carries no psi term.
//   Reading 1 (c_h): the largest speed the step allows under the CFL
//     condition of the MHD waves, c_h = C / (dt sum_d 1/dx_d), constant over
//     the step.
//   Reading 2 (damping): the source is applied once per full step by its
//     exact solution, psi <- psi exp(-alpha c_h dt / dh), dh = min_d dx_d,
//     alpha = c_h dh / c_p^2 a configuration constant (default 0.1).
#pragma once
#include "mhd_oracle.hpp"

namespace orc {

// GLM state slots: conserved cell variables, the cell field and psi.
enum { G_RHO = 0, G_MX, G_MY, G_MZ, G_EN, G_BX, G_BY, G_BZ, G_PSI, NG };
// GLM primitives: rho, v, B, p, psi.
enum { GP_RHO = 0, GP_VX, GP_VY, GP_VZ, GP_BX, GP_BY, GP_BZ, GP_PR, GP_PSI, NGP };

template <class R> struct GlmSim {
  Config c{};
  double alpha = 0.1;
  int ndim = 2, G = 2;
  int n[3] = {1, 1, 1};
  double dx[3] = {1, 1, 1};
  bool periodic[3] = {true, true, true};
  std::array<Field<R>, NG> U0, U1, U2, Lq;
  Field<R> P[NGP];
  Field<R> Wp[9], Wm[9];  // reconstructed states of the current direction
  Field<R> Fx[NG];        // face fluxes of the current direction (face f at index f)
  R ch = R(0.0);  // cleaning speed of the current step
  R time = R(0.0);
  long long fallbacks = 0;
  int bad = 0;

  GlmSim(const Config& cfg, double alpha_) : c(cfg), alpha(alpha_) {
    ndim = cfg.ndim;
    if (ndim != 2 && ndim != 3) throw std::invalid_argument("ndim must be 2 or 3");
    G = cfg.recon == RECON_PLM ? 2 : 3;
    n[0] = cfg.nx; n[1] = cfg.ny; n[2] = ndim == 3 ? cfg.nz : 1;
    for (int d = 0; d < 3; d++) dx[d] = (cfg.x1[d] - cfg.x0[d]) / n[d];
    for (int d = 0; d < 3; d++) periodic[d] = cfg.bc[2 * d] == BC_PERIODIC;
    auto initf = [&](Field<R>& f) { f.init(n[0], n[1], n[2], G, ndim); };
    for (auto* S : {&U0, &U1, &U2, &Lq}) for (auto& f : *S) initf(f);
    for (auto& f : P) initf(f);
    for (auto& f : Wp) initf(f);
    for (auto& f : Wm) initf(f);
    for (auto& f : Fx) initf(f);
  }
  int lo(int d) const { return (d < ndim) ? -G : 0; }
  int hi(int d) const { return (d < ndim) ? n[d] + G : 0; }

  // Ghost cells: periodic axes first, then outflow (zero-gradient copies of
  // every variable), each pass over the full padded transverse range.
  void fill_ghosts(std::array<Field<R>, NG>& S) {
    for (int pass = 0; pass < 2; pass++)
      for (int d = 0; d < ndim; d++) {
        if ((pass == 0) != periodic[d]) continue;
        int t1 = (d + 1) % 3, t2 = (d + 2) % 3, N = n[d];
        for (int a = lo(t1); a <= hi(t1); a++)
          for (int b = lo(t2); b <= hi(t2); b++)
            for (int gi = -G; gi <= N + G; gi++) {
              if (gi >= 0 && gi < N) continue;
              int src = periodic[d] ? ((gi % N) + N) % N : (gi < 0 ? 0 : N - 1);
              int xd[3], xs[3];
              xd[t1] = a; xd[t2] = b; xd[d] = gi;
              xs[t1] = a; xs[t2] = b; xs[d] = src;
              for (int q = 0; q < NG; q++) S[q](xd[0], xd[1], xd[2]) = S[q](xs[0], xs[1], xs[2]);
            }
      }
  }

  void compute_prims(std::array<Field<R>, NG>& S) {
    g_flops.phase = PH_C2P;
    for (int k = lo(2); k < (ndim == 3 ? hi(2) : 1); k++)
      for (int j = lo(1); j < hi(1); j++)
        for (int i = lo(0); i < hi(0); i++) {
          R V[NP];
          cons_to_prim(S[G_RHO](i, j, k), S[G_MX](i, j, k), S[G_MY](i, j, k), S[G_MZ](i, j, k), S[G_EN](i, j, k),
                       S[G_BX](i, j, k), S[G_BY](i, j, k), S[G_BZ](i, j, k), c.gamma, V);
          for (int q = 0; q < NP; q++) P[q](i, j, k) = V[q];  // P_* and GP_* agree on the first 8 slots
          P[GP_PSI](i, j, k) = S[G_PSI](i, j, k);
          bool interior = i >= 0 && i < n[0] && j >= 0 && j < n[1] && k >= 0 && k < n[2];
          if (interior && (!(value(V[P_RHO]) > 0.0) || !(value(V[P_PR]) > 0.0))) bad = 1;
        }
  }

  // Reconstruction in direction d of the 9 sweep-frame primitives
  // (rho, v_n, v_t1, v_t2, B_n, B_t1, B_t2, p, psi) for cells [-1, n_d] of the
  // interior rows, with the positivity fallback of the CT scheme.
  void reconstruct(int d) {
    g_flops.phase = PH_RECON;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int comp[9] = {GP_RHO, GP_VX + d, GP_VX + t1, GP_VX + t2, GP_BX + d, GP_BX + t1, GP_BX + t2, GP_PR, GP_PSI};
    int ext[3] = {n[0], n[1], n[2]};
    for (int k = 0; k < ext[2]; k++)
      for (int j = 0; j < ext[1]; j++)
        for (int i = 0; i < ext[0]; i++) {
          int x[3] = {i, j, k};
          if (x[d] != 0) continue;  // one pencil per transverse position
          for (int cidx = -1; cidx <= n[d]; cidx++) {
            x[d] = cidx;
            R wp[9], wm[9], wc[9];
            for (int q = 0; q < 9; q++) {
              R s5[5];
              for (int m = -2; m <= 2; m++) {
                int y[3] = {x[0], x[1], x[2]};
                y[d] += m;
                bool need = c.recon != RECON_PLM || (m >= -1 && m <= 1);
                s5[m + 2] = need ? P[comp[q]](y[0], y[1], y[2]) : R(0.0);
              }
              wc[q] = s5[2];
              if (c.recon == RECON_PLM) recon_plm(s5, wp[q], wm[q]);
              else if (c.recon == RECON_WENOZ) recon_wenoz(s5, wp[q], wm[q]);
              else recon_ppm(s5, wp[q], wm[q]);
            }
            if (!(wp[0] > R(0.0)) || !(wm[0] > R(0.0)) || !(wp[7] > R(0.0)) || !(wm[7] > R(0.0))) {
              branch(51);
              for (int q = 0; q < 9; q++) wp[q] = wm[q] = wc[q];
              if (cidx >= 0 && cidx < n[d]) fallbacks++;
            }
            for (int q = 0; q < 9; q++) {
              Wp[q](x[0], x[1], x[2]) = wp[q];
              Wm[q](x[0], x[1], x[2]) = wm[q];
            }
          }
        }
  }

  // Face fluxes in direction d at faces [0, n_d] of the interior rows: the
  // exact (B_n, psi) solution, then the MHD solver with normal field B_m.
  void riemann(int d) {
    g_flops.phase = PH_RIEMANN;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++)
        for (int i = 0; i < n[0]; i++) {
          int x[3] = {i, j, k};
          if (x[d] != 0) continue;
          for (int f = 0; f <= n[d]; f++) {
            int xr[3] = {x[0], x[1], x[2]}, xl[3] = {x[0], x[1], x[2]};
            xr[d] = f;
            xl[d] = f - 1;
            R WL[9], WR[9];
            for (int q = 0; q < 9; q++) {
              WL[q] = Wp[q](xl[0], xl[1], xl[2]);
              WR[q] = Wm[q](xr[0], xr[1], xr[2]);
            }
            R Bm = R(0.5) * (WL[4] + WR[4]) - (WR[8] - WL[8]) / (R(2.0) * ch);
            R psim = R(0.5) * (WL[8] + WR[8]) - R(0.5) * ch * (WR[4] - WL[4]);
            R wl7[NW] = {WL[0], WL[1], WL[2], WL[3], WL[5], WL[6], WL[7]};
            R wr7[NW] = {WR[0], WR[1], WR[2], WR[3], WR[5], WR[6], WR[7]};
            R F7[NW], ing[NI];
            if (c.riemann == RS_HLLD) riemann_hlld(wl7, wr7, Bm, c.gamma, F7, ing);
            else riemann_hll(wl7, wr7, Bm, c.gamma, F7, ing);
            Fx[G_RHO](xr[0], xr[1], xr[2]) = F7[W_RHO];
            Fx[G_MX + d](xr[0], xr[1], xr[2]) = F7[W_VN];
            Fx[G_MX + t1](xr[0], xr[1], xr[2]) = F7[W_VT1];
            Fx[G_MX + t2](xr[0], xr[1], xr[2]) = F7[W_VT2];
            Fx[G_EN](xr[0], xr[1], xr[2]) = F7[W_PR];  // the energy flux sits in the last sweep slot
            Fx[G_BX + d](xr[0], xr[1], xr[2]) = psim;
            Fx[G_BX + t1](xr[0], xr[1], xr[2]) = F7[W_BT1];
            Fx[G_BX + t2](xr[0], xr[1], xr[2]) = F7[W_BT2];
            Fx[G_PSI](xr[0], xr[1], xr[2]) = (ch * ch) * Bm;
          }
        }
  }

  // One stage increment L(S) (Eq. FV with the GLM fluxes), dt included.
  void stage_increment(std::array<Field<R>, NG>& S, R dt) {
    g_flops.phase = PH_GHOST;
    fill_ghosts(S);
    compute_prims(S);
    for (int d = 0; d < ndim; d++) {
      reconstruct(d);
      riemann(d);
      g_flops.phase = PH_FLUXDIFF;
      const R dtdx = dt / R(dx[d]);
      for (int k = 0; k < n[2]; k++)
        for (int j = 0; j < n[1]; j++)
          for (int i = 0; i < n[0]; i++) {
            int xp[3] = {i, j, k};
            xp[d] += 1;
            for (int q = 0; q < NG; q++) {
              R term = -(dtdx * (Fx[q](xp[0], xp[1], xp[2]) - Fx[q](i, j, k)));
              Lq[q](i, j, k) = d == 0 ? term : Lq[q](i, j, k) + term;
            }
          }
    }
  }

  template <class Fn> void each_cell(Fn fn) {
    for (int q = 0; q < NG; q++)
      for (int k = 0; k < n[2]; k++)
        for (int j = 0; j < n[1]; j++)
          for (int i = 0; i < n[0]; i++) fn(q, i, j, k);
  }

  // Cleaning speed of a step of size dt (reading 1).
  R cleaning_speed(R dt) const {
    R s(0.0);
    for (int d = 0; d < ndim; d++) s = d == 0 ? R(1.0 / dx[d]) : s + R(1.0 / dx[d]);
    return R(c.cfl) / (dt * s);
  }

  // One step: SSP-RK2 / RK3 of the GLM system (Eq. RK3 with the reading of
  // its last weight), then the damping of psi (reading 2).
  void step(R dt) {
    ch = cleaning_speed(dt);
    stage_increment(U0, dt);
    g_flops.phase = PH_RK;
    each_cell([&](int q, int i, int j, int k) { U1[q](i, j, k) = U0[q](i, j, k) + Lq[q](i, j, k); });
    stage_increment(U1, dt);
    g_flops.phase = PH_RK;
    if (c.rk == 2) {
      each_cell([&](int q, int i, int j, int k) {
        U0[q](i, j, k) = R(0.5) * ((U0[q](i, j, k) + U1[q](i, j, k)) + Lq[q](i, j, k));
      });
    } else {
      each_cell([&](int q, int i, int j, int k) {
        U2[q](i, j, k) = R(0.25) * ((R(3.0) * U0[q](i, j, k) + U1[q](i, j, k)) + Lq[q](i, j, k));
      });
      stage_increment(U2, dt);
      g_flops.phase = PH_RK;
      each_cell([&](int q, int i, int j, int k) {
        U0[q](i, j, k) = ((U0[q](i, j, k) + R(2.0) * U2[q](i, j, k)) + R(2.0) * Lq[q](i, j, k)) / R(3.0);
      });
    }
    double dh = dx[0];
    for (int d = 1; d < ndim; d++) dh = dx[d] < dh ? dx[d] : dh;
    R decay = R(std::exp(-alpha * value(ch) * value(dt) / dh));
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++)
        for (int i = 0; i < n[0]; i++) U0[G_PSI](i, j, k) = U0[G_PSI](i, j, k) * decay;
    time = time + dt;
  }

  // CFL step of the MHD waves (as in the CT scheme, with the cell field).
  R cfl_dt() {
    fill_ghosts(U0);
    compute_prims(U0);
    g_flops.phase = PH_CFL;
    R lmax(0.0);
    R idx[3];
    for (int d = 0; d < 3; d++) idx[d] = R(1.0) / R(dx[d]);
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++)
        for (int i = 0; i < n[0]; i++) {
          R V[NP];
          for (int q = 0; q < NP; q++) V[q] = P[q](i, j, k);
          R lam = cfl_rate(V, idx, ndim, c.gamma);
          if (lmax < lam) lmax = lam;
        }
    return R(c.cfl) / lmax;
  }
};

}  // namespace orc
