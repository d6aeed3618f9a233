// ============================================================================
// ORACLE — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded FP64 CPU implementation of one finite-volume
// time step of ideal MHD on a uniform Cartesian grid with constrained transport,
// written from the method's mathematics (paper §2: Eq. cons_law, Eq. mhd,
// Eq. Energy, Eq. FV, Eq. RK3, Eq. reconstruct, the primitive-recovery and
// Riemann-flux equations of §2.2).  It exists to check the CUDA library against.
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
// it.  It shares no code with the CUDA path.
//
// Every function is written in the order of the formula it follows; nothing is
// fused, blocked or reordered for speed.  Where the paper is silent the reading
// taken is stated at the function.
//
// Parity pins (tests/test_oracle_*.py): closed forms, exact Riemann solutions,
// conservation, div B, symmetries, convergence orders.  No paper-printed values
// exist for this method (the paper prints performance only), so paper-value
// parity is unpinned; the mathematical pins replace it.
// ============================================================================
#pragma once
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <vector>

#include "scalar.hpp"

namespace orc {

using std::fabs;
using std::sqrt;

enum { RECON_PLM = 0, RECON_WENOZ = 1, RECON_PPM = 2 };
enum { RS_HLL = 0, RS_HLLD = 1 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };
// Edge-field weights (the paper names the UCT-HLLD average for its benchmarks):
// the UCT form with HLL coefficients, or with the HLLD solver's own coefficients.
enum { EMF_UCT_HLL = 0, EMF_UCT_HLLD = 1 };

// Thresholds of the degenerate HLLD branches (reading: the paper is silent).
constexpr double HLLD_DEGEN_EPS = 1e-12;  // |D_a| below this * rho_a (S_a-u_a)(S_a-S_M)
constexpr double HLLD_BN_EPS = 1e-12;     // Bn^2/2 below this * pT*: no rotational waves
constexpr double WENOZ_EPS = 1e-40;       // WENO-Z epsilon (reading)

struct Config {
  int ndim;
  int nx, ny, nz;
  double x0[3], x1[3];
  double gamma;
  int recon, riemann, rk;
  double cfl;
  int bc[6];  // x-, x+, y-, y+, z-, z+
  double p_floor;  // floor on the recovered pressure (0: none)
  int emf;         // EMF_UCT_HLL or EMF_UCT_HLLD (needs the HLLD solver)
};

// For the branch signature, min/max of (nearly) equal arguments is one
// neutral decision: the two arguments are then usually the same function
// (e.g. u_L = u_R = (u_i + u_i+1)/2 when both cells take the shared slope),
// so which one is returned changes neither the value nor the derivative.
template <class R> inline bool near_tie(R a, R b) {
  double x = value(a), y = value(b);
  return std::fabs(x - y) <= 1e-12 * (std::fabs(x) + std::fabs(y));
}
template <class R> inline R rmin(R a, R b) {
  bool sb = b < a;
  branch(near_tie(a, b) ? 10 : (sb ? 11 : 12));
  return sb ? b : a;
}
template <class R> inline R rmax(R a, R b) {
  bool sb = a < b;
  branch(near_tie(a, b) ? 10 : (sb ? 13 : 14));
  return sb ? b : a;
}
// |x| where the kink at 0 is a branch of the scheme
template <class R> inline R rabs(R x) {
  branch(x < R(0.0) ? 15 : 16);
  return fabs(x);
}

// minmod(a, b): 0 if a*b <= 0, else the argument of smaller magnitude; on a tie
// |a| == |b| the first argument is returned (both are equal then).
template <class R> inline R minmod(R a, R b) {
  const R zero(0.0);
  if ((a > zero && b > zero) || (a < zero && b < zero)) {
    bool sb = fabs(b) < fabs(a);
    branch(sb ? 1 : 2);
    return sb ? b : a;
  }
  branch(3);
  return zero;
}

// ---------------------------------------------------------------------------
// Padded field: indices i in [-G, nx+G], j in [-G, ny+G], k in [-G, nz+G]
// (k in [0,0] in 2D).  The extra slot at n+G holds the outermost face of a
// face-centred array.  Face arrays store, at index i, the face at x0 + i*dx
// (the left face of cell i).
// ---------------------------------------------------------------------------
template <class R> struct Field {
  int G = 0, Gz = 0, ex = 0, ey = 0, ez = 0;
  std::vector<R> a;
  void init(int nx, int ny, int nz, int g, int ndim) {
    G = g;
    Gz = ndim == 3 ? g : 0;
    ex = nx + 2 * g + 1;
    ey = ny + 2 * g + 1;
    ez = ndim == 3 ? nz + 2 * g + 1 : 1;
    a.assign((size_t)ex * ey * ez, R(0.0));
  }
  R& operator()(int i, int j, int k) { return a[((size_t)(k + Gz) * ey + (j + G)) * ex + (i + G)]; }
  const R& operator()(int i, int j, int k) const { return a[((size_t)(k + Gz) * ey + (j + G)) * ex + (i + G)]; }
};

// State slots.  Cell-centred conserved variables (Eq. mhd): rho, m = rho v, E.
// 3D: slots 5,6,7 are the staggered face fields Bx, By, Bz.
// 2D: slots 5,6 are the face fields Bx, By; slot 7 is the cell-centred Bz,
//     evolved by finite-volume fluxes like rho, m and E.
enum { Q_RHO = 0, Q_MX, Q_MY, Q_MZ, Q_EN, Q_B0, Q_B1, Q_B2, NQ };
// Primitive slots (Eq. reconstruct: V = {rho, v, B, p}), cell-centred.
enum { P_RHO = 0, P_VX, P_VY, P_VZ, P_BX, P_BY, P_BZ, P_PR, NP };
// Reconstructed / Riemann variables in the frame of a sweep with normal n and
// cyclic transverse directions t1 = (n+1)%3, t2 = (n+2)%3.
enum { W_RHO = 0, W_VN, W_VT1, W_VT2, W_BT1, W_BT2, W_PR, NW };
// Face ingredients kept for the UCT electric field: the weights a^L, a^R of the
// two sides' induction fluxes, the dissipation coefficients d^L, d^R of their
// transverse fields and the reconstructed normal velocities, such that the
// flux of either transverse field component B_t at the face is
//   a^L F_L + a^R F_R + d^L B_t,L - d^R B_t,R,   F = u B_t - v_t B_n.
// UCT-HLL: a^L = a+, a^R = a-, d^L = d^R = d (I_DR repeats I_DD).
enum { I_AP = 0, I_AM, I_DD, I_UL, I_UR, I_DR, NI };

template <class R> using State = std::array<Field<R>, NQ>;

// ---------------------------------------------------------------------------
// Pointwise physics
// ---------------------------------------------------------------------------

// Fast magnetosonic speed along a direction with normal field Bn (§2.1 system):
//   cf^2 = [ (G p + B^2) + sqrt((G p + B^2)^2 - 4 G p Bn^2) ] / (2 rho).
// The discriminant is >= 0 analytically; round-off below zero is clamped to 0.
template <class R> inline R fast_speed(R rho, R p, R B2, R Bn, double gamma) {
  R gp = R(gamma) * p;
  R s = gp + B2;
  R disc = s * s - (R(4.0) * gp) * (Bn * Bn);
  if (disc < R(0.0)) {
    disc = R(0.0);
    branch(17);
  }
  R cf2 = (R(0.5) * (s + sqrt(disc))) / rho;
  return sqrt(cf2);
}

// Conservative -> primitive recovery (§2.2, unnumbered equation after
// Eq. reconstruct; Eq. Energy):  v = m / rho,
//   p = (G - 1) (E - rho v^2 / 2 - B^2 / 2),
// with the cell-centred field given.  1/rho is formed once.
template <class R>
inline void cons_to_prim(R rho, R mx, R my, R mz, R en, R bx, R by, R bz, double gamma, R V[NP]) {
  R inv = R(1.0) / rho;
  R vx = mx * inv, vy = my * inv, vz = mz * inv;
  R kin = R(0.5) * ((mx * vx + my * vy) + mz * vz);
  R B2 = (bx * bx + by * by) + bz * bz;
  R p = R(gamma - 1.0) * ((en - kin) - R(0.5) * B2);
  V[P_RHO] = rho; V[P_VX] = vx; V[P_VY] = vy; V[P_VZ] = vz;
  V[P_BX] = bx; V[P_BY] = by; V[P_BZ] = bz; V[P_PR] = p;
}

// Conserved state and physical flux of Eq. mhd in a sweep frame (normal n):
// U = (rho, rho u, rho v, rho w, Bt1, Bt2, E),
// F = (rho u, rho u^2 + pT - Bn^2, rho u v - Bn Bt1, rho u w - Bn Bt2,
//      u Bt1 - v Bn, u Bt2 - w Bn, (E + pT) u - Bn (v.B)),  pT = p + B^2/2.
// The flux of the normal field component is identically zero.
template <class R> struct SideState {
  R U[NW], F[NW];
  R pT, B2, vB, E;
};
template <class R> inline SideState<R> side_state(const R W[NW], R bn, double gamma) {
  SideState<R> s;
  R rho = W[W_RHO], u = W[W_VN], v = W[W_VT1], w = W[W_VT2];
  R b1 = W[W_BT1], b2 = W[W_BT2], p = W[W_PR];
  s.B2 = (bn * bn + b1 * b1) + b2 * b2;
  s.pT = p + R(0.5) * s.B2;
  s.vB = (u * bn + v * b1) + w * b2;
  R v2 = (u * u + v * v) + w * w;
  s.E = (p / R(gamma - 1.0) + R(0.5) * rho * v2) + R(0.5) * s.B2;
  s.U[0] = rho; s.U[1] = rho * u; s.U[2] = rho * v; s.U[3] = rho * w;
  s.U[4] = b1; s.U[5] = b2; s.U[6] = s.E;
  s.F[0] = rho * u;
  s.F[1] = (rho * u * u + s.pT) - bn * bn;
  s.F[2] = rho * u * v - bn * b1;
  s.F[3] = rho * u * w - bn * b2;
  s.F[4] = u * b1 - v * bn;
  s.F[5] = u * b2 - w * bn;
  s.F[6] = (s.E + s.pT) * u - bn * s.vB;
  return s;
}

// Outer signal speeds shared by HLL and HLLD (Miyoshi & Kusano 2005 estimate):
//   S_L = min(u_L, u_R) - max(cf_L, cf_R),  S_R = max(u_L, u_R) + max(cf_L, cf_R).
// Also the UCT ingredients (reading of the UCT-HLL electric field):
//   aR = max(0, S_R), aL = min(0, S_L),
//   a+ = aR / (aR - aL), a- = -aL / (aR - aL), d = -aR aL / (aR - aL),
//   plus the reconstructed normal velocities u_L and u_R.
template <class R>
inline void signal_speeds(const R WL[NW], const R WR[NW], const SideState<R>& L, const SideState<R>& Rs, R bn,
                          double gamma, R& SL, R& SR, R ing[NI]) {
  R cfL = fast_speed(WL[W_RHO], WL[W_PR], L.B2, bn, gamma);
  R cfR = fast_speed(WR[W_RHO], WR[W_PR], Rs.B2, bn, gamma);
  R cmax = rmax(cfL, cfR);
  SL = rmin(WL[W_VN], WR[W_VN]) - cmax;
  SR = rmax(WL[W_VN], WR[W_VN]) + cmax;
  R aR = rmax(R(0.0), SR), aL = rmin(R(0.0), SL);
  R inv = R(1.0) / (aR - aL);
  ing[I_AP] = aR * inv;
  ing[I_AM] = -(aL * inv);
  ing[I_DD] = -((aR * aL) * inv);
  ing[I_UL] = WL[W_VN];
  ing[I_UR] = WR[W_VN];
  ing[I_DR] = ing[I_DD];
}

// HLL flux (Harten, Lax & van Leer; the dissipative form of the Riemann flux in §2.2):
//   F = (aR F_L - aL F_R + aR aL (U_R - U_L)) / (aR - aL), with upwind limits.
template <class R>
inline void riemann_hll(const R WL[NW], const R WR[NW], R bn, double gamma, R F[NW], R ing[NI]) {
  SideState<R> L = side_state(WL, bn, gamma), Rs = side_state(WR, bn, gamma);
  R SL, SR;
  signal_speeds(WL, WR, L, Rs, bn, gamma, SL, SR, ing);
  if (SL >= R(0.0)) { branch(21); for (int q = 0; q < NW; q++) F[q] = L.F[q]; return; }
  if (SR <= R(0.0)) { branch(22); for (int q = 0; q < NW; q++) F[q] = Rs.F[q]; return; }
  branch(23);
  R inv = R(1.0) / (SR - SL);
  for (int q = 0; q < NW; q++)
    F[q] = ((SR * L.F[q] - SL * Rs.F[q]) + (SR * SL) * (Rs.U[q] - L.U[q])) * inv;
}

// HLLD flux (Miyoshi & Kusano 2005), restated from its mathematics: five waves
// S_L < S*_L < S_M < S*_R < S_R separating U_L, U*_L, U**_L, U**_R, U*_R, U_R;
// normal velocity and total pressure continuous across the fan.
//
// With uct_hlld the UCT ingredients are the HLLD solver's own coefficients
// (reading of the UCT-HLLD average; the paper cites it without formulas).
// In every region of the fan the flux of a transverse field component B_t is
// linear in the two sides' (v_t, B_t), with coefficients made of the wave
// speeds, rho* and the star ratio e = B*_t / B_t (the same for both
// components).  Written in the form a^L F_L + a^R F_R + d^L B_t,L - d^R B_t,R:
//   0 <= S_L:              a^L = 1, a^R = 0, d^L = d^R = 0;
//   S_L < 0 <= S*_L:       a^L = 1, a^R = 0, d^L = S_L (e_L - 1), d^R = 0;
//   S*_L < 0 <= S*_R:      a^L = S*_R / (S*_R - S*_L), a^R = -S*_L / (S*_R - S*_L),
//                          d^L = a^L ((S_L - S*_L) e_L - S_L),
//                          d^R = a^R (S_R - (S_R - S*_R) e_R);
//   S*_R < 0 <= S_R:       a^L = 0, a^R = 1, d^L = 0, d^R = S_R (1 - e_R);
//   S_R < 0:               a^L = 0, a^R = 1, d^L = d^R = 0.
// (The double-star row follows from the double-star transverse states, in
// which v_t,L enters with weight -sgn(B_n) sqrt(rho*_L rho*_R) S*_R / (sqrt(rho*_L) + sqrt(rho*_R)),
// i.e. -B_n a^L with S*_R - S*_L = |B_n| (1/sqrt(rho*_L) + 1/sqrt(rho*_R)).)
template <class R>
inline void riemann_hlld(const R WL[NW], const R WR[NW], R bn, double gamma, R F[NW], R ing[NI],
                         bool uct_hlld = false) {
  SideState<R> L = side_state(WL, bn, gamma), Rs = side_state(WR, bn, gamma);
  R SL, SR;
  signal_speeds(WL, WR, L, Rs, bn, gamma, SL, SR, ing);
  auto set_weights = [&](R aL, R aR, R dL, R dR) {
    if (!uct_hlld) return;
    ing[I_AP] = aL; ing[I_AM] = aR; ing[I_DD] = dL; ing[I_DR] = dR;
  };
  if (SL > R(0.0)) {
    branch(31);
    for (int q = 0; q < NW; q++) F[q] = L.F[q];
    set_weights(R(1.0), R(0.0), R(0.0), R(0.0));
    return;
  }
  if (SR < R(0.0)) {
    branch(32);
    for (int q = 0; q < NW; q++) F[q] = Rs.F[q];
    set_weights(R(0.0), R(1.0), R(0.0), R(0.0));
    return;
  }

  const R zero(0.0);
  R rhoL = WL[W_RHO], uL = WL[W_VN], rhoR = WR[W_RHO], uR = WR[W_VN];
  R sdL = SL - uL, sdR = SR - uR;
  // Middle (contact) speed and star total pressure.
  R den = sdR * rhoR - sdL * rhoL;
  R SM = (((sdR * rhoR) * uR - (sdL * rhoL) * uL) - Rs.pT + L.pT) / den;
  R pTs = (((sdR * rhoR) * L.pT - (sdL * rhoL) * Rs.pT) + ((rhoL * rhoR) * (sdR * sdL)) * (uR - uL)) / den;

  // Star states on each side.
  struct Star { R rho, v, w, b1, b2, E, vB, S, e; };  // e = B*_t / B_t
  auto star = [&](const R W[NW], const SideState<R>& s, R S) {
    Star o;
    R rho = W[W_RHO], u = W[W_VN], v = W[W_VT1], w = W[W_VT2], b1 = W[W_BT1], b2 = W[W_BT2];
    R sd = S - u, sm = S - SM;
    o.rho = (rho * sd) / sm;
    R rsm = (rho * sd) * sm;
    R D = rsm - bn * bn;
    if (fabs(D) < R(HLLD_DEGEN_EPS) * rsm) {
      branch(33);
      o.v = v; o.w = w; o.b1 = b1; o.b2 = b2;
      o.e = R(1.0);
    } else {
      R invD = R(1.0) / D;
      R cv = (bn * (SM - u)) * invD;
      o.v = v - b1 * cv;
      o.w = w - b2 * cv;
      R cb = ((rho * sd) * sd - bn * bn) * invD;
      o.b1 = b1 * cb;
      o.b2 = b2 * cb;
      o.e = cb;
    }
    o.vB = (SM * bn + o.v * o.b1) + o.w * o.b2;
    o.E = (((sd * s.E - s.pT * u) + pTs * SM) + bn * (s.vB - o.vB)) / sm;
    o.S = S;
    return o;
  };
  Star sL = star(WL, L, SL), sR = star(WR, Rs, SR);
  auto Ustar = [&](const Star& o, R v, R w, R b1, R b2, R E, R out[NW]) {
    out[0] = o.rho; out[1] = o.rho * SM; out[2] = o.rho * v; out[3] = o.rho * w;
    out[4] = b1; out[5] = b2; out[6] = E;
  };
  R UsL[NW], UsR[NW];
  Ustar(sL, sL.v, sL.w, sL.b1, sL.b2, sL.E, UsL);
  Ustar(sR, sR.v, sR.w, sR.b1, sR.b2, sR.E, UsR);

  // Rotational (Alfven) waves; absent when the normal field vanishes.
  R SsL = SM, SsR = SM;
  R UssL[NW], UssR[NW];
  bool rot = !(R(0.5) * (bn * bn) < R(HLLD_BN_EPS) * pTs);
  branch(rot ? 34 : 35);
  if (rot) {
    R sqL = sqrt(sL.rho), sqR = sqrt(sR.rho);
    SsL = SM - rabs(bn) / sqL;
    SsR = SM + rabs(bn) / sqR;
    R sgn = bn > zero ? R(1.0) : R(-1.0);
    R inv = R(1.0) / (sqL + sqR);
    R vss = ((sqL * sL.v + sqR * sR.v) + (sR.b1 - sL.b1) * sgn) * inv;
    R wss = ((sqL * sL.w + sqR * sR.w) + (sR.b2 - sL.b2) * sgn) * inv;
    R b1ss = ((sqL * sR.b1 + sqR * sL.b1) + ((sqL * sqR) * (sR.v - sL.v)) * sgn) * inv;
    R b2ss = ((sqL * sR.b2 + sqR * sL.b2) + ((sqL * sqR) * (sR.w - sL.w)) * sgn) * inv;
    R vBss = (SM * bn + vss * b1ss) + wss * b2ss;
    R EssL = sL.E - (sqL * (sL.vB - vBss)) * sgn;
    R EssR = sR.E + (sqR * (sR.vB - vBss)) * sgn;
    Ustar(sL, vss, wss, b1ss, b2ss, EssL, UssL);
    Ustar(sR, vss, wss, b1ss, b2ss, EssR, UssR);
  }

  // Flux at x/t = 0 from the wave fan, Rankine-Hugoniot across each wave.
  branch(SsL >= zero ? 36 : (SM >= zero ? 37 : (SsR >= zero ? 38 : 39)));
  if (SsL >= zero) {  // S_L <= 0 <= S*_L
    for (int q = 0; q < NW; q++) F[q] = L.F[q] + SL * (UsL[q] - L.U[q]);
  } else if (SM >= zero) {  // S*_L <= 0 <= S_M
    for (int q = 0; q < NW; q++) {
      R FsL = L.F[q] + SL * (UsL[q] - L.U[q]);
      F[q] = FsL + SsL * (UssL[q] - UsL[q]);
    }
  } else if (SsR >= zero) {  // S_M < 0 <= S*_R
    for (int q = 0; q < NW; q++) {
      R FsR = Rs.F[q] + SR * (UsR[q] - Rs.U[q]);
      F[q] = FsR + SsR * (UssR[q] - UsR[q]);
    }
  } else {  // S*_R < 0 <= S_R
    for (int q = 0; q < NW; q++) F[q] = Rs.F[q] + SR * (UsR[q] - Rs.U[q]);
  }
  if (!uct_hlld) return;
  if (SsL >= zero) {
    set_weights(R(1.0), zero, SL * (sL.e - R(1.0)), zero);
  } else if (SsR >= zero) {  // only with rotational waves: S*_L < 0 <= S*_R
    R aL = SsR / (SsR - SsL), aR = -SsL / (SsR - SsL);
    set_weights(aL, aR, aL * ((SL - SsL) * sL.e - SL), aR * (SR - (SR - SsR) * sR.e));
  } else {
    set_weights(zero, R(1.0), zero, SR * (R(1.0) - sR.e));
  }
}

// ---------------------------------------------------------------------------
// Reconstruction of one variable (Eq. reconstruct).  s[m] = V_{i+m-2},
// m = 0..4 (PLM uses s[1..3]).  Returns V^L_{i+1/2} (plus) and V^R_{i-1/2} (minus).
// ---------------------------------------------------------------------------

// Piecewise-linear with the minmod limiter.
template <class R> inline void recon_plm(const R s[5], R& plus, R& minus) {
  R d = minmod(s[2] - s[1], s[3] - s[2]);
  plus = s[2] + R(0.5) * d;
  minus = s[2] - R(0.5) * d;
}

// Fifth-order WENO-Z (Borges et al. 2008) value at the right face of the middle
// cell of a 5-point stencil a[0..4] = V_{i-2..i+2}: candidate third-order
// values q_k, Jiang-Shu smoothness indicators beta_k, tau5 = |beta_0 - beta_2|,
// alpha_k = d_k (1 + (tau5 / (beta_k + eps))^2), d = (1/10, 6/10, 3/10).
// Readings: eps = 1e-40, exponent 2, applied componentwise to primitives.
//
// The indicators, tau5, the ratios tau5 / (beta_k + eps) and the factors
// 1 + ratio^2 depend only on the five cell values, not on the face: the
// mirrored stencil of the cell's left face has the same ones with beta_0 and
// beta_2 exchanged.  wenoz_shared forms them (one face's worth, as the formula
// states them); wenoz_face calls it for each face.  The flop count of
// wenoz_shared is what an implementation that forms them once per cell saves.
template <class R> inline void wenoz_shared(R a0, R a1, R a2, R a3, R a4, R& h0, R& h1, R& h2) {
  R t;
  t = (a0 - R(2.0) * a1) + a2;
  R u = (a0 - R(4.0) * a1) + R(3.0) * a2;
  R b0 = R(13.0 / 12.0) * (t * t) + R(0.25) * (u * u);
  t = (a1 - R(2.0) * a2) + a3;
  u = a1 - a3;
  R b1 = R(13.0 / 12.0) * (t * t) + R(0.25) * (u * u);
  t = (a2 - R(2.0) * a3) + a4;
  u = (R(3.0) * a2 - R(4.0) * a3) + a4;
  R b2 = R(13.0 / 12.0) * (t * t) + R(0.25) * (u * u);
  R tau = rabs(b0 - b2);
  R r0 = tau / (b0 + R(WENOZ_EPS));
  R r1 = tau / (b1 + R(WENOZ_EPS));
  R r2 = tau / (b2 + R(WENOZ_EPS));
  h0 = R(1.0) + r0 * r0;
  h1 = R(1.0) + r1 * r1;
  h2 = R(1.0) + r2 * r2;
}
template <class R> inline R wenoz_face(R a0, R a1, R a2, R a3, R a4) {
  R q0 = ((R(2.0) * a0 - R(7.0) * a1) + R(11.0) * a2) / R(6.0);
  R q1 = ((-a1 + R(5.0) * a2) + R(2.0) * a3) / R(6.0);
  R q2 = ((R(2.0) * a2 + R(5.0) * a3) - a4) / R(6.0);
  R h0, h1, h2;
  wenoz_shared(a0, a1, a2, a3, a4, h0, h1, h2);
  R al0 = R(0.1) * h0;
  R al1 = R(0.6) * h1;
  R al2 = R(0.3) * h2;
  R sum = (al0 + al1) + al2;
  return ((al0 * q0 + al1 * q1) + al2 * q2) / sum;
}
template <class R> inline void recon_wenoz(const R s[5], R& plus, R& minus) {
  plus = wenoz_face(s[0], s[1], s[2], s[3], s[4]);
  minus = wenoz_face(s[4], s[3], s[2], s[1], s[0]);
}

// Piecewise-parabolic (Colella & Woodward 1984) in method-of-lines form, no
// characteristic tracing (reading).  Fourth-order face value
//   V_{i+1/2} = 7/12 (V_i + V_{i+1}) - 1/12 (V_{i-1} + V_{i+2}),
// clipped to the range of its two neighbours, then the CW84 monotonicity
// constraints on the parabola of cell i.
template <class R> inline R ppm_face(R a, R b, R c, R d) {  // a=V_{i-1}, b=V_i, c=V_{i+1}, d=V_{i+2}
  R f = R(7.0 / 12.0) * (b + c) - R(1.0 / 12.0) * (a + d);
  R lo = rmin(b, c), hi = rmax(b, c);
  if (f < lo) { f = lo; branch(41); }
  if (f > hi) { f = hi; branch(42); }
  return f;
}
template <class R> inline void recon_ppm(const R s[5], R& plus, R& minus) {
  R vc = s[2];
  R vp = ppm_face(s[1], s[2], s[3], s[4]);
  R vm = ppm_face(s[0], s[1], s[2], s[3]);
  if ((vp - vc) * (vc - vm) <= R(0.0)) {
    branch(43);
    vp = vc;
    vm = vc;
  } else {
    R dv = vp - vm;
    R v6 = R(6.0) * (vc - R(0.5) * (vm + vp));
    if (dv * v6 > dv * dv) { branch(44); vm = R(3.0) * vc - R(2.0) * vp; }
    else if (-(dv * dv) > dv * v6) { branch(45); vp = R(3.0) * vc - R(2.0) * vm; }
  }
  plus = vp;
  minus = vm;
}

// CFL rate of one cell (reading; the paper is silent):
//   sum over active d of (|v_d| + cf_d) / dx_d,
// with cf_d the fast speed along d using the cell-centred field component B_d.
template <class R> inline R cfl_rate(const R V[NP], const R idx[3], int ndim, double gamma) {
  R B2 = (V[P_BX] * V[P_BX] + V[P_BY] * V[P_BY]) + V[P_BZ] * V[P_BZ];
  R lam(0.0);
  for (int d = 0; d < ndim; d++) {
    R cf = fast_speed(V[P_RHO], V[P_PR], B2, V[P_BX + d], gamma);
    R term = (fabs(V[P_VX + d]) + cf) * idx[d];
    lam = d == 0 ? term : lam + term;
  }
  return lam;
}

// ---------------------------------------------------------------------------
// The scheme on a grid.
// ---------------------------------------------------------------------------
template <class R> struct Sim {
  Config c{};
  int ndim = 2, G = 2;
  int n[3] = {1, 1, 1};
  double dx[3] = {1, 1, 1};
  bool periodic[3] = {true, true, true};
  State<R> U0, U1, U2, Lq;   // RK registers and the stage increment
  Field<R> P[NP];            // primitives of the stage input
  Field<R> Wp[3][NW], Wm[3][NW];  // reconstructed V^L_{i+1/2}, V^R_{i-1/2} per direction
  Field<R> F[3][NW];         // Riemann flux at each face, per direction
  Field<R> I[3][NI];         // UCT ingredients at each face
  Field<R> E[3];             // edge electric fields E_x, E_y, E_z
  R time = R(0.0);
  long long fallbacks = 0;   // cells where reconstruction fell back to first order
  long long floors = 0;      // interior cells whose recovered pressure was raised to the floor
  int bad = 0;               // set when a non-positive density or pressure is met
  long long bad_cell = -1;

  explicit Sim(const Config& cfg) : c(cfg) {
    ndim = cfg.ndim;
    if (ndim != 2 && ndim != 3) throw std::invalid_argument("ndim must be 2 or 3");
    if (cfg.emf == EMF_UCT_HLLD && cfg.riemann != RS_HLLD)
      throw std::invalid_argument("UCT-HLLD edge fields need the HLLD solver");
    G = cfg.recon == RECON_PLM ? 2 : 3;
    n[0] = cfg.nx; n[1] = cfg.ny; n[2] = ndim == 3 ? cfg.nz : 1;
    for (int d = 0; d < 3; d++) dx[d] = (cfg.x1[d] - cfg.x0[d]) / n[d];
    for (int d = 0; d < 3; d++) periodic[d] = cfg.bc[2 * d] == BC_PERIODIC;
    auto initf = [&](Field<R>& f) { f.init(n[0], n[1], n[2], G, ndim); };
    for (auto* S : {&U0, &U1, &U2, &Lq}) for (auto& f : *S) initf(f);
    for (auto& f : P) initf(f);
    for (int d = 0; d < 3; d++) {
      for (auto& f : Wp[d]) initf(f);
      for (auto& f : Wm[d]) initf(f);
      for (auto& f : F[d]) initf(f);
      for (auto& f : I[d]) initf(f);
      initf(E[d]);
    }
  }

  int lo(int d) const { return (d < ndim) ? -G : 0; }
  int hi(int d) const { return (d < ndim) ? n[d] + G : 0; }  // inclusive (extra slot)
  bool is_face(int q, int d) const {  // slot q is a face array with normal d
    if (q == Q_B0) return d == 0;
    if (q == Q_B1) return d == 1;
    if (q == Q_B2) return ndim == 3 && d == 2;
    return false;
  }

  // ---- Ghost zones (§2.2: "specified initial and boundary conditions") ----
  // Reading: periodic axes are filled first (x, y, z), then outflow axes
  // (x, y, z); each pass covers the full padded transverse range so edges and
  // corners take the values of the last pass.  Periodic: wrap.  Outflow: the
  // cell-centred conserved variables and the transverse face fields are copied
  // from the last interior layer; the normal face field in each ghost cell is
  // set so that the discrete div B of that ghost cell vanishes.
  void fill_ghosts(State<R>& S) {
    g_flops.phase = PH_GHOST;
    for (int pass = 0; pass < 2; pass++)
      for (int d = 0; d < ndim; d++) {
        if ((pass == 0) != periodic[d]) continue;
        if (periodic[d]) fill_periodic(S, d);
        else fill_outflow(S, d);
      }
  }
  template <class Fn> void each_transverse(int d, Fn fn, int shrink = 0) {
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    for (int a = lo(t1); a <= hi(t1) - (t1 < ndim ? shrink : 0); a++)
      for (int b = lo(t2); b <= hi(t2) - (t2 < ndim ? shrink : 0); b++) fn(t1, a, t2, b);
  }
  static void set3(int* x, int d, int v) { x[d] = v; }
  void fill_periodic(State<R>& S, int d) {
    int N = n[d];
    each_transverse(d, [&](int t1, int a, int t2, int b) {
      for (int g = -G; g <= N + G; g++) {
        if (g >= 0 && g < N) continue;
        int src = ((g % N) + N) % N;
        int xd[3], xs[3];
        xd[t1] = a; xd[t2] = b; xd[d] = g;
        xs[t1] = a; xs[t2] = b; xs[d] = src;
        for (int q = 0; q < NQ; q++) S[q](xd[0], xd[1], xd[2]) = S[q](xs[0], xs[1], xs[2]);
      }
    });
  }
  void fill_outflow(State<R>& S, int d) {
    int N = n[d];
    // copies
    each_transverse(d, [&](int t1, int a, int t2, int b) {
      for (int side = 0; side < 2; side++)
        for (int m = 1; m <= G + (side == 1 ? 1 : 0); m++) {
          int g = side == 0 ? -m : N - 1 + m;
          int src = side == 0 ? 0 : N - 1;
          int xd[3], xs[3];
          xd[t1] = a; xd[t2] = b; xd[d] = g;
          xs[t1] = a; xs[t2] = b; xs[d] = src;
          for (int q = 0; q < NQ; q++) {
            if (is_face(q, d)) continue;
            S[q](xd[0], xd[1], xd[2]) = S[q](xs[0], xs[1], xs[2]);
          }
        }
    });
    // normal face field from div B = 0 in each ghost cell
    int qn = Q_B0 + d;
    each_transverse(d, [&](int t1, int a, int t2, int b) {
      auto divT = [&](int cell) {  // sum over active transverse t of (B_t(+) - B_t(-)) / dx_t
        int x[3];
        x[t1] = a; x[t2] = b; x[d] = cell;
        R s(0.0);
        bool first = true;
        for (int t : {t1, t2}) {
          if (t >= ndim) continue;
          int xp[3] = {x[0], x[1], x[2]};
          xp[t] += 1;
          R term = (S[Q_B0 + t](xp[0], xp[1], xp[2]) - S[Q_B0 + t](x[0], x[1], x[2])) / R(dx[t]);
          s = first ? term : s + term;
          first = false;
        }
        return s;
      };
      for (int m = 1; m <= G; m++) {  // left: face -m from face -m+1
        int cell = -m;
        int x[3], xp[3];
        x[t1] = a; x[t2] = b; x[d] = cell;
        xp[t1] = a; xp[t2] = b; xp[d] = cell + 1;
        S[qn](x[0], x[1], x[2]) = S[qn](xp[0], xp[1], xp[2]) + R(dx[d]) * divT(cell);
      }
      for (int m = 0; m < G; m++) {  // right: face N+m+1 from face N+m
        int cell = N + m;
        int x[3], xp[3];
        x[t1] = a; x[t2] = b; x[d] = cell;
        xp[t1] = a; xp[t2] = b; xp[d] = cell + 1;
        S[qn](xp[0], xp[1], xp[2]) = S[qn](x[0], x[1], x[2]) - R(dx[d]) * divT(cell);
      }
    }, 1);
  }

  // ---- c2p on every cell that has both faces (all padded cells) ----
  void compute_prims(State<R>& S, bool count_floors = true) {
    g_flops.phase = PH_C2P;
    for (int k = lo(2); k < (ndim == 3 ? hi(2) : 1); k++)
      for (int j = lo(1); j < hi(1); j++)
        for (int i = lo(0); i < hi(0); i++) {
          R bx = R(0.5) * (S[Q_B0](i, j, k) + S[Q_B0](i + 1, j, k));
          R by = R(0.5) * (S[Q_B1](i, j, k) + S[Q_B1](i, j + 1, k));
          R bz = ndim == 3 ? R(0.5) * (S[Q_B2](i, j, k) + S[Q_B2](i, j, k + 1)) : S[Q_B2](i, j, k);
          R V[NP];
          cons_to_prim(S[Q_RHO](i, j, k), S[Q_MX](i, j, k), S[Q_MY](i, j, k), S[Q_MZ](i, j, k), S[Q_EN](i, j, k),
                       bx, by, bz, c.gamma, V);
          // Pressure floor (reading; the paper is silent): the recovered
          // pressure is raised to p_floor when below it; the conserved energy
          // is left unchanged, so the update stays conservative.
          if (V[P_PR] < R(c.p_floor)) {
            branch(52);
            V[P_PR] = R(c.p_floor);
            if (count_floors && i >= 0 && i < n[0] && j >= 0 && j < n[1] && k >= 0 && k < n[2]) floors++;
          }
          for (int q = 0; q < NP; q++) P[q](i, j, k) = V[q];
        }
  }
  void check_interior_prims() {
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++)
        for (int i = 0; i < n[0]; i++) {
          double r = value(P[P_RHO](i, j, k)), p = value(P[P_PR](i, j, k));
          if (!(r > 0.0) || !(p > 0.0)) {
            long long id = ((long long)k * n[1] + j) * n[0] + i;
            if (!bad || id < bad_cell) bad_cell = id;
            bad = 1;
          }
        }
  }

  // ---- Reconstruction in direction d for cells in [-1, n_d] x transverse [-1, n_t] ----
  void reconstruct(int d) {
    g_flops.phase = PH_RECON;
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int comp[NW] = {P_RHO, P_VX + d, P_VX + t1, P_VX + t2, P_BX + t1, P_BX + t2, P_PR};
    int lo1 = t1 < ndim ? -1 : 0, hi1 = t1 < ndim ? n[t1] : 0;
    int lo2 = t2 < ndim ? -1 : 0, hi2 = t2 < ndim ? n[t2] : 0;
    for (int a = lo1; a <= hi1; a++)
      for (int b = lo2; b <= hi2; b++)
        for (int cidx = -1; cidx <= n[d]; cidx++) {
          int x[3];
          x[t1] = a; x[t2] = b; x[d] = cidx;
          R wp[NW], wm[NW], wc[NW];
          for (int q = 0; q < NW; q++) {
            R s[5];
            for (int m = -2; m <= 2; m++) {
              int y[3] = {x[0], x[1], x[2]};
              y[d] += m;
              bool need = c.recon != RECON_PLM || (m >= -1 && m <= 1);
              s[m + 2] = need ? P[comp[q]](y[0], y[1], y[2]) : R(0.0);
            }
            wc[q] = s[2];
            if (c.recon == RECON_PLM) recon_plm(s, wp[q], wm[q]);
            else if (c.recon == RECON_WENOZ) recon_wenoz(s, wp[q], wm[q]);
            else recon_ppm(s, wp[q], wm[q]);
          }
          // Positivity fallback (reading): first order in this cell if a
          // reconstructed density or pressure is not positive.
          if (!(wp[W_RHO] > R(0.0)) || !(wm[W_RHO] > R(0.0)) || !(wp[W_PR] > R(0.0)) || !(wm[W_PR] > R(0.0))) {
            branch(51);
            for (int q = 0; q < NW; q++) wp[q] = wm[q] = wc[q];
            fallbacks++;
          }
          for (int q = 0; q < NW; q++) {
            Wp[d][q](x[0], x[1], x[2]) = wp[q];
            Wm[d][q](x[0], x[1], x[2]) = wm[q];
          }
        }
  }

  // ---- Riemann fluxes at faces [0, n_d] x transverse [-1, n_t] ----
  void riemann(int d, State<R>& S) {
    g_flops.phase = PH_RIEMANN;
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int lo1 = t1 < ndim ? -1 : 0, hi1 = t1 < ndim ? n[t1] : 0;
    int lo2 = t2 < ndim ? -1 : 0, hi2 = t2 < ndim ? n[t2] : 0;
    for (int a = lo1; a <= hi1; a++)
      for (int b = lo2; b <= hi2; b++)
        for (int f = 0; f <= n[d]; f++) {
          int x[3], xl[3];
          x[t1] = a; x[t2] = b; x[d] = f;
          xl[t1] = a; xl[t2] = b; xl[d] = f - 1;
          R WL[NW], WR[NW], Fx[NW], ing[NI];
          for (int q = 0; q < NW; q++) {
            WL[q] = Wp[d][q](xl[0], xl[1], xl[2]);
            WR[q] = Wm[d][q](x[0], x[1], x[2]);
          }
          R bn = S[Q_B0 + d](x[0], x[1], x[2]);
          if (c.riemann == RS_HLLD) riemann_hlld(WL, WR, bn, c.gamma, Fx, ing, c.emf == EMF_UCT_HLLD);
          else riemann_hll(WL, WR, bn, c.gamma, Fx, ing);
          for (int q = 0; q < NW; q++) F[d][q](x[0], x[1], x[2]) = Fx[q];
          for (int q = 0; q < NI; q++) I[d][q](x[0], x[1], x[2]) = ing[q];
        }
  }

  // ---- UCT edge electric field E_c (reading of the UCT-HLL average) ----
  // At the edge at a-face index p_a, b-face index p_b (cyclic a, b, c):
  //   E_c = -(a+_a u^W B_b^W + a-_a u^E B_b^E) + d_a (B_b^E - B_b^W)
  //         + (a+_b u^S B_a^S + a-_b u^N B_a^N) - d_b (B_a^N - B_a^S),
  // with the a-face ingredients averaged over the two a-faces touching the
  // edge, B_b^{W,E} the minmod reconstructions of the b-face field along a to
  // the edge from either side, and likewise for the b-faces.
  // UCT-HLLD: the same form with the HLLD coefficients and separate d^L, d^R:
  //   E_c = -(a^L_a u^W B_b^W + a^R_a u^E B_b^E) + (d^R_a B_b^E - d^L_a B_b^W)
  //         + (a^L_b u^S B_a^S + a^R_b u^N B_a^N) - (d^R_b B_a^N - d^L_b B_a^S).
  R face_to_edge(Field<R>& B, int x[3], int along, bool from_minus) {
    // Field B sampled at x - e_along (from_minus) or x, reconstructed to the
    // edge plane between them with a minmod slope along `along`.
    int c0[3] = {x[0], x[1], x[2]};
    if (from_minus) c0[along] -= 1;
    int cm[3] = {c0[0], c0[1], c0[2]}, cp[3] = {c0[0], c0[1], c0[2]};
    cm[along] -= 1;
    cp[along] += 1;
    R v = B(c0[0], c0[1], c0[2]);
    R dl = v - B(cm[0], cm[1], cm[2]);
    R dr = B(cp[0], cp[1], cp[2]) - v;
    R s = minmod(dl, dr);
    return from_minus ? v + R(0.5) * s : v - R(0.5) * s;
  }
  void compute_emf(int cc, State<R>& S) {
    g_flops.phase = PH_EMF;
    int a = (cc + 1) % 3, b = (cc + 2) % 3;
    int ext[3];
    ext[a] = n[a];      // face index range [0, n_a]
    ext[b] = n[b];      // face index range [0, n_b]
    ext[cc] = n[cc] - 1; // cell index range [0, n_c - 1]
    for (int k = 0; k <= ext[2]; k++)
      for (int j = 0; j <= ext[1]; j++)
        for (int i = 0; i <= ext[0]; i++) {
          int x[3] = {i, j, k};
          int xb[3] = {i, j, k}, xa[3] = {i, j, k};
          xb[b] -= 1;  // the other a-face touching the edge
          xa[a] -= 1;  // the other b-face touching the edge
          R h(0.5);
          R apa = h * (I[a][I_AP](xb[0], xb[1], xb[2]) + I[a][I_AP](i, j, k));
          R ama = h * (I[a][I_AM](xb[0], xb[1], xb[2]) + I[a][I_AM](i, j, k));
          R dda = h * (I[a][I_DD](xb[0], xb[1], xb[2]) + I[a][I_DD](i, j, k));
          R uW = h * (I[a][I_UL](xb[0], xb[1], xb[2]) + I[a][I_UL](i, j, k));
          R uE = h * (I[a][I_UR](xb[0], xb[1], xb[2]) + I[a][I_UR](i, j, k));
          R apb = h * (I[b][I_AP](xa[0], xa[1], xa[2]) + I[b][I_AP](i, j, k));
          R amb = h * (I[b][I_AM](xa[0], xa[1], xa[2]) + I[b][I_AM](i, j, k));
          R ddb = h * (I[b][I_DD](xa[0], xa[1], xa[2]) + I[b][I_DD](i, j, k));
          R vS = h * (I[b][I_UL](xa[0], xa[1], xa[2]) + I[b][I_UL](i, j, k));
          R vN = h * (I[b][I_UR](xa[0], xa[1], xa[2]) + I[b][I_UR](i, j, k));
          R BbW = face_to_edge(S[Q_B0 + b], x, a, true);
          R BbE = face_to_edge(S[Q_B0 + b], x, a, false);
          R BaS = face_to_edge(S[Q_B0 + a], x, b, true);
          R BaN = face_to_edge(S[Q_B0 + a], x, b, false);
          R e;
          if (c.emf == EMF_UCT_HLLD) {
            R dra = h * (I[a][I_DR](xb[0], xb[1], xb[2]) + I[a][I_DR](i, j, k));
            R drb = h * (I[b][I_DR](xa[0], xa[1], xa[2]) + I[b][I_DR](i, j, k));
            e = ((-(apa * uW * BbW + ama * uE * BbE) + (dra * BbE - dda * BbW)) + (apb * vS * BaS + amb * vN * BaN)) -
                (drb * BaN - ddb * BaS);
          } else
            e = ((-(apa * uW * BbW + ama * uE * BbE) + dda * (BbE - BbW)) + (apb * vS * BaS + amb * vN * BaN)) -
                ddb * (BaN - BaS);
          E[cc](i, j, k) = e;
        }
  }

  // ---- One stage increment L(S), including the factor dt (reading of Eq. FV) ----
  void stage_increment(State<R>& S, R dt) {
    fill_ghosts(S);
    compute_prims(S);
    check_interior_prims();
    for (int d = 0; d < ndim; d++) {
      reconstruct(d);
      riemann(d, S);
    }
    // Eq. FV: L = - sum_d dt/dx_d (F_{+1/2} - F_{-1/2}) for the cell-centred variables.
    g_flops.phase = PH_FLUXDIFF;
    R dtdx[3];
    for (int d = 0; d < 3; d++) dtdx[d] = dt / R(dx[d]);
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++)
        for (int i = 0; i < n[0]; i++) {
          R acc[6];
          for (int d = 0; d < ndim; d++) {
            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            int xp[3] = {i, j, k};
            xp[d] += 1;
            auto diff = [&](int w) { return F[d][w](xp[0], xp[1], xp[2]) - F[d][w](i, j, k); };
            // map sweep-frame flux components back to (rho, mx, my, mz, E, Bz_cell)
            R dv[6];
            dv[0] = diff(W_RHO);
            R dm[3];
            dm[d] = diff(W_VN); dm[t1] = diff(W_VT1); dm[t2] = diff(W_VT2);
            dv[1] = dm[0]; dv[2] = dm[1]; dv[3] = dm[2];
            dv[4] = diff(W_PR);  // energy flux is stored in the last slot
            // 2D cell Bz: transverse component z of the x (t2) or y (t1) sweep
            dv[5] = ndim == 2 ? (d == 0 ? diff(W_BT2) : diff(W_BT1)) : R(0.0);
            for (int v = 0; v < 6; v++) {
              R term = -(dtdx[d] * dv[v]);
              acc[v] = d == 0 ? term : acc[v] + term;
            }
          }
          for (int v = 0; v < 5; v++) Lq[v](i, j, k) = acc[v];
          if (ndim == 2) Lq[Q_B2](i, j, k) = acc[5];
        }
    // Edge electric fields and the CT increment  L_B = -dt curl E.
    if (ndim == 3) for (int cc = 0; cc < 3; cc++) compute_emf(cc, S);
    else compute_emf(2, S);
    g_flops.phase = PH_CT;
    for (int d = 0; d < ndim; d++) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      int ext[3] = {n[0] - 1, n[1] - 1, n[2] - 1};
      if (!periodic[d]) ext[d] = n[d];
      for (int k = 0; k <= ext[2]; k++)
        for (int j = 0; j <= ext[1]; j++)
          for (int i = 0; i <= ext[0]; i++) {
            // (curl E)_d = d(E_d2)/d(x_d1) - d(E_d1)/d(x_d2); in 2D only E_z
            // exists and only x, y derivatives are taken.
            int p1[3] = {i, j, k}, p2[3] = {i, j, k};
            p1[d1] += 1;
            p2[d2] += 1;
            bool has1 = d1 < ndim, has2 = d2 < ndim;
            R t_1(0.0), t_2(0.0);
            if (has1) t_1 = (E[d2](p1[0], p1[1], p1[2]) - E[d2](i, j, k)) * (dt / R(dx[d1]));
            if (has2) t_2 = (E[d1](p2[0], p2[1], p2[2]) - E[d1](i, j, k)) * (dt / R(dx[d2]));
            R val = (has1 && has2) ? -(t_1 - t_2) : (has1 ? -t_1 : t_2);
            Lq[Q_B0 + d](i, j, k) = val;
          }
    }
  }

  // Apply a stage combine  out = (c0 * U0 + c1 * S + L) * c2  (or / 3) to every
  // evolved cell and face.  Eq. RK3 and the SSP-RK2 analogue.
  template <class Fn> void each_updated(Fn fn) {
    for (int q = 0; q < NQ; q++) {
      int ext[3] = {n[0] - 1, n[1] - 1, n[2] - 1};
      for (int d = 0; d < ndim; d++)
        if (is_face(q, d) && !periodic[d]) ext[d] = n[d];
      for (int k = 0; k <= ext[2]; k++)
        for (int j = 0; j <= ext[1]; j++)
          for (int i = 0; i <= ext[0]; i++) fn(q, i, j, k);
    }
  }

  // One time step of size dt (Eq. RK3; SSP-RK2 = Heun for rk == 2).
  void step(R dt) {
    // stage 1:  U* = U^n + L^n
    stage_increment(U0, dt);
    g_flops.phase = PH_RK;
    each_updated([&](int q, int i, int j, int k) { U1[q](i, j, k) = U0[q](i, j, k) + Lq[q](i, j, k); });
    stage_increment(U1, dt);
    g_flops.phase = PH_RK;
    if (c.rk == 2) {
      // U^{n+1} = (U^n + U* + L*) / 2
      each_updated([&](int q, int i, int j, int k) {
        U0[q](i, j, k) = R(0.5) * ((U0[q](i, j, k) + U1[q](i, j, k)) + Lq[q](i, j, k));
      });
    } else {
      // U** = (3 U^n + U* + L*) / 4
      each_updated([&](int q, int i, int j, int k) {
        U2[q](i, j, k) = R(0.25) * ((R(3.0) * U0[q](i, j, k) + U1[q](i, j, k)) + Lq[q](i, j, k));
      });
      stage_increment(U2, dt);
      g_flops.phase = PH_RK;
      // U^{n+1} = (U^n + 2 U** + 2 L**) / 3.  Reading: Eq. RK3 as printed
      // weights L** by 1/3, which is inconsistent (for u' = lambda u it gives
      // 1 + 2z/3 + ...); the cited Shu-Osher SSP-RK3 weights it by 2/3.
      each_updated([&](int q, int i, int j, int k) {
        U0[q](i, j, k) = ((U0[q](i, j, k) + R(2.0) * U2[q](i, j, k)) + R(2.0) * Lq[q](i, j, k)) / R(3.0);
      });
    }
    time = time + dt;
  }

  // CFL time step (reading; the paper is silent):
  //   dt = C / max_cells sum_d (|v_d| + cf_d) / dx_d  on the interior cells of U^n,
  // with cf_d the fast speed along d using the cell-centred field component B_d.
  R cfl_dt() {
    fill_ghosts(U0);
    compute_prims(U0, false);  // floors are counted in the stages' passes only
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

// ---------------------------------------------------------------------------
// Functionals of the final state and the map from initial primitives, for the
// gradient of a final-state functional with respect to the initial density
// and velocity (the step sizes are given, i.e. frozen).
// ---------------------------------------------------------------------------
enum { FUNC_MAGNETIC_ENERGY = 0, FUNC_MISFIT = 1 };

// Initial conserved state from primitives (Eq. Energy): m = rho v,
// E = p/(G-1) + rho v^2/2 + B^2/2 with the cell field the mean of the faces
// (2D B_z: the cell value); p and the field are held fixed.
template <class R>
void set_from_prims(Sim<R>& s, const R* rho, const R* vx, const R* vy, const R* vz, const double* p,
                    const double* const* B) {
  // faces (and the 2D cell B_z) as constants
  for (int q = Q_B0; q <= Q_B2; q++) {
    int e[3] = {s.n[0], s.n[1], s.n[2]};
    for (int d = 0; d < s.ndim; d++)
      if (s.is_face(q, d)) e[d] += 1;
    const double* src = B[q - Q_B0];
    for (int k = 0; k < e[2]; k++)
      for (int j = 0; j < e[1]; j++)
        for (int i = 0; i < e[0]; i++) s.U0[q](i, j, k) = R(*src++);
  }
  const double gm1 = s.c.gamma - 1.0;
  size_t c = 0;
  for (int k = 0; k < s.n[2]; k++)
    for (int j = 0; j < s.n[1]; j++)
      for (int i = 0; i < s.n[0]; i++, c++) {
        R bx = R(0.5) * (s.U0[Q_B0](i, j, k) + s.U0[Q_B0](i + 1, j, k));
        R by = R(0.5) * (s.U0[Q_B1](i, j, k) + s.U0[Q_B1](i, j + 1, k));
        R bz = s.ndim == 3 ? R(0.5) * (s.U0[Q_B2](i, j, k) + s.U0[Q_B2](i, j, k + 1)) : s.U0[Q_B2](i, j, k);
        R v2 = (vx[c] * vx[c] + vy[c] * vy[c]) + vz[c] * vz[c];
        R B2 = (bx * bx + by * by) + bz * bz;
        s.U0[Q_RHO](i, j, k) = rho[c];
        s.U0[Q_MX](i, j, k) = rho[c] * vx[c];
        s.U0[Q_MY](i, j, k) = rho[c] * vy[c];
        s.U0[Q_MZ](i, j, k) = rho[c] * vz[c];
        s.U0[Q_EN](i, j, k) = (R(p[c] / gm1) + (R(0.5) * rho[c]) * v2) + R(0.5) * B2;
      }
}

// J = 1/2 sum_cells |B_c|^2 dV (magnetic energy), or
// J = 1/2 sum_cells sum_q (U_q - T_q)^2 dV over the cell-centred conserved
// variables (rho, m, E; in 2D also B_z) for a target state T (misfit).
template <class R> R functional(Sim<R>& s, int which, const double* const* target) {
  s.fill_ghosts(s.U0);
  double dV = s.dx[0] * s.dx[1] * (s.ndim == 3 ? s.dx[2] : 1.0);
  R J(0.0);
  size_t c = 0;
  for (int k = 0; k < s.n[2]; k++)
    for (int j = 0; j < s.n[1]; j++)
      for (int i = 0; i < s.n[0]; i++, c++) {
        R cellsum(0.0);
        if (which == FUNC_MAGNETIC_ENERGY) {
          R bx = R(0.5) * (s.U0[Q_B0](i, j, k) + s.U0[Q_B0](i + 1, j, k));
          R by = R(0.5) * (s.U0[Q_B1](i, j, k) + s.U0[Q_B1](i, j + 1, k));
          R bz = s.ndim == 3 ? R(0.5) * (s.U0[Q_B2](i, j, k) + s.U0[Q_B2](i, j, k + 1)) : s.U0[Q_B2](i, j, k);
          cellsum = (bx * bx + by * by) + bz * bz;
        } else {
          int nq = s.ndim == 2 ? 6 : 5;
          for (int q = 0; q < nq; q++) {
            int slot = q < 5 ? q : Q_B2;
            R dq = s.U0[slot](i, j, k) - R(target[q][c]);
            cellsum = q == 0 ? dq * dq : cellsum + dq * dq;
          }
        }
        J = J + cellsum;
      }
  return R(0.5 * dV) * J;
}

// J after nsteps steps of the given sizes from the initial primitives.
template <class R>
R run_functional(const Config& cfg, const R* rho, const R* vx, const R* vy, const R* vz, const double* p,
                 const double* const* B, const double* dts, int nsteps, int which, const double* const* target,
                 int* bad) {
  Sim<R> s(cfg);
  set_from_prims(s, rho, vx, vy, vz, p, B);
  for (int t = 0; t < nsteps; t++) s.step(R(dts[t]));
  if (bad) *bad = s.bad;
  return functional(s, which, target);
}

}  // namespace orc
