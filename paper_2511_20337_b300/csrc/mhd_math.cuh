// Pointwise device arithmetic of the MHD step: primitive recovery, fast
// magnetosonic speed, sweep-frame states and fluxes, HLL and HLLD Riemann
// solvers, and the PLM / WENO-Z / PPM reconstructions (paper §2.2).
//
// Two flavours of arithmetic:
//   *_ieee : fixed-order IEEE operations (__dadd_rn & co., no contraction)
//            for the primitive recovery and the CFL speed, so that those
//            values are reproducible to the bit;
//   the rest: free FMA contraction and reciprocals formed once per quantity.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mhd {

// Thresholds of the degenerate HLLD branches and the WENO-Z epsilon
// (the paper is silent; values shared by every part of the library).
constexpr double kHlldDegenEps = 1e-12;
constexpr double kHlldBnEps = 1e-12;
constexpr double kWenozEps = 1e-40;

// ---------------------------------------------------------------------------
// reciprocal / square root
// ---------------------------------------------------------------------------
#ifndef MHD_FAST_RCP
#define MHD_FAST_RCP 1
#endif

// 1/x.  Fast form: the hardware's ~20-bit reciprocal seed (PTX
// rcp.approx.ftz.f64) refined by one cubic Newton-Raphson step
//   e = 1 - x r,  r' = r + r (e + e^2),
// whose relative error is e^3 (< 2^-59 from a 2^-20 seed) plus rounding, i.e.
// within about one ulp of the correctly rounded 1/x for normal, nonzero x.
__device__ __forceinline__ double rcp(double x) {
#if MHD_FAST_RCP
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
#else
  return 1.0 / x;
#endif
}

// ---------------------------------------------------------------------------
// IEEE fixed-order pieces (bitwise reproducible)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double a_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double s_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double m_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double d_(double a, double b) { return __ddiv_rn(a, b); }

// Conservative -> primitive (§2.2): v = m / rho, p = (G-1)(E - m.v/2 - B^2/2),
// 1/rho formed once; operation order fixed.
struct Prim8 {
  double rho, vx, vy, vz, bx, by, bz, p;
};
__device__ __forceinline__ Prim8 c2p_ieee(double rho, double mx, double my, double mz, double en, double bx,
                                          double by, double bz, double gm1) {
  Prim8 o;
  double inv = d_(1.0, rho);
  o.vx = m_(mx, inv);
  o.vy = m_(my, inv);
  o.vz = m_(mz, inv);
  double kin = m_(0.5, a_(a_(m_(mx, o.vx), m_(my, o.vy)), m_(mz, o.vz)));
  double B2 = a_(a_(m_(bx, bx), m_(by, by)), m_(bz, bz));
  o.p = m_(gm1, s_(s_(en, kin), m_(0.5, B2)));
  o.rho = rho;
  o.bx = bx;
  o.by = by;
  o.bz = bz;
  return o;
}

// Fast magnetosonic speed along a direction with normal component bn:
//   cf^2 = [(G p + B^2) + sqrt((G p + B^2)^2 - 4 G p bn^2)] / (2 rho).
__device__ __forceinline__ double fast_speed_ieee(double rho, double p, double B2, double bn, double gamma) {
  double gp = m_(gamma, p);
  double s = a_(gp, B2);
  double disc = s_(m_(s, s), m_(m_(4.0, gp), m_(bn, bn)));
  if (disc < 0.0) disc = 0.0;
  double cf2 = d_(m_(0.5, a_(s, __dsqrt_rn(disc))), rho);
  return __dsqrt_rn(cf2);
}

// ---------------------------------------------------------------------------
// Sweep-frame physics.  W = (rho, u, v, w, b1, b2, p): normal velocity u,
// transverse (v, w) and transverse field (b1, b2) in the cyclic order of the
// sweep; bn is the staggered normal field at the face.
// ---------------------------------------------------------------------------
struct W7 {
  double rho, u, v, w, b1, b2, p;
};
struct Flux7 {
  double f[7];  // rho, m_n, m_t1, m_t2, B_t1, B_t2, E
};

struct Side {
  double U[7], F[7];
  double pT, B2, vB, E, irho;
};

__device__ __forceinline__ void side_state(const W7& W, double bn, double igm1, Side& s) {
  s.B2 = fma(bn, bn, fma(W.b1, W.b1, W.b2 * W.b2));
  s.pT = fma(0.5, s.B2, W.p);
  s.vB = fma(W.u, bn, fma(W.v, W.b1, W.w * W.b2));
  double v2 = fma(W.u, W.u, fma(W.v, W.v, W.w * W.w));
  s.E = fma(W.p, igm1, 0.5 * fma(W.rho, v2, s.B2));
  double mu = W.rho * W.u;
  s.U[0] = W.rho;
  s.U[1] = mu;
  s.U[2] = W.rho * W.v;
  s.U[3] = W.rho * W.w;
  s.U[4] = W.b1;
  s.U[5] = W.b2;
  s.U[6] = s.E;
  s.F[0] = mu;
  s.F[1] = fma(mu, W.u, s.pT) - bn * bn;
  s.F[2] = fma(mu, W.v, -bn * W.b1);
  s.F[3] = fma(mu, W.w, -bn * W.b2);
  s.F[4] = fma(W.u, W.b1, -W.v * bn);
  s.F[5] = fma(W.u, W.b2, -W.w * bn);
  s.F[6] = fma(s.E + s.pT, W.u, -bn * s.vB);
}

__device__ __forceinline__ double fast_speed(double rho_inv, double p, double B2, double bn, double gamma) {
  double gp = gamma * p;
  double s = gp + B2;
  double disc = fma(s, s, -(4.0 * gp) * (bn * bn));
  disc = fmax(disc, 0.0);
  return sqrt(0.5 * (s + sqrt(disc)) * rho_inv);
}

// Outer speed estimate S_L, S_R (Miyoshi & Kusano 2005) and the UCT-HLL
// ingredients a+ = aR/(aR-aL), a- = -aL/(aR-aL), d = -aR aL/(aR-aL).
struct Ingr {
  double ap, am, dd, uL, uR;
};
__device__ __forceinline__ void speeds(const W7& L, const W7& R, const Side& sl, const Side& sr, double bn,
                                       double gamma, double& SL, double& SR, Ingr& ing) {
  double cfL = fast_speed(sl.irho, L.p, sl.B2, bn, gamma);
  double cfR = fast_speed(sr.irho, R.p, sr.B2, bn, gamma);
  double cmax = fmax(cfL, cfR);
  SL = fmin(L.u, R.u) - cmax;
  SR = fmax(L.u, R.u) + cmax;
  double aR = fmax(0.0, SR), aL = fmin(0.0, SL);
  double inv = rcp(aR - aL);
  ing.ap = aR * inv;
  ing.am = -aL * inv;
  ing.dd = -(aR * aL) * inv;
  ing.uL = L.u;
  ing.uR = R.u;
}

__device__ __forceinline__ void riemann_hll(const W7& L, const W7& R, double bn, double gamma, double igm1,
                                            Flux7& F, Ingr& ing) {
  Side sl, sr;
  side_state(L, bn, igm1, sl);
  side_state(R, bn, igm1, sr);
  sl.irho = rcp(L.rho);
  sr.irho = rcp(R.rho);
  double SL, SR;
  speeds(L, R, sl, sr, bn, gamma, SL, SR, ing);
  if (SL >= 0.0) {
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = sl.F[q];
  } else if (SR <= 0.0) {
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = sr.F[q];
  } else {
    double inv = rcp(SR - SL);
    double sls = SR * SL;
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = (fma(SR, sl.F[q], -SL * sr.F[q]) + sls * (sr.U[q] - sl.U[q])) * inv;
  }
}

// HLLD (Miyoshi & Kusano 2005): waves S_L < S*_L < S_M < S*_R < S_R with
// continuous normal velocity and total pressure across the fan.  Only the
// side of the contact that holds x/t = 0 is assembled into the flux.
__device__ __forceinline__ void riemann_hlld(const W7& L, const W7& R, double bn, double gamma, double igm1,
                                             Flux7& F, Ingr& ing) {
  Side sl, sr;
  side_state(L, bn, igm1, sl);
  side_state(R, bn, igm1, sr);
  sl.irho = rcp(L.rho);
  sr.irho = rcp(R.rho);
  double SL, SR;
  speeds(L, R, sl, sr, bn, gamma, SL, SR, ing);
  if (SL > 0.0) {
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = sl.F[q];
    return;
  }
  if (SR < 0.0) {
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = sr.F[q];
    return;
  }
  const double bn2 = bn * bn;
  double sdL = SL - L.u, sdR = SR - R.u;
  double rsL = sdL * L.rho, rsR = sdR * R.rho;  // rho (S - u)
  double iden = rcp(rsR - rsL);
  double SM = ((rsR * R.u - rsL * L.u) - sr.pT + sl.pT) * iden;
  double pTs = (fma(rsR, sl.pT, -rsL * sr.pT) + (L.rho * rsR) * sdL * (R.u - L.u)) * iden;

  // star states, both sides (transverse parts are needed for the ** states)
  double smL = SL - SM, smR = SR - SM;
  double ismL = rcp(smL), ismR = rcp(smR);
  double rhosL = rsL * ismL, rhosR = rsR * ismR;
  double vsL, wsL, b1sL, b2sL, vsR, wsR, b1sR, b2sR;
  {
    double rsm = rsL * smL, D = rsm - bn2;
    if (fabs(D) < kHlldDegenEps * rsm) {
      vsL = L.v; wsL = L.w; b1sL = L.b1; b2sL = L.b2;
    } else {
      double iD = rcp(D);
      double cv = bn * (SM - L.u) * iD;
      vsL = fma(-L.b1, cv, L.v);
      wsL = fma(-L.b2, cv, L.w);
      double cb = fma(rsL, sdL, -bn2) * iD;
      b1sL = L.b1 * cb;
      b2sL = L.b2 * cb;
    }
  }
  {
    double rsm = rsR * smR, D = rsm - bn2;
    if (fabs(D) < kHlldDegenEps * rsm) {
      vsR = R.v; wsR = R.w; b1sR = R.b1; b2sR = R.b2;
    } else {
      double iD = rcp(D);
      double cv = bn * (SM - R.u) * iD;
      vsR = fma(-R.b1, cv, R.v);
      wsR = fma(-R.b2, cv, R.w);
      double cb = fma(rsR, sdR, -bn2) * iD;
      b1sR = R.b1 * cb;
      b2sR = R.b2 * cb;
    }
  }
  // the side of the contact that contains x/t = 0
  const bool left = SM >= 0.0;
  const W7& A = left ? L : R;
  const Side& sa = left ? sl : sr;
  double S = left ? SL : SR, sd = left ? sdL : sdR, ism = left ? ismL : ismR, rhos = left ? rhosL : rhosR;
  double vs = left ? vsL : vsR, ws = left ? wsL : wsR, b1s = left ? b1sL : b1sR, b2s = left ? b2sL : b2sR;
  double vBs = fma(SM, bn, fma(vs, b1s, ws * b2s));
  double Es = (fma(sd, sa.E, -sa.pT * A.u) + fma(pTs, SM, bn * (sa.vB - vBs))) * ism;
  double Us[7] = {rhos, rhos * SM, rhos * vs, rhos * ws, b1s, b2s, Es};
  double Uss[7] = {Us[0], Us[1], Us[2], Us[3], Us[4], Us[5], Us[6]};
  double c2 = 0.0;  // speed of the rotational wave on this side, if x/t = 0 lies beyond it
  if (!(0.5 * bn2 < kHlldBnEps * pTs)) {
    double sqL = sqrt(rhosL), sqR = sqrt(rhosR);
    double abn = fabs(bn);
    double Ss = left ? SM - abn / sqL : SM + abn / sqR;
    c2 = left ? (Ss < 0.0 ? Ss : 0.0) : (Ss >= 0.0 ? Ss : 0.0);
    double sgn = bn > 0.0 ? 1.0 : -1.0;
    double isum = rcp(sqL + sqR);
    double vss = (fma(sqL, vsL, sqR * vsR) + (b1sR - b1sL) * sgn) * isum;
    double wss = (fma(sqL, wsL, sqR * wsR) + (b2sR - b2sL) * sgn) * isum;
    double sq2 = sqL * sqR;
    double b1ss = (fma(sqL, b1sR, sqR * b1sL) + sq2 * (vsR - vsL) * sgn) * isum;
    double b2ss = (fma(sqL, b2sR, sqR * b2sL) + sq2 * (wsR - wsL) * sgn) * isum;
    double vBss = fma(SM, bn, fma(vss, b1ss, wss * b2ss));
    double sqa = left ? -sqL : sqR;
    Uss[2] = rhos * vss;
    Uss[3] = rhos * wss;
    Uss[4] = b1ss;
    Uss[5] = b2ss;
    Uss[6] = fma(sqa * (vBs - vBss), sgn, Es);
  }
#pragma unroll
  for (int q = 0; q < 7; q++) F.f[q] = fma(S, Us[q] - sa.U[q], sa.F[q]) + c2 * (Uss[q] - Us[q]);
}

// ---------------------------------------------------------------------------
// Reconstruction (Eq. reconstruct).  s0..s4 = V_{i-2..i+2}; plus = V^L_{i+1/2},
// minus = V^R_{i-1/2}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double minmod(double a, double b) {
  if ((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0)) return (fabs(b) < fabs(a)) ? b : a;
  return 0.0;
}

__device__ __forceinline__ void recon_plm(double s1, double s2, double s3, double& plus, double& minus) {
  double d = 0.5 * minmod(s2 - s1, s3 - s2);
  plus = s2 + d;
  minus = s2 - d;
}

// WENO-Z value at the right face of the middle cell of a0..a4 (Borges et al. 2008).
__device__ __forceinline__ double wenoz_face(double a0, double a1, double a2, double a3, double a4) {
  const double i6 = 1.0 / 6.0;
  double q0 = fma(2.0, a0, fma(-7.0, a1, 11.0 * a2)) * i6;
  double q1 = fma(-1.0, a1, fma(5.0, a2, 2.0 * a3)) * i6;
  double q2 = fma(2.0, a2, fma(5.0, a3, -a4)) * i6;
  double t = fma(-2.0, a1, a0) + a2, u = fma(-4.0, a1, a0) + 3.0 * a2;
  double b0 = fma(13.0 / 12.0, t * t, 0.25 * (u * u));
  t = fma(-2.0, a2, a1) + a3;
  u = a1 - a3;
  double b1 = fma(13.0 / 12.0, t * t, 0.25 * (u * u));
  t = fma(-2.0, a3, a2) + a4;
  u = fma(3.0, a2, -4.0 * a3) + a4;
  double b2 = fma(13.0 / 12.0, t * t, 0.25 * (u * u));
  double tau = fabs(b0 - b2);
  double r0 = tau * rcp(b0 + kWenozEps);
  double r1 = tau * rcp(b1 + kWenozEps);
  double r2 = tau * rcp(b2 + kWenozEps);
  double al0 = 0.1 * fma(r0, r0, 1.0);
  double al1 = 0.6 * fma(r1, r1, 1.0);
  double al2 = 0.3 * fma(r2, r2, 1.0);
  return fma(al0, q0, fma(al1, q1, al2 * q2)) * rcp(al0 + al1 + al2);
}

__device__ __forceinline__ double ppm_face(double a, double b, double c, double d) {
  double f = fma(7.0 / 12.0, b + c, -(1.0 / 12.0) * (a + d));
  double lo = fmin(b, c), hi = fmax(b, c);
  return fmin(fmax(f, lo), hi);
}
__device__ __forceinline__ void recon_ppm(double s0, double s1, double s2, double s3, double s4, double& plus,
                                          double& minus) {
  double vp = ppm_face(s1, s2, s3, s4);
  double vm = ppm_face(s0, s1, s2, s3);
  if ((vp - s2) * (s2 - vm) <= 0.0) {
    vp = s2;
    vm = s2;
  } else {
    double dv = vp - vm;
    double v6 = 6.0 * (s2 - 0.5 * (vm + vp));
    if (dv * v6 > dv * dv) vm = fma(3.0, s2, -2.0 * vp);
    else if (-(dv * dv) > dv * v6) vp = fma(3.0, s2, -2.0 * vm);
  }
  plus = vp;
  minus = vm;
}

}  // namespace mhd
