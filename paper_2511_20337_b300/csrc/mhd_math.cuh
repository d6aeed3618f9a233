// Pointwise device arithmetic of the MHD step: primitive recovery, fast
// magnetosonic speed, sweep-frame states and fluxes, HLL and HLLD Riemann
// solvers, and the PLM / WENO-Z / PPM reconstructions (paper §2.2).
//
// Two flavours of arithmetic:
//   *_ieee : fixed-order IEEE operations (correctly rounded sums, products,
//            quotients and square roots, each rounded once) for the
//            primitive recovery and the CFL speed, so that those values match
//            the oracle to the bit;
//   the rest: fused multiply-adds written out as fma(), reciprocals formed
//            once per quantity.  The library is compiled without implicit
//            contraction, so every kernel that inlines these functions rounds
//            them identically (the batched and single-grid paths agree to the
//            bit).
// Both write single products, sums and differences in the exact DFMA forms
// below (fmul, fadd, fsub), which the FP64 pipe issues faster.
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
// Products, sums and differences as fused multiply-adds.  The FP64 pipe issues
// DMUL and DADD at about 5/6 of the rate of DFMA (mhd_probe_fp64_forms), so
// the hot arithmetic writes a b, a + b and a - b in the exact DFMA forms
//   fma(a, b, -0) = a b,  fma(a, 1, b) = a + b,  fma(b, -1, a) = a - b
// (x + (-0) = x for every x, and a product with +-1 is exact), and scales by
// constants held in registers.  The constants come from a mutable device
// table, so the compiler can fold them neither back into DMUL / DADD nor into
// constant operands.  Every result is the same, to the bit, as the plain
// operation's.
// ---------------------------------------------------------------------------
enum {
  RK_NZ = 0, RK_ONE, RK_MONE, RK_HALF, RK_MHALF, RK_3_8, RK_QUARTER, RK_FOUR, RK_EPS, RK_2EPS,
  // WENO-Z
  RK_13_12, RK_M2, RK_3, RK_M4, RK_WEPS, RK_2, RK_5, RK_0_6, RK_0_3, RK_6,
  // PPM
  RK_7_12, RK_1_12,
  // WENO-Z: the q_0 stencil times 6 d_0, and 6 d_k (d = 1/10, 6/10, 3/10)
  RK_0_2, RK_M0_7, RK_1_1, RK_3_6, RK_1_8,
  // bound factor of c2p_fast's pressure
  RK_PB,
  // WENO-Z indicators scaled by 4 (recon_wenoz_c)
  RK_13_3, RK_4WEPS,
  RK_NK
};
__device__ double kRegK[RK_NK] = {-0.0, 1.0, -1.0, 0.5, -0.5, 0.375, 0.25, 4.0, kHlldDegenEps, 2.0 * kHlldBnEps,
                                  13.0 / 12.0, -2.0, 3.0, -4.0, kWenozEps, 2.0, 5.0, 0.6, 0.3, 6.0,
                                  7.0 / 12.0, 1.0 / 12.0,
                                  0.2, -0.7, 1.1, 3.6, 1.8,
                                  1e-14,
                                  13.0 / 3.0, 4.0 * kWenozEps};
__device__ __forceinline__ double rk(int i) { return __ldg(&kRegK[i]); }
__device__ __forceinline__ double fmul(double a, double b) { return fma(a, b, rk(RK_NZ)); }
__device__ __forceinline__ double fadd(double a, double b) { return fma(a, rk(RK_ONE), b); }
__device__ __forceinline__ double fsub(double a, double b) { return fma(b, rk(RK_MONE), a); }
__device__ __forceinline__ double kmul(int i, double x) { return fma(rk(i), x, rk(RK_NZ)); }  // rk(i) x

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
// within about one ulp of the correctly rounded 1/x.
// Valid range: normal x with |x| < 2^1022 (so that 1/x is normal too).  The
// seed flushes subnormals: a subnormal or zero x gives an infinite seed and a
// NaN result, and |x| >= 2^1022 a zero seed and result 0.  The solvers call it
// on densities, wave-speed differences and denominators that the degenerate
// branches keep away from zero, all normal for physical states.
__device__ __forceinline__ double rcp(double x) {
#if MHD_FAST_RCP
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, rk(RK_ONE));
  return fma(r, fma(e, e, e), r);
#else
  return 1.0 / x;
#endif
}

// ---------------------------------------------------------------------------
// IEEE fixed-order pieces (bitwise reproducible)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double a_(double a, double b) { return fadd(a, b); }  // = __dadd_rn
__device__ __forceinline__ double s_(double a, double b) { return fsub(a, b); }  // = __dsub_rn
__device__ __forceinline__ double m_(double a, double b) { return fmul(a, b); }  // = __dmul_rn
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
  double kin = m_(rk(RK_HALF), a_(a_(m_(mx, o.vx), m_(my, o.vy)), m_(mz, o.vz)));
  double B2 = a_(a_(m_(bx, bx), m_(by, by)), m_(bz, bz));
  o.p = m_(gm1, s_(s_(en, kin), m_(rk(RK_HALF), B2)));
  o.rho = rho;
  o.bx = bx;
  o.by = by;
  o.bz = bz;
  return o;
}

// The same recovery with one refined reciprocal and fused sums, within a few
// ulps of c2p_ieee, for the passes whose primitives decide nothing the oracle
// must reproduce bit for bit (every pass but the CFL one).  pbound receives
// 1e-14 (G-1)(|E| + (m.v + B^2)/2), far above the difference from c2p_ieee's
// pressure (about ten roundings of those magnitudes): where the pressure lies
// that close to a threshold the caller takes c2p_ieee's instead, so the floor
// and positivity decisions are the IEEE ones.
__device__ __forceinline__ Prim8 c2p_fast(double rho, double mx, double my, double mz, double en, double bx,
                                          double by, double bz, double gm1, double& pbound) {
  Prim8 o;
  const double inv = rcp(rho);
  o.vx = fmul(mx, inv);
  o.vy = fmul(my, inv);
  o.vz = fmul(mz, inv);
  const double kin2 = fma(mx, o.vx, fma(my, o.vy, fmul(mz, o.vz)));  // m.v = 2 x kinetic energy
  const double B2 = fma(bx, bx, fma(by, by, fmul(bz, bz)));
  o.p = fmul(gm1, fma(rk(RK_MHALF), kin2, fma(rk(RK_MHALF), B2, en)));
  pbound = fmul(gm1, kmul(RK_PB, fma(rk(RK_HALF), fadd(kin2, B2), fabs(en))));
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
  double disc = s_(m_(s, s), m_(m_(rk(RK_FOUR), gp), m_(bn, bn)));
  if (disc < 0.0) disc = 0.0;
  double cf2 = d_(m_(rk(RK_HALF), a_(s, __dsqrt_rn(disc))), rho);
  return __dsqrt_rn(cf2);
}

// ---------------------------------------------------------------------------
// Predicates, min/max and sign changes on the integer pipes.  On this GPU the
// FP64 pipe is the bottleneck and a double compare (DSETP) costs as much of it
// as a fused multiply-add, so comparisons, selections and sign flips use the
// bit patterns: a non-negative double orders like its bits as a signed
// integer, and key(x) = bits ^ ((bits >> 63) & 0x7fff...) orders every
// non-NaN double like a signed integer.
// ---------------------------------------------------------------------------
constexpr long long kSign = (long long)0x8000000000000000ULL;
constexpr long long kMag = 0x7fffffffffffffffLL;

__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double from_bits(long long b) { return __longlong_as_double(b); }
__device__ __forceinline__ long long order_key(double x) {
  long long b = bits(x);
  return b ^ ((b >> 63) & kMag);
}
__device__ __forceinline__ bool gt0(double x) { return bits(x) > 0; }                     // x > 0
__device__ __forceinline__ bool lt0(double x) { long long b = bits(x); return b < 0 && b != kSign; }  // x < 0
__device__ __forceinline__ bool ge0(double x) { return !lt0(x); }                         // x >= 0
__device__ __forceinline__ double imin(double a, double b) { return order_key(b) < order_key(a) ? b : a; }
__device__ __forceinline__ double imax(double a, double b) { return order_key(a) < order_key(b) ? b : a; }
// both arguments non-negative
__device__ __forceinline__ double imax_pos(double a, double b) { return bits(a) < bits(b) ? b : a; }
__device__ __forceinline__ bool lt_pos(double a, double b) { return bits(a) < bits(b); }   // a < b, b >= 0
// |x| by clearing the sign bit on the integer pipes (the same value as fabs)
__device__ __forceinline__ double dabs(double x) { return from_bits(bits(x) & kMag); }
// x * (s > 0 ? 1 : -1) by flipping the sign bit
__device__ __forceinline__ double times_sign(double x, double s) {
  return from_bits(bits(x) ^ (gt0(s) ? 0LL : kSign));
}
// -x when c, else x (the sign bit, on the integer pipes: a negated value that
// is selected or stored would otherwise be formed by an FP64 add)
__device__ __forceinline__ double neg_if(double x, bool c) { return from_bits(bits(x) ^ (c ? kSign : 0LL)); }
// lt_pos(|x|, y): false for y < 0, else |x| < y, with the bit patterns
// shifted left by one (dropping the sign), which compare like the
// magnitudes.  Clearing the sign bit with a mask instead is turned by the
// compiler into an FP64 absolute value.
__device__ __forceinline__ bool lt_abs(double x, double y) {
  return bits(y) >= 0 && ((unsigned long long)bits(x) << 1) < ((unsigned long long)bits(y) << 1);
}

// sqrt(x) and 1/sqrt(x) for x > 0 from the hardware's ~20-bit reciprocal
// square-root seed (PTX rsqrt.approx.ftz.f64), refined by one third-order
// step of the binomial series  (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ...,
// e = 1 - x y^2: relative error O(e^3) plus rounding, about one ulp.
// Valid range: positive normal x.  The seed flushes subnormals, so a
// subnormal or zero x gives NaN; fsqrt0 returns 0 for x below the smallest
// normal double (negative, zero or subnormal), and the CFL rate's fast speed
// sends a discriminant below 1e-290 to 0 before taking its root.
__device__ __forceinline__ double rsqrt_seed(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
__device__ __forceinline__ double fsqrt(double x) {
  double y = rsqrt_seed(x);
  double s = fmul(x, y);
  double e = fma(-s, y, rk(RK_ONE));
  double t = fmul(fma(rk(RK_3_8), e, rk(RK_HALF)), e);
  return fma(s, t, s);
}
__device__ __forceinline__ double frsqrt(double x) {
  double y = rsqrt_seed(x);
  double e = fma(-fmul(x, y), y, rk(RK_ONE));
  double t = fmul(fma(rk(RK_3_8), e, rk(RK_HALF)), e);
  return fma(y, t, y);
}
// sqrt(x) for any x, 0 below the smallest normal double (the seed of 0 or of a
// subnormal is infinite; sqrt of a subnormal is below 1.5e-154 anyway)
constexpr long long kMinNormalBits = 0x0010000000000000LL;
__device__ __forceinline__ double fsqrt0(double x) { return bits(x) >= kMinNormalBits ? fsqrt(x) : 0.0; }

// fast_speed_ieee with its square roots and division replaced by the refined
// seeds (about one ulp each), everything else in the same IEEE operations:
// the discriminant is bit-identical, so the result stays within ~10 ulp of
// fast_speed_ieee even where the discriminant cancels.  Used to find the
// candidates for the largest CFL rate, which fast_speed_ieee then decides.
__device__ __forceinline__ double fast_speed_near_ieee(double rho, double p, double B2, double bn, double gamma) {
  double gp = m_(gamma, p);
  double s = a_(gp, B2);
  double disc = s_(m_(s, s), m_(m_(rk(RK_FOUR), gp), m_(bn, bn)));
  double sq = lt_pos(disc, 1e-290) ? 0.0 : fsqrt(disc);  // 0 for disc <= 0 and for subnormal disc
  double cf2 = m_(m_(rk(RK_HALF), a_(s, sq)), rcp(rho));
  return fsqrt(cf2);
}
// a * b rounded once, never contracted into a neighbouring add
__device__ __forceinline__ double mul_rn(double a, double b) { return fmul(a, b); }

// ---------------------------------------------------------------------------
// Sweep-frame physics.  W = (rho, u, v, w, b1, b2, p): normal velocity u,
// transverse (v, w) and transverse field (b1, b2) in the cyclic order of the
// sweep; bn is the staggered normal field at the face.
// ---------------------------------------------------------------------------
template <class T> struct W7T {
  T rho, u, v, w, b1, b2, p;
};
template <class T> struct Flux7T {
  T f[7];  // rho, m_n, m_t1, m_t2, B_t1, B_t2, E
};
using W7 = W7T<double>;
using Flux7 = Flux7T<double>;

// Conserved state U = (rho, rho u, rho v, rho w, b1, b2, E) and flux of Eq. mhd
// along the normal (F of b_n is zero), pT = p + B^2/2, plus the fast speed.
template <class T> struct SideT {
  T U[7], F[7];
  T pT, B2, vB, cf, n;  // cf: fast speed (reverse mode), n: its numerator (forward solvers)
};
using Side = SideT<double>;

// Fast magnetosonic speed cf^2 = n / (2 rho) with the numerator
// n = (G p + B^2) + sqrt((G p + B^2)^2 - 4 G p bn^2).
template <class T>
__device__ __forceinline__ T fast_speed_num(T p, T B2, T bn2, double gamma) {
  T gp = mul_rn(T(gamma), p);
  T s = fadd(gp, B2);
  T disc = fma(s, s, -fmul(kmul(RK_FOUR, gp), bn2));
  if (lt0(disc)) disc = T(0.0);
  return fadd(s, fsqrt0(disc));
}
template <class T>
__device__ __forceinline__ T fast_speed(T rho, T p, T B2, T bn2, double gamma) {
  return fsqrt(fmul(fast_speed_num(p, B2, bn2, gamma), kmul(RK_HALF, rcp(rho))));
}
// max(cf_L, cf_R), the only use of the two fast speeds in the solvers' outer
// wave speeds, with one reciprocal and one square root: the side with the
// larger n / rho is found by comparing n_L rho_R with n_R rho_L; the result is
// that side's fast_speed (a near-tie may pick the other side, ~1 ulp away).
template <class T>
__device__ __forceinline__ T fast_speed_max(T nL, T rhoL, T nR, T rhoR) {
  const bool right = lt_pos(fmul(nL, rhoR), fmul(nR, rhoL));
  return fsqrt(fmul(right ? nR : nL, kmul(RK_HALF, rcp(right ? rhoR : rhoL))));
}

// With CF the side's fast speed goes to s.cf, else its numerator to s.n.
template <class T, bool CF = true>
__device__ __forceinline__ void side_state(const W7T<T>& W, T bn, T bn2, double gamma, double igm1, SideT<T>& s) {
  s.B2 = fma(W.b1, W.b1, fma(W.b2, W.b2, bn2));
  s.pT = fma(rk(RK_HALF), s.B2, W.p);
  s.vB = fma(W.u, bn, fma(W.v, W.b1, fmul(W.w, W.b2)));
  T v2 = fma(W.u, W.u, fma(W.v, W.v, fmul(W.w, W.w)));
  T E = fma(W.p, T(igm1), kmul(RK_HALF, fma(W.rho, v2, s.B2)));
  T mu = fmul(W.rho, W.u);
  s.U[0] = W.rho;
  s.U[1] = mu;
  s.U[2] = fmul(W.rho, W.v);
  s.U[3] = fmul(W.rho, W.w);
  s.U[4] = W.b1;
  s.U[5] = W.b2;
  s.U[6] = E;
  s.F[0] = mu;
  s.F[1] = fsub(fma(mu, W.u, s.pT), bn2);
  s.F[2] = fma(mu, W.v, -fmul(bn, W.b1));
  s.F[3] = fma(mu, W.w, -fmul(bn, W.b2));
  s.F[4] = fma(W.u, W.b1, -fmul(W.v, bn));
  s.F[5] = fma(W.u, W.b2, -fmul(W.w, bn));
  s.F[6] = fma(fadd(E, s.pT), W.u, -fmul(bn, s.vB));
  if (CF) s.cf = fast_speed(W.rho, W.p, s.B2, bn2, gamma);
  else s.n = fast_speed_num(W.p, s.B2, bn2, gamma);
}

// Outer speed estimate S_L, S_R (Miyoshi & Kusano 2005) and the UCT-HLL
// ingredients a+ = aR/(aR-aL), a- = -aL/(aR-aL), d = -aR aL/(aR-aL).  With
// the UCT-HLLD weights (riemann_hlld<T, true>) ap, am, dd, dr hold a^L, a^R,
// d^L, d^R instead.
template <class T> struct IngrT {
  T ap, am, dd, uL, uR, dr;
};
using Ingr = IngrT<double>;
template <class T>
__device__ __forceinline__ void speeds(const W7T<T>& L, const W7T<T>& R, T cmax, T& SL, T& SR, IngrT<T>& ing) {
  SL = fsub(imin(L.u, R.u), cmax);
  SR = fadd(imax(L.u, R.u), cmax);
  T aR = gt0(SR) ? SR : T(0.0), aL = lt0(SL) ? SL : T(0.0);
  T inv = rcp(fsub(aR, aL));
  ing.ap = fmul(aR, inv);
  ing.am = fmul(-aL, inv);
  ing.dd = fmul(-fmul(aR, aL), inv);
  ing.uL = L.u;
  ing.uR = R.u;
}

template <class T>
__device__ __forceinline__ void riemann_hll(const W7T<T>& L, const W7T<T>& R, T bn, double gamma, double igm1,
                                            Flux7T<T>& F, IngrT<T>& ing) {
  const T bn2 = bn * bn;
  SideT<T> sl, sr;
  side_state<T, false>(L, bn, bn2, gamma, igm1, sl);
  side_state<T, false>(R, bn, bn2, gamma, igm1, sr);
  T SL, SR;
  speeds(L, R, fast_speed_max(sl.n, L.rho, sr.n, R.rho), SL, SR, ing);
  if (ge0(SL)) {
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = sl.F[q];
  } else if (!gt0(SR)) {
#pragma unroll
    for (int q = 0; q < 7; q++) F.f[q] = sr.F[q];
  } else {
    T inv = rcp(fsub(SR, SL));
    T sls = fmul(SR, SL);
#pragma unroll
    for (int q = 0; q < 7; q++)
      F.f[q] = fmul(fma(sls, fsub(sr.U[q], sl.U[q]), fma(SR, sl.F[q], -fmul(SL, sr.F[q]))), inv);
  }
}

// Total field, total pressure and fast speed of one side (all that HLLD needs
// from both sides before the contact speed is known).
template <class T> struct SideLiteT {
  T B2, pT, cf;
};
template <class T>
__device__ __forceinline__ void side_lite(const W7T<T>& W, T bn2, double gamma, SideLiteT<T>& s) {
  s.B2 = fma(W.b1, W.b1, fma(W.b2, W.b2, bn2));
  s.pT = fma(rk(RK_HALF), s.B2, W.p);
  s.cf = fast_speed(W.rho, W.p, s.B2, bn2, gamma);
}
// The same with the fast-speed numerator (see fast_speed_max), for the forward solver.
template <class T> struct SideNumT {
  T B2, pT, n;
};
template <class T>
__device__ __forceinline__ void side_num(const W7T<T>& W, T bn2, double gamma, SideNumT<T>& s) {
  s.B2 = fma(W.b1, W.b1, fma(W.b2, W.b2, bn2));
  s.pT = fma(rk(RK_HALF), s.B2, W.p);
  s.n = fast_speed_num(W.p, s.B2, bn2, gamma);
}
// Conserved state, energy, v.B and flux of one side, given its total field and
// pressure (l: any side record with B2 and pT).
template <class T, class SideInfo>
__device__ __forceinline__ void side_full(const W7T<T>& W, T bn, T bn2, double igm1, const SideInfo& l, T U[7],
                                          T F[7], T& vB) {
  vB = fma(W.u, bn, fma(W.v, W.b1, fmul(W.w, W.b2)));
  T v2 = fma(W.u, W.u, fma(W.v, W.v, fmul(W.w, W.w)));
  T E = fma(W.p, T(igm1), kmul(RK_HALF, fma(W.rho, v2, l.B2)));
  T mu = fmul(W.rho, W.u);
  U[0] = W.rho;
  U[1] = mu;
  U[2] = fmul(W.rho, W.v);
  U[3] = fmul(W.rho, W.w);
  U[4] = W.b1;
  U[5] = W.b2;
  U[6] = E;
  F[0] = mu;
  F[1] = fsub(fma(mu, W.u, l.pT), bn2);
  F[2] = fma(mu, W.v, -fmul(bn, W.b1));
  F[3] = fma(mu, W.w, -fmul(bn, W.b2));
  F[4] = fma(W.u, W.b1, -fmul(W.v, bn));
  F[5] = fma(W.u, W.b2, -fmul(W.w, bn));
  F[6] = fma(fadd(E, l.pT), W.u, -fmul(bn, vB));
}

// HLLD (Miyoshi & Kusano 2005): waves S_L < S*_L < S_M < S*_R < S_R with
// continuous normal velocity and total pressure across the fan.  Both sides
// give their total pressure and fast speed; the star transverse states of
// both sides feed the double-star state; conserved states, energies and the
// flux are assembled only on the side of the contact that holds x/t = 0.
//
// UCT: the edge-field weights of the HLLD flux itself (UCT-HLLD).  In every
// region of the fan the flux of a transverse field component equals
// a^L F_L + a^R F_R + d^L B_L - d^R B_R with F = u B_t - v_t B_n, and with
// e = B*_t / B_t the star ratio of a side:
//   supersonic:          (1, 0, 0, 0) or (0, 1, 0, 0);
//   S_L < 0 <= S*_L:     (1, 0, S_L (e_L - 1), 0);
//   S*_L < 0 <= S*_R:    a^L = S*_R / (S*_R - S*_L), a^R = -S*_L / (S*_R - S*_L),
//                        d^L = a^L ((S_L - S*_L) e_L - S_L), d^R = a^R (S_R - (S_R - S*_R) e_R);
//   S*_R < 0 <= S_R:     (0, 1, 0, S_R (1 - e_R)).
template <class T, bool UCT = false>
__device__ __forceinline__ void riemann_hlld(const W7T<T>& L, const W7T<T>& R, T bn, double gamma, double igm1,
                                             Flux7T<T>& F, IngrT<T>& ing) {
  const T bn2 = fmul(bn, bn);
  SideNumT<T> ll, lr;
  side_num(L, bn2, gamma, ll);
  side_num(R, bn2, gamma, lr);
  // outer speeds and UCT ingredients
  T cmax = fast_speed_max(ll.n, L.rho, lr.n, R.rho);
  T SL = fsub(imin(L.u, R.u), cmax), SR = fadd(imax(L.u, R.u), cmax);
  {
    T aR = gt0(SR) ? SR : T(0.0), aL = lt0(SL) ? SL : T(0.0);
    T inv = rcp(fsub(aR, aL));
    ing.ap = fmul(aR, inv);
    ing.am = fmul(-aL, inv);
    ing.dd = fmul(-fmul(aR, aL), inv);
    ing.uL = L.u;
    ing.uR = R.u;
  }
  if (gt0(SL) || lt0(SR)) {  // supersonic: the upwind physical flux
    const bool up_left = gt0(SL);
    T U[7], vB;
    side_full(up_left ? L : R, bn, bn2, igm1, up_left ? ll : lr, U, F.f, vB);
    if (UCT) {
      ing.ap = up_left ? T(1.0) : T(0.0);
      ing.am = up_left ? T(0.0) : T(1.0);
      ing.dd = T(0.0);
      ing.dr = T(0.0);
    }
    return;
  }
  T sdL = fsub(SL, L.u), sdR = fsub(SR, R.u);
  T rsL = fmul(sdL, L.rho), rsR = fmul(sdR, R.rho);  // rho (S - u)
  T iden = rcp(fsub(rsR, rsL));
  T SM = fmul(fadd(fsub(fma(rsR, R.u, -fmul(rsL, L.u)), lr.pT), ll.pT), iden);
  T pTs = fmul(fma(fmul(fmul(L.rho, rsR), sdL), fsub(R.u, L.u), fma(rsR, ll.pT, -fmul(rsL, lr.pT))), iden);

  // star transverse states of both sides
  T smL = fsub(SL, SM), smR = fsub(SR, SM);
  T ismL = rcp(smL), ismR = rcp(smR);
  T rhosL = fmul(rsL, ismL), rhosR = fmul(rsR, ismR);
  T vsL, wsL, b1sL, b2sL, vsR, wsR, b1sR, b2sR;
  T eL(1.0), eR(1.0);  // star ratios B*_t / B_t (UCT weights)
  {
    T rsm = mul_rn(rsL, smL), D = fsub(rsm, bn2);
    if (lt_abs(D, kmul(RK_EPS, rsm))) {
      vsL = L.v; wsL = L.w; b1sL = L.b1; b2sL = L.b2;
    } else {
      T iD = rcp(D);
      T cv = fmul(fmul(bn, fsub(SM, L.u)), iD);
      vsL = fma(-L.b1, cv, L.v);
      wsL = fma(-L.b2, cv, L.w);
      T cb = fmul(fma(rsL, sdL, -bn2), iD);
      b1sL = fmul(L.b1, cb);
      b2sL = fmul(L.b2, cb);
      if (UCT) eL = cb;
    }
  }
  {
    T rsm = mul_rn(rsR, smR), D = fsub(rsm, bn2);
    if (lt_abs(D, kmul(RK_EPS, rsm))) {
      vsR = R.v; wsR = R.w; b1sR = R.b1; b2sR = R.b2;
    } else {
      T iD = rcp(D);
      T cv = fmul(fmul(bn, fsub(SM, R.u)), iD);
      vsR = fma(-R.b1, cv, R.v);
      wsR = fma(-R.b2, cv, R.w);
      T cb = fmul(fma(rsR, sdR, -bn2), iD);
      b1sR = fmul(R.b1, cb);
      b2sR = fmul(R.b2, cb);
      if (UCT) eR = cb;
    }
  }
  if (UCT) {  // the single-star region of the contact's side; replaced below in the double-star one
    const bool lc = ge0(SM);
    ing.ap = lc ? T(1.0) : T(0.0);
    ing.am = lc ? T(0.0) : T(1.0);
    ing.dd = lc ? fmul(SL, fsub(eL, T(1.0))) : T(0.0);
    ing.dr = lc ? T(0.0) : fmul(SR, fsub(T(1.0), eR));
  }
  // the side of the contact that contains x/t = 0
  const bool left = ge0(SM);
  const W7T<T>& A = left ? L : R;
  T Ua[7], vBa;
  side_full(A, bn, bn2, igm1, left ? ll : lr, Ua, F.f, vBa);
  const T pTa = left ? ll.pT : lr.pT;
  const T S = left ? SL : SR, sd = left ? sdL : sdR, ism = left ? ismL : ismR;
  const T rhos = left ? rhosL : rhosR;
  const T vs = left ? vsL : vsR, ws = left ? wsL : wsR, b1s = left ? b1sL : b1sR, b2s = left ? b2sL : b2sR;
  T vBs = fma(SM, bn, fma(vs, b1s, fmul(ws, b2s)));
  T Es = fmul(fadd(fma(sd, Ua[6], -fmul(pTa, A.u)), fma(pTs, SM, fmul(bn, fsub(vBa, vBs)))), ism);
  T Us[7] = {rhos, fmul(rhos, SM), fmul(rhos, vs), fmul(rhos, ws), b1s, b2s, Es};
#pragma unroll
  for (int q = 0; q < 7; q++) F.f[q] = fma(S, fsub(Us[q], Ua[q]), F.f[q]);
  // rotational (Alfven) waves, absent when the normal field vanishes
  if (!lt_pos(bn2, kmul(RK_2EPS, pTs))) {  // 0.5 bn2 >= eps pTs, scaled by 2 exactly
    T iqL = frsqrt(rhosL), iqR = frsqrt(rhosR);  // 1/sqrt(rho*)
    T sqL = fmul(rhosL, iqL), sqR = fmul(rhosR, iqR);  // sqrt(rho*)
    T abn = dabs(bn);
    T Ss = left ? fma(-abn, iqL, SM) : fma(abn, iqR, SM);
    bool beyond = left ? lt0(Ss) : ge0(Ss);      // x/t = 0 lies between S*_a and S_M
    if (UCT && beyond) {                         // S*_L < 0 <= S*_R
      T SsL = fma(-abn, iqL, SM), SsR = fma(abn, iqR, SM);
      T iw = rcp(fsub(SsR, SsL));
      T aL = fmul(SsR, iw), aR = fmul(-SsL, iw);
      ing.ap = aL;
      ing.am = aR;
      ing.dd = fmul(aL, fma(fsub(SL, SsL), eL, -SL));
      ing.dr = fmul(aR, fma(fsub(SsR, SR), eR, SR));
    }
    if (beyond) {
      T isum = rcp(fadd(sqL, sqR));
      T vss = fmul(fma(sqL, vsL, fma(sqR, vsR, times_sign(fsub(b1sR, b1sL), bn))), isum);
      T wss = fmul(fma(sqL, wsL, fma(sqR, wsR, times_sign(fsub(b2sR, b2sL), bn))), isum);
      T sq2 = fmul(sqL, sqR);
      T b1ss = fmul(fma(sqL, b1sR, fma(sqR, b1sL, times_sign(fmul(sq2, fsub(vsR, vsL)), bn))), isum);
      T b2ss = fmul(fma(sqL, b2sR, fma(sqR, b2sL, times_sign(fmul(sq2, fsub(wsR, wsL)), bn))), isum);
      T vBss = fma(SM, bn, fma(vss, b1ss, fmul(wss, b2ss)));
      // Es + s_a sign(B_n) (vB* - vB**) with s_a = -sqrt(rho*_L) on the left, sqrt(rho*_R) on the
      // right: both signs go into one flip of the difference
      T Ess = fma(left ? sqL : sqR, neg_if(fsub(vBs, vBss), gt0(bn) == left), Es);
      // F += S*_a (U** - U*): the density and normal momentum are continuous
      F.f[2] = fma(Ss, fma(rhos, vss, -Us[2]), F.f[2]);
      F.f[3] = fma(Ss, fma(rhos, wss, -Us[3]), F.f[3]);
      F.f[4] = fma(Ss, fsub(b1ss, b1s), F.f[4]);
      F.f[5] = fma(Ss, fsub(b2ss, b2s), F.f[5]);
      F.f[6] = fma(Ss, fsub(Ess, Es), F.f[6]);
    }
  }
}

// ---------------------------------------------------------------------------
// Reconstruction (Eq. reconstruct).  s0..s4 = V_{i-2..i+2}; plus = V^L_{i+1/2},
// minus = V^R_{i-1/2}.
// ---------------------------------------------------------------------------
// minmod(a, b): 0 when the signs differ (or either is 0), else the argument of
// smaller magnitude, on integer pipes.  For two doubles of the same sign the
// bit patterns, read as signed integers, order like the magnitudes (the
// magnitude bits sit below the sign bit), so no mask is needed; a masked
// compare (bits & 0x7fff...) is turned by the compiler into two FP64 absolute
// values, 2 of the FP64 pipe's instructions per call.
__device__ __forceinline__ double minmod(double a, double b) {
  long long ia = bits(a), ib = bits(b);
  if ((ia ^ ib) < 0) return 0.0;
  return ib < ia ? b : a;
}

// PLM from the two one-sided differences of cell value s2 (a marching sweep
// carries the right difference of a cell over as the left one of the next).
__device__ __forceinline__ void recon_plm_d(double s2, double dl, double dr, double& plus, double& minus) {
  double d = minmod(dl, dr);
  plus = fma(rk(RK_HALF), d, s2);
  minus = fma(rk(RK_MHALF), d, s2);
}
__device__ __forceinline__ void recon_plm(double s1, double s2, double s3, double& plus, double& minus) {
  recon_plm_d(s2, fsub(s2, s1), fsub(s3, s2), plus, minus);
}

// WENO-Z (Borges et al. 2008) values at both faces of the middle cell of
// a0..a4 = V_{i-2..i+2}: candidate values q_k, Jiang-Shu indicators beta_k,
// tau5 = |beta_0 - beta_2|, alpha_k = d_k (1 + (tau5 / (beta_k + eps))^2),
// d = (1/10, 6/10, 3/10), value = sum alpha_k q_k / sum alpha_k.  The
// mirrored (minus-face) stencil has the same indicators with beta_0 and
// beta_2 exchanged, so the ratios r_k = tau5 / (beta_k + eps) and the factors
// g_k = 1 + r_k^2 are formed once for both faces, and so is the middle
// weight d_1 g_1.  The candidates are formed as 6 q_k and the normalisation
// as 6 sum_k alpha_k = sum_k (6 d_k) g_k.
// Two of the minus face's candidates are the plus-face candidates of the
// cell before: both faces meet at x_{i-1/2}, where the stencils of cells
// i-2..i and i-1..i+1 give one value whichever cell they are seen from.  So
// qm1, qm2 (6 q_1, 6 q_2 of the minus face) come in, and the plus face's
// 6 q_2, 6 q_1 -- the next cell's qm1, qm2 -- go out in the same variables.
__device__ __forceinline__ void wenoz_from_indicators(double a0, double a1, double a2, double a3, double a4,
                                                      double be0, double be1, double be2, double& qm1,
                                                      double& qm2, double& plus, double& minus) {
  // be_k = s (beta_k + eps), the epsilon already added in a free addend slot
  // of the indicators' FMAs, with s = 1 (marching sweep) or 4 (recon_wenoz_c):
  // an exact power of two, so it cancels in the ratios to the bit; tau5 =
  // |be_0 - be_2| / s up to its sign, which the squares of r_k drop
  const double tau = fsub(be0, be2);
  const double r0 = fmul(tau, rcp(be0));
  const double r1 = fmul(tau, rcp(be1));
  const double r2 = fmul(tau, rcp(be2));
  const double g0 = fma(r0, r0, rk(RK_ONE)), g1 = fma(r1, r1, rk(RK_ONE)), g2 = fma(r2, r2, rk(RK_ONE));
  // alpha_k = d_k g_k: the plus face weighs (g0, g1, g2), the minus face (g2, g1, g0)
  const double w1 = kmul(RK_0_6, g1);
  const double K1 = kmul(RK_3_6, g1);  // 6 d_1 g_1
  {  // plus face: stencils (a0 a1 a2), (a1 a2 a3), (a2 a3 a4); 6 q_k, and 6 d_0 q_0 with d_0
     // folded into the stencil's coefficients (q_0 is used by one face only)
    const double q0 = fma(rk(RK_0_2), a0, fma(rk(RK_M0_7), a1, kmul(RK_1_1, a2)));
    const double q1 = fma(rk(RK_5), a2, fma(rk(RK_2), a3, -a1));
    const double q2 = fma(rk(RK_2), a2, fma(rk(RK_5), a3, -a4));
    const double num = fma(g0, q0, fma(w1, q1, fmul(kmul(RK_0_3, g2), q2)));
    const double den = fma(rk(RK_0_6), g0, fma(rk(RK_1_8), g2, K1));  // 6 sum alpha_k
    plus = fmul(num, rcp(den));
    // minus face: the mirrored stencils with g2, g1, g0; q1, q2 from the cell before
    const double q0m = fma(rk(RK_0_2), a4, fma(rk(RK_M0_7), a3, kmul(RK_1_1, a2)));
    const double numm = fma(g2, q0m, fma(w1, qm1, fmul(kmul(RK_0_3, g0), qm2)));
    const double denm = fma(rk(RK_0_6), g2, fma(rk(RK_1_8), g0, K1));
    minus = fmul(numm, rcp(denm));
    qm1 = q2;
    qm2 = q1;
  }
}

// The minus face's 6 q_1 and 6 q_2 of the cell whose window starts with
// a0..a3, formed as the plus face of the cell before forms them (its q_2 and
// q_1), so that a march gives the same bits wherever it starts.
__device__ __forceinline__ void wenoz_minus_q12(double a0, double a1, double a2, double a3, double& qm1,
                                                double& qm2) {
  qm1 = fma(rk(RK_2), a1, fma(rk(RK_5), a2, -a3));
  qm2 = fma(rk(RK_5), a1, fma(rk(RK_2), a2, -a0));
}

// beta_k = (13/12) (a_{j-1} - 2 a_j + a_{j+1})^2 + (1/4) u_k^2, the curvature
// term belonging to the three-cell stencil centred at j = i-1, i, i+1 and u_k
// the stencil's one-sided combination.  A sweep marching along a pencil
// carries, per variable, what consecutive cells share (WzCarry for the window
// of cell i):
//   P0, P1 = the curvature terms of the stencils centred at a1 and a2, each
//            plus the WENO-Z epsilon (so every indicator arrives as beta + eps),
//   h      = u_0 / 2 = (a0 - 4 a1 + 3 a2) / 2,
//   d      = a3 - a2,
//   m1, m2 = 6 q_1, 6 q_2 of the minus face (wenoz_from_indicators).
// With t2 = (a4 - a3) - d the curvature at a3, u_2 / 2 = t2 / 2 - d and
// u_1 / 2 = (a1 - a3) / 2; the next cell's u_0 / 2 = u_1 / 2 + 2 d.
// wenoz_start forms the carry of a segment's first window with the very
// operations the march would have used (differences of neighbours, their
// difference, (a0 - a2)/2 + 2 (a2 - a1)), so every cell's result is the same
// to the bit wherever a segment starts.  (The march keeps the halved u_k:
// the scaled form of recon_wenoz_c, one instruction fewer per cell and
// variable, measured 2.5 % slower in these sweeps.)
struct WzCarry {
  double P0, P1, h, d, m1, m2;
};
__device__ __forceinline__ WzCarry wenoz_start(double a0, double a1, double a2, double a3) {
  WzCarry c;
  const double d01 = fsub(a1, a0), d12 = fsub(a2, a1);
  c.d = fsub(a3, a2);
  const double t0 = fsub(d12, d01), t1 = fsub(c.d, d12);
  c.P0 = fma(kmul(RK_13_12, t0), t0, rk(RK_WEPS));
  c.P1 = fma(kmul(RK_13_12, t1), t1, rk(RK_WEPS));
  c.h = fma(rk(RK_2), d12, fma(rk(RK_HALF), a0, kmul(RK_MHALF, a2)));
  wenoz_minus_q12(a0, a1, a2, a3, c.m1, c.m2);
  return c;
}
__device__ __forceinline__ void recon_wenoz_m(double a0, double a1, double a2, double a3, double a4, WzCarry& c,
                                              double& plus, double& minus) {
  const double d34 = fsub(a4, a3);
  const double t2 = fsub(d34, c.d);
  const double P2 = fma(kmul(RK_13_12, t2), t2, rk(RK_WEPS));
  const double h2 = fma(rk(RK_HALF), t2, -c.d);                  // (3 a2 - 4 a3 + a4) / 2
  const double h1 = fma(rk(RK_HALF), a1, kmul(RK_MHALF, a3));    // (a1 - a3) / 2
  const double b0 = fma(c.h, c.h, c.P0);
  const double b1 = fma(h1, h1, c.P1);
  const double b2 = fma(h2, h2, P2);
  c.h = fma(rk(RK_2), c.d, h1);                                  // (a1 - 4 a2 + 3 a3) / 2, for cell i+1
  c.P0 = c.P1;
  c.P1 = P2;
  c.d = d34;
  wenoz_from_indicators(a0, a1, a2, a3, a4, b0, b1, b2, c.m1, c.m2, plus, minus);
}

// The same reconstruction from the curvatures alone (the GLM sweep carries
// two per variable): c0, c1 of the stencils centred at a1, a2 in, that of a3
// out in c2.  The indicators are formed as 4 (beta_k + eps) = (13/3) t^2 +
// u_k^2 + 4 eps: each term is the unscaled one times an exact power of two
// (13/3 = 4 x 13/12 and 4 eps are exact scalings in binary), so the ratios
// are the same to the bit, and the factor 1/4 of u_k^2 goes away.
struct Curv {
  double t, k;  // a_{j-1} - 2 a_j + a_{j+1} and 13/3 of it
};
__device__ __forceinline__ Curv curv_of(double t) {
  Curv c;
  c.t = t;
  c.k = kmul(RK_13_3, t);
  return c;
}
__device__ __forceinline__ Curv curv(double l, double m, double r) { return curv_of(fadd(fma(rk(RK_M2), m, l), r)); }
__device__ __forceinline__ void recon_wenoz_c(double a0, double a1, double a2, double a3, double a4, const Curv& c0,
                                              const Curv& c1, Curv& c2, double& plus, double& minus) {
  // 4 (beta_k + eps), the epsilon in the one-sided term's addend slot
  double u = fma(rk(RK_3), a2, fma(rk(RK_M4), a1, a0));
  double b0 = fma(c0.k, c0.t, fma(u, u, rk(RK_4WEPS)));
  u = fsub(a1, a3);
  double b1 = fma(c1.k, c1.t, fma(u, u, rk(RK_4WEPS)));
  c2 = curv(a2, a3, a4);
  u = fma(rk(RK_3), a2, fma(rk(RK_M4), a3, a4));
  double b2 = fma(c2.k, c2.t, fma(u, u, rk(RK_4WEPS)));
  double qm1, qm2;
  wenoz_minus_q12(a0, a1, a2, a3, qm1, qm2);
  wenoz_from_indicators(a0, a1, a2, a3, a4, b0, b1, b2, qm1, qm2, plus, minus);
}
__device__ __forceinline__ void recon_wenoz(double a0, double a1, double a2, double a3, double a4, double& plus,
                                            double& minus) {
  WzCarry c = wenoz_start(a0, a1, a2, a3);
  recon_wenoz_m(a0, a1, a2, a3, a4, c, plus, minus);
}

__device__ __forceinline__ double ppm_face(double a, double b, double c, double d) {
  double f = fma(rk(RK_7_12), fadd(b, c), -kmul(RK_1_12, fadd(a, d)));
  double lo = imin(b, c), hi = imax(b, c);
  return imin(imax(f, lo), hi);
}
// Piecewise-parabolic (Colella & Woodward 1984), method-of-lines form:
// fourth-order face values clipped to their neighbours, then the parabola of
// the cell flattened at an extremum or steepened on the overshooting side.
__device__ __forceinline__ void recon_ppm(double s0, double s1, double s2, double s3, double s4, double& plus,
                                          double& minus) {
  double vp = ppm_face(s1, s2, s3, s4);
  double vm = ppm_face(s0, s1, s2, s3);
  if (!gt0(fmul(fsub(vp, s2), fsub(s2, vm)))) {
    vp = s2;
    vm = s2;
  } else {
    double dv = fsub(vp, vm);
    double v6 = kmul(RK_6, fma(rk(RK_MHALF), fadd(vm, vp), s2));
    double x = fmul(dv, v6), y = fmul(dv, dv);
    if (order_key(y) < order_key(x)) vm = fma(rk(RK_3), s2, -kmul(RK_2, vp));
    else if (order_key(x) < ~bits(y)) vp = fma(rk(RK_3), s2, -kmul(RK_2, vm));  // x < -y: y >= 0, key(-y) = ~bits(y)
  }
  plus = vp;
  minus = vm;
}

}  // namespace mhd
