// Hand-written reverse (vector-Jacobian product) of the HLL and HLLD solvers
// of mhd_math.cuh.  Each function first repeats the forward arithmetic of its
// solver, with the same operations in the same order, so that every branch
// (wave fan, degeneracies, min/max, clamps) is decided by the same values;
// it then walks the operations backwards, accumulating cotangents.  The
// derivative conventions are those of the forward-mode numbers of
// mhd_dual.cuh: a clamped or selected quantity passes the derivative of the
// branch taken, sqrt(0) has derivative 0.
#pragma once
#include "mhd_math.cuh"

namespace mhd {

// Cotangents of one side's sweep-frame primitives W = (rho, u, v, w, b1, b2, p).
struct W7b {
  double rho = 0.0, u = 0.0, v = 0.0, w = 0.0, b1 = 0.0, b2 = 0.0, p = 0.0;
};

// fast_speed: cotangents of rho, p, B2, bn2 from that of cf.
__device__ __forceinline__ void fast_speed_vjp(double rho, double p, double B2, double bn2, double gamma, double cfb,
                                               double& rhob, double& pb, double& B2b, double& bn2b) {
  const double gp = mul_rn(gamma, p);
  const double s = fadd(gp, B2);
  double disc = fma(s, s, fmul(-(kmul(RK_FOUR, gp)), bn2));
  if (lt0(disc)) disc = 0.0;
  const double sq = fsqrt0(disc);
  const double irho = rcp(rho);
  const double h = kmul(RK_HALF, irho);
  const double t = fadd(s, sq);
  const double cf = fsqrt(fmul(t, h));
  // reverse
  const double cf2b = fmul(cfb, (kmul(RK_HALF, rcp(cf))));
  const double tb = fmul(cf2b, h);
  rhob = fma((kmul(RK_HALF, (fmul(cf2b, t)))), (-(fmul(irho, irho))), rhob);
  double sb = tb, gpb = 0.0;
  if (gt0(disc)) {
    const double discb = fmul(tb, (kmul(RK_HALF, rcp(sq))));
    sb = fma(discb, (kmul(RK_2, s)), sb);
    gpb = fma(discb, (kmul(RK_M4, bn2)), gpb);
    bn2b = fma(discb, (kmul(RK_M4, gp)), bn2b);
  }
  gpb = fadd(gpb, sb);
  B2b = fadd(B2b, sb);
  pb = fma(gamma, gpb, pb);
}

// Total field and total pressure of one side (side_num): cotangents of W
// and bn2 from those of B2 (direct uses) and pT.
__device__ __forceinline__ void side_num_vjp(const W7& W, double B2b, double pTb, W7b& Wb, double& bn2b) {
  Wb.p = fadd(Wb.p, pTb);
  B2b = fma(rk(RK_HALF), pTb, B2b);
  Wb.b1 = fma((kmul(RK_2, W.b1)), B2b, Wb.b1);
  Wb.b2 = fma((kmul(RK_2, W.b2)), B2b, Wb.b2);
  bn2b = fadd(bn2b, B2b);
}

// Conserved state U, flux F and v.B of one side (side_full) given its B2 and
// pT: cotangents of W, bn, bn2, B2 and pT from those of U, F and v.B.
__device__ __forceinline__ void side_full_vjp(const W7& W, double bn, double igm1, double B2, double pT,
                                              const double Ub[7], const double Fb[7], double vBb, W7b& Wb,
                                              double& bnb, double& bn2b, double& B2b, double& pTb) {
  const double vB = fma(W.u, bn, fma(W.v, W.b1, fmul(W.w, W.b2)));
  const double v2 = fma(W.u, W.u, fma(W.v, W.v, fmul(W.w, W.w)));
  const double E = fma(W.p, igm1, kmul(RK_HALF, fma(W.rho, v2, B2)));
  const double mu = fmul(W.rho, W.u);
  double mub = fadd(Fb[0], Ub[1]);
  double Eb = Ub[6];
  // F1 = mu u + pT - bn2
  mub = fma(Fb[1], W.u, mub);
  Wb.u = fma(Fb[1], mu, Wb.u);
  pTb = fadd(pTb, Fb[1]);
  bn2b = fsub(bn2b, Fb[1]);
  // F2 = mu v - bn b1, F3 = mu w - bn b2
  mub = fma(Fb[2], W.v, fma(Fb[3], W.w, mub));
  Wb.v = fma(Fb[2], mu, Wb.v);
  Wb.w = fma(Fb[3], mu, Wb.w);
  bnb = fma(-Fb[2], W.b1, fma(-Fb[3], W.b2, bnb));
  Wb.b1 = fma(-Fb[2], bn, Wb.b1);
  Wb.b2 = fma(-Fb[3], bn, Wb.b2);
  // F4 = u b1 - v bn, F5 = u b2 - w bn
  Wb.u = fma(Fb[4], W.b1, fma(Fb[5], W.b2, Wb.u));
  Wb.b1 = fma(Fb[4], W.u, Wb.b1);
  Wb.b2 = fma(Fb[5], W.u, Wb.b2);
  Wb.v = fma(-Fb[4], bn, Wb.v);
  Wb.w = fma(-Fb[5], bn, Wb.w);
  bnb = fma(-Fb[4], W.v, fma(-Fb[5], W.w, bnb));
  // F6 = (E + pT) u - bn vB
  Eb = fma(Fb[6], W.u, Eb);
  pTb = fma(Fb[6], W.u, pTb);
  Wb.u = fma(Fb[6], (fadd(E, pT)), Wb.u);
  bnb = fma(-Fb[6], vB, bnb);
  vBb = fma(-Fb[6], bn, vBb);
  // U = (rho, mu, rho v, rho w, b1, b2, E)
  Wb.rho = fma(Ub[2], W.v, fma(Ub[3], W.w, fadd(Wb.rho, Ub[0])));
  Wb.v = fma(Ub[2], W.rho, Wb.v);
  Wb.w = fma(Ub[3], W.rho, Wb.w);
  Wb.b1 = fadd(Wb.b1, Ub[4]);
  Wb.b2 = fadd(Wb.b2, Ub[5]);
  // mu = rho u
  Wb.rho = fma(mub, W.u, Wb.rho);
  Wb.u = fma(mub, W.rho, Wb.u);
  // E = p/(G-1) + (rho v2 + B2)/2
  Wb.p = fma(Eb, igm1, Wb.p);
  Wb.rho = fma((kmul(RK_HALF, Eb)), v2, Wb.rho);
  const double v2b = fmul((kmul(RK_HALF, Eb)), W.rho);
  B2b = fma(rk(RK_HALF), Eb, B2b);
  Wb.u = fma((kmul(RK_2, W.u)), v2b, Wb.u);
  Wb.v = fma((kmul(RK_2, W.v)), v2b, Wb.v);
  Wb.w = fma((kmul(RK_2, W.w)), v2b, Wb.w);
  // vB = u bn + v b1 + w b2
  Wb.u = fma(vBb, bn, Wb.u);
  bnb = fma(vBb, W.u, bnb);
  Wb.v = fma(vBb, W.b1, Wb.v);
  Wb.b1 = fma(vBb, W.v, Wb.b1);
  Wb.w = fma(vBb, W.b2, Wb.w);
  Wb.b2 = fma(vBb, W.w, Wb.b2);
}

// Outer speeds and UCT ingredients (speeds / the head of riemann_hlld), with
// cmax = max(cf_L, cf_R) as fast_speed_max forms it: cotangents of uL, uR
// and cmax from those of the ingredients and of SL, SR.
__device__ __forceinline__ void speeds_vjp(double uL, double uR, double cmax, const double Ib[5], double SLb,
                                           double SRb, double& uLb, double& uRb, double& cmaxb) {
  const bool min_right = order_key(uR) < order_key(uL);     // imin picks uR
  const bool max_right = order_key(uL) < order_key(uR);     // imax picks uR
  const double SL = fsub((min_right ? uR : uL), cmax);
  const double SR = fadd((max_right ? uR : uL), cmax);
  const double aR = gt0(SR) ? SR : 0.0, aL = lt0(SL) ? SL : 0.0;
  const double inv = rcp(fsub(aR, aL));
  // ap = aR inv, am = -aL inv, dd = -(aR aL) inv
  const double invb = fma(Ib[0], aR, fma(-Ib[1], aL, fmul(-Ib[2], (fmul(aR, aL)))));
  double aRb = fmul(fma(-Ib[2], aL, Ib[0]), inv);
  double aLb = fmul(fma(-Ib[2], aR, -Ib[1]), inv);
  const double denb = fmul(invb, (-(fmul(inv, inv))));
  aRb = fadd(aRb, denb);
  aLb = fsub(aLb, denb);
  if (gt0(SR)) SRb += aRb;
  if (lt0(SL)) SLb += aLb;
  uLb = fadd(uLb, Ib[3]);
  uRb = fadd(uRb, Ib[4]);
  if (max_right) uRb += SRb;
  else uLb += SRb;
  if (min_right) uRb += SLb;
  else uLb += SLb;
  cmaxb = fadd(cmaxb, fsub(SRb, SLb));
}

// The side that sets cmax (fast_speed_max's choice) and the reverse of its
// fast speed: cotangents of that side's rho, p, B2 and of bn2 from cmax's.
__device__ __forceinline__ bool cmax_right(double nL, double rhoL, double nR, double rhoR) {
  return lt_pos(fmul(nL, rhoR), fmul(nR, rhoL));
}
__device__ __forceinline__ void cmax_vjp(const W7& L, const W7& R, bool right, double B2L, double B2R, double bn2,
                                         double gamma, double cmaxb, W7b& Lb, W7b& Rb, double& B2bL, double& B2bR,
                                         double& bn2b) {
  const W7& W = right ? R : L;
  double rhob = 0.0, pb = 0.0, B2b = 0.0;
  fast_speed_vjp(W.rho, W.p, right ? B2R : B2L, bn2, gamma, cmaxb, rhob, pb, B2b, bn2b);
  if (right) { Rb.rho += rhob; Rb.p += pb; B2bR += B2b; }
  else { Lb.rho += rhob; Lb.p += pb; B2bL += B2b; }
}

// ---------------------------------------------------------------------------
// HLL
// ---------------------------------------------------------------------------
__device__ __forceinline__ void riemann_hll_vjp(const W7& L, const W7& R, double bn, double gamma, double igm1,
                                                const double Fb[7], const double Ib[5], W7b& Lb, W7b& Rb,
                                                double& bnb) {
  const double bn2 = fmul(bn, bn);
  Side sl, sr;
  side_state<double, false>(L, bn, bn2, gamma, igm1, sl);
  side_state<double, false>(R, bn, bn2, gamma, igm1, sr);
  const bool c_right = cmax_right(sl.n, L.rho, sr.n, R.rho);
  const double cmax = fast_speed_max(sl.n, L.rho, sr.n, R.rho);
  const double SL = fsub(imin(L.u, R.u), cmax), SR = fadd(imax(L.u, R.u), cmax);
  double ULb[7] = {0, 0, 0, 0, 0, 0, 0}, FLb[7] = {0, 0, 0, 0, 0, 0, 0};
  double URb[7] = {0, 0, 0, 0, 0, 0, 0}, FRb[7] = {0, 0, 0, 0, 0, 0, 0};
  double SLb = 0.0, SRb = 0.0;
  if (ge0(SL)) {
#pragma unroll
    for (int q = 0; q < 7; q++) FLb[q] = Fb[q];
  } else if (!gt0(SR)) {
#pragma unroll
    for (int q = 0; q < 7; q++) FRb[q] = Fb[q];
  } else {
    // F = (SR SL (UR - UL) + SR FL - SL FR) inv,  inv = 1/(SR - SL)
    const double inv = rcp(fsub(SR, SL));
    const double sls = fmul(SR, SL);
    double invb = 0.0, slsb = 0.0;
#pragma unroll
    for (int q = 0; q < 7; q++) {
      const double dU = fsub(sr.U[q], sl.U[q]);
      const double N = fma(sls, dU, fma(SR, sl.F[q], fmul(-SL, sr.F[q])));
      const double Nb = fmul(Fb[q], inv);
      invb = fma(Fb[q], N, invb);
      slsb = fma(Nb, dU, slsb);
      URb[q] = fma(Nb, sls, URb[q]);
      ULb[q] = fma(-Nb, sls, ULb[q]);
      SRb = fma(Nb, sl.F[q], SRb);
      FLb[q] = fma(Nb, SR, FLb[q]);
      SLb = fma(-Nb, sr.F[q], SLb);
      FRb[q] = fma(-Nb, SL, FRb[q]);
    }
    SRb = fma(slsb, SL, SRb);
    SLb = fma(slsb, SR, SLb);
    const double db = fmul(invb, (-(fmul(inv, inv))));
    SRb = fadd(SRb, db);
    SLb = fsub(SLb, db);
  }
  double uLb = 0.0, uRb = 0.0, cmaxb = 0.0;
  speeds_vjp(L.u, R.u, cmax, Ib, SLb, SRb, uLb, uRb, cmaxb);
  Lb.u = fadd(Lb.u, uLb);
  Rb.u = fadd(Rb.u, uRb);
  double bn2b = 0.0, B2bL = 0.0, pTbL = 0.0, B2bR = 0.0, pTbR = 0.0;
  side_full_vjp(L, bn, igm1, sl.B2, sl.pT, ULb, FLb, 0.0, Lb, bnb, bn2b, B2bL, pTbL);
  side_full_vjp(R, bn, igm1, sr.B2, sr.pT, URb, FRb, 0.0, Rb, bnb, bn2b, B2bR, pTbR);
  cmax_vjp(L, R, c_right, sl.B2, sr.B2, bn2, gamma, cmaxb, Lb, Rb, B2bL, B2bR, bn2b);
  side_num_vjp(L, B2bL, pTbL, Lb, bn2b);
  side_num_vjp(R, B2bR, pTbR, Rb, bn2b);
  bnb = fma((kmul(RK_2, bn)), bn2b, bnb);
}

// ---------------------------------------------------------------------------
// HLLD
// ---------------------------------------------------------------------------
// Star transverse state of one side (both branches of riemann_hlld), with the
// intermediates the reverse needs.
struct StarT {
  double sd, rs, sm, ism, rhos, vs, ws, b1s, b2s;
  double iD, cv, cb;  // regular branch only
  bool degen;
};
__device__ __forceinline__ void star_side(const W7& W, double S, double SM, double bn, double bn2, StarT& t) {
  t.sd = fsub(S, W.u);
  t.rs = fmul(t.sd, W.rho);
  t.sm = fsub(S, SM);
  t.ism = rcp(t.sm);
  t.rhos = fmul(t.rs, t.ism);
  const double rsm = mul_rn(t.rs, t.sm), D = fsub(rsm, bn2);
  t.degen = lt_abs(D, fmul(kHlldDegenEps, rsm));
  if (t.degen) {
    t.vs = W.v; t.ws = W.w; t.b1s = W.b1; t.b2s = W.b2;
    t.iD = t.cv = t.cb = 0.0;
  } else {
    t.iD = rcp(D);
    t.cv = fmul((fmul(bn, (fsub(SM, W.u)))), t.iD);
    t.vs = fma(-W.b1, t.cv, W.v);
    t.ws = fma(-W.b2, t.cv, W.w);
    t.cb = fmul(fma(t.rs, t.sd, -bn2), t.iD);
    t.b1s = fmul(W.b1, t.cb);
    t.b2s = fmul(W.b2, t.cb);
  }
}
// Cotangents of one side's star quantities, accumulated by the reverse.
struct StarB {
  double rhos = 0.0, vs = 0.0, ws = 0.0, b1s = 0.0, b2s = 0.0, ism = 0.0, sd = 0.0, rs = 0.0;
  double cb = 0.0;  // the star ratio e = B*_t / B_t itself (UCT-HLLD weights)
};
// Reverse of star_side down to rs and sd (their own reverse, rs = sd rho and
// sd = S - u, runs after the contact-speed reverse has added to them).
template <bool UCT = false>
__device__ __forceinline__ void star_side_vjp(const W7& W, double SM, double bn, double bn2, const StarT& t, StarB& b,
                                              W7b& Wb, double& Sb, double& SMb, double& bnb, double& bn2b) {
  double smb = 0.0;
  if (t.degen) {
    Wb.v = fadd(Wb.v, b.vs);
    Wb.w = fadd(Wb.w, b.ws);
    Wb.b1 = fadd(Wb.b1, b.b1s);
    Wb.b2 = fadd(Wb.b2, b.b2s);
  } else {
    Wb.b1 = fma(b.b1s, t.cb, fma(-b.vs, t.cv, Wb.b1));
    Wb.b2 = fma(b.b2s, t.cb, fma(-b.ws, t.cv, Wb.b2));
    Wb.v = fadd(Wb.v, b.vs);
    Wb.w = fadd(Wb.w, b.ws);
    const double cbb = UCT ? fma(b.b1s, W.b1, fma(b.b2s, W.b2, b.cb)) : fma(b.b1s, W.b1, fmul(b.b2s, W.b2));
    const double cvb = fma(-b.vs, W.b1, -(fmul(b.ws, W.b2)));
    // cb = (rs sd - bn2) iD
    const double Nbb = fmul(cbb, t.iD);
    double iDb = fmul(cbb, fma(t.rs, t.sd, -bn2));
    b.rs = fma(Nbb, t.sd, b.rs);
    b.sd = fma(Nbb, t.rs, b.sd);
    bn2b = fsub(bn2b, Nbb);
    // cv = bn (SM - u) iD
    const double du = fsub(SM, W.u);
    const double Nvb = fmul(cvb, t.iD);
    iDb = fma(cvb, (fmul(bn, du)), iDb);
    bnb = fma(Nvb, du, bnb);
    SMb = fma(Nvb, bn, SMb);
    Wb.u = fma(-Nvb, bn, Wb.u);
    // iD = 1/D, D = rs sm - bn2
    const double Db = fmul(iDb, (-(fmul(t.iD, t.iD))));
    bn2b = fsub(bn2b, Db);
    b.rs = fma(Db, t.sm, b.rs);
    smb = fma(Db, t.rs, smb);
  }
  // rhos = rs ism, ism = 1/sm, sm = S - SM
  b.rs = fma(b.rhos, t.ism, b.rs);
  b.ism = fma(b.rhos, t.rs, b.ism);
  smb = fma(b.ism, (-(fmul(t.ism, t.ism))), smb);
  Sb = fadd(Sb, smb);
  SMb = fsub(SMb, smb);
}

// UCT: the solver's own edge-field weights (riemann_hlld<T, true>); Ib[6]
// holds the cotangents of (a^L, a^R, d^L, u_L, u_R, d^R).  They replace the
// outer-speed weights in every branch, so those pass no cotangent.
template <bool UCT = false>
__device__ __forceinline__ void riemann_hlld_vjp(const W7& L, const W7& R, double bn, double gamma, double igm1,
                                                 const double Fb[7], const double* Ib, W7b& Lb, W7b& Rb,
                                                 double& bnb) {
  const double Ih[5] = {UCT ? 0.0 : Ib[0], UCT ? 0.0 : Ib[1], UCT ? 0.0 : Ib[2], Ib[3], Ib[4]};
  const double bn2 = fmul(bn, bn);
  SideNumT<double> ll, lr;
  side_num(L, bn2, gamma, ll);
  side_num(R, bn2, gamma, lr);
  const bool c_right = cmax_right(ll.n, L.rho, lr.n, R.rho);
  const double cmax = fast_speed_max(ll.n, L.rho, lr.n, R.rho);
  const double SL = fsub(imin(L.u, R.u), cmax), SR = fadd(imax(L.u, R.u), cmax);
  double SLb = 0.0, SRb = 0.0, bn2b = 0.0;
  double B2bL = 0.0, pTbL = 0.0, B2bR = 0.0, pTbR = 0.0;
  if (gt0(SL) || lt0(SR)) {  // supersonic: the upwind physical flux
    const bool up_left = gt0(SL);
    const double Ub[7] = {0, 0, 0, 0, 0, 0, 0};
    if (up_left) side_full_vjp(L, bn, igm1, ll.B2, ll.pT, Ub, Fb, 0.0, Lb, bnb, bn2b, B2bL, pTbL);
    else side_full_vjp(R, bn, igm1, lr.B2, lr.pT, Ub, Fb, 0.0, Rb, bnb, bn2b, B2bR, pTbR);
  } else {
    // ---- primal, as in riemann_hlld ----
    const double sdL = fsub(SL, L.u), sdR = fsub(SR, R.u);
    const double rsL = fmul(sdL, L.rho), rsR = fmul(sdR, R.rho);
    const double iden = rcp(fsub(rsR, rsL));
    const double NM = fadd((fsub(fma(rsR, R.u, fmul(-rsL, L.u)), lr.pT)), ll.pT);
    const double SM = fmul(NM, iden);
    const double a1 = fmul((fmul(L.rho, rsR)), sdL);
    const double Np = fma(a1, fsub(R.u, L.u), fma(rsR, ll.pT, fmul(-rsL, lr.pT)));
    const double pTs = fmul(Np, iden);
    StarT tL, tR;
    star_side(L, SL, SM, bn, bn2, tL);
    star_side(R, SR, SM, bn, bn2, tR);
    const bool left = ge0(SM);
    const W7& A = left ? L : R;
    const StarT& ta = left ? tL : tR;
    const double pTa = left ? ll.pT : lr.pT, B2a = left ? ll.B2 : lr.B2;
    const double S = left ? SL : SR;
    double Ua[7], Fa[7], vBa;
    side_full(A, bn, bn2, igm1, left ? ll : lr, Ua, Fa, vBa);
    const double vBs = fma(SM, bn, fma(ta.vs, ta.b1s, fmul(ta.ws, ta.b2s)));
    const double NE = fadd(fma(ta.sd, Ua[6], fmul(-pTa, A.u)), fma(pTs, SM, fmul(bn, (fsub(vBa, vBs)))));
    const double Es = fmul(NE, ta.ism);
    const double Us[7] = {ta.rhos, fmul(ta.rhos, SM), fmul(ta.rhos, ta.vs), fmul(ta.rhos, ta.ws), ta.b1s, ta.b2s, Es};
    StarB bL, bR;
    StarB& ba = left ? bL : bR;
    double SMb = 0.0, pTsb = 0.0, Sb = 0.0, Esb = 0.0, vBsb = 0.0;
    double Usb[7] = {0, 0, 0, 0, 0, 0, 0};
    // star ratios of the UCT-HLLD weights (1 on a degenerate side)
    const double eL = tL.degen ? 1.0 : tL.cb, eR = tR.degen ? 1.0 : tR.cb;
    bool dstar = false;  // the double-star weights replaced the single-star ones
    // ---- rotational waves ----
    if (!lt_pos(kmul(RK_HALF, bn2), fmul(kHlldBnEps, pTs))) {
      const double iqL = frsqrt(tL.rhos), iqR = frsqrt(tR.rhos);
      const double sqL = fmul(tL.rhos, iqL), sqR = fmul(tR.rhos, iqR);
      const double abn = dabs(bn);
      const double Ss = left ? fma(-abn, iqL, SM) : fma(abn, iqR, SM);
      const bool beyond = left ? lt0(Ss) : ge0(Ss);
      if (beyond) {
        const double sg = gt0(bn) ? 1.0 : -1.0;
        const double isum = rcp(fadd(sqL, sqR));
        const double Nv = fma(sqL, tL.vs, fma(sqR, tR.vs, times_sign(fsub(tR.b1s, tL.b1s), bn)));
        const double Nw = fma(sqL, tL.ws, fma(sqR, tR.ws, times_sign(fsub(tR.b2s, tL.b2s), bn)));
        const double vss = fmul(Nv, isum), wss = fmul(Nw, isum);
        const double sq2 = fmul(sqL, sqR);
        const double N1 = fma(sqL, tR.b1s, fma(sqR, tL.b1s, times_sign(fmul(sq2, (fsub(tR.vs, tL.vs))), bn)));
        const double N2 = fma(sqL, tR.b2s, fma(sqR, tL.b2s, times_sign(fmul(sq2, (fsub(tR.ws, tL.ws))), bn)));
        const double b1ss = fmul(N1, isum), b2ss = fmul(N2, isum);
        const double vBss = fma(SM, bn, fma(vss, b1ss, fmul(wss, b2ss)));
        const double sqa = neg_if(left ? sqL : sqR, left);  // -sqrt(rho*_L) on the left
        const double dvB = fsub(vBs, vBss);
        const double Ess = fma(sqa, times_sign(dvB, bn), Es);
        // F2..F6 += S*_a (U** - U*)
        double Ssb = fma(Fb[2], fma(ta.rhos, vss, -Us[2]),
                         fma(Fb[3], fma(ta.rhos, wss, -Us[3]),
                             fma(Fb[4], fsub(b1ss, ta.b1s), fma(Fb[5], fsub(b2ss, ta.b2s), fmul(Fb[6], fsub(Ess, Es))))));
        ba.rhos = fma(Ss, fma(Fb[2], vss, fmul(Fb[3], wss)), ba.rhos);
        double vssb = fmul(fmul(Fb[2], Ss), ta.rhos), wssb = fmul(fmul(Fb[3], Ss), ta.rhos);
        Usb[2] = fma(-Fb[2], Ss, Usb[2]);
        Usb[3] = fma(-Fb[3], Ss, Usb[3]);
        double b1ssb = fmul(Fb[4], Ss), b2ssb = fmul(Fb[5], Ss);
        ba.b1s = fma(-Fb[4], Ss, ba.b1s);
        ba.b2s = fma(-Fb[5], Ss, ba.b2s);
        const double Essb = fmul(Fb[6], Ss);
        Esb = fma(-Fb[6], Ss, Esb);
        // Ess = Es + sqa sg (vBs - vBss)
        Esb = fadd(Esb, Essb);
        const double sqab = fmul(fmul(Essb, sg), dvB);
        vBsb = fma((fmul(Essb, sqa)), sg, vBsb);
        const double vBssb = fmul(fmul(-Essb, sqa), sg);
        double sqLb = left ? neg_if(sqab, true) : 0.0, sqRb = left ? 0.0 : sqab;
        // vBss = SM bn + vss b1ss + wss b2ss
        SMb = fma(vBssb, bn, SMb);
        bnb = fma(vBssb, SM, bnb);
        vssb = fma(vBssb, b1ss, vssb);
        b1ssb = fma(vBssb, vss, b1ssb);
        wssb = fma(vBssb, b2ss, wssb);
        b2ssb = fma(vBssb, wss, b2ssb);
        // b1ss, b2ss
        double isumb = fma(b1ssb, N1, fma(b2ssb, N2, fma(vssb, Nv, fmul(wssb, Nw))));
        const double N1b = fmul(b1ssb, isum), N2b = fmul(b2ssb, isum), Nvb = fmul(vssb, isum), Nwb = fmul(wssb, isum);
        sqLb = fma(N1b, tR.b1s, fma(N2b, tR.b2s, fma(Nvb, tL.vs, fma(Nwb, tL.ws, sqLb))));
        sqRb = fma(N1b, tL.b1s, fma(N2b, tL.b2s, fma(Nvb, tR.vs, fma(Nwb, tR.ws, sqRb))));
        bR.b1s = fma(N1b, sqL, fma(Nvb, sg, bR.b1s));
        bL.b1s = fma(N1b, sqR, fma(-Nvb, sg, bL.b1s));
        bR.b2s = fma(N2b, sqL, fma(Nwb, sg, bR.b2s));
        bL.b2s = fma(N2b, sqR, fma(-Nwb, sg, bL.b2s));
        const double t1 = fmul(N1b, sg), t2 = fmul(N2b, sg);
        const double sq2b = fma(t1, (fsub(tR.vs, tL.vs)), fmul(t2, (fsub(tR.ws, tL.ws))));
        bR.vs = fma(t1, sq2, fma(Nvb, sqR, bR.vs));
        bL.vs = fma(-t1, sq2, fma(Nvb, sqL, bL.vs));
        bR.ws = fma(t2, sq2, fma(Nwb, sqR, bR.ws));
        bL.ws = fma(-t2, sq2, fma(Nwb, sqL, bL.ws));
        sqLb = fma(sq2b, sqR, sqLb);
        sqRb = fma(sq2b, sqL, sqRb);
        // isum = 1/(sqL + sqR)
        const double db = fmul(isumb, (-(fmul(isum, isum))));
        sqLb = fadd(sqLb, db);
        sqRb = fadd(sqRb, db);
        // Ss
        SMb = fadd(SMb, Ssb);
        double iqLb = 0.0, iqRb = 0.0, abnb;
        if (left) {
          abnb = fmul(-Ssb, iqL);
          iqLb = fma(-Ssb, abn, iqLb);
        } else {
          abnb = fmul(Ssb, iqR);
          iqRb = fma(Ssb, abn, iqRb);
        }
        bnb = fadd(bnb, neg_if(abnb, lt0(bn)));
        if (UCT) {  // a^L = S*_R w, a^R = -S*_L w, w = 1/(S*_R - S*_L); d^L = a^L kL, d^R = a^R kR
          dstar = true;
          const double SsL = fma(-abn, iqL, SM), SsR = fma(abn, iqR, SM);
          const double iw = rcp(fsub(SsR, SsL));
          const double aL = fmul(SsR, iw), aR = fmul(-SsL, iw);
          const double kL = fma(fsub(SL, SsL), eL, -SL), kR = fma(fsub(SsR, SR), eR, SR);
          const double aLb = fma(Ib[2], kL, Ib[0]), aRb = fma(Ib[5], kR, Ib[1]);
          const double kLb = fmul(Ib[2], aL), kRb = fmul(Ib[5], aR);
          // kL = (S_L - S*_L) e_L - S_L, kR = (S*_R - S_R) e_R + S_R
          SLb = fma(kLb, fsub(eL, 1.0), SLb);
          SRb = fma(kRb, fsub(1.0, eR), SRb);
          double SsLb = fmul(-kLb, eL), SsRb = fmul(kRb, eR);
          if (!tL.degen) bL.cb = fma(kLb, fsub(SL, SsL), bL.cb);
          if (!tR.degen) bR.cb = fma(kRb, fsub(SsR, SR), bR.cb);
          SsRb = fma(aLb, iw, SsRb);
          SsLb = fma(-aRb, iw, SsLb);
          const double iwb = fma(aLb, SsR, fmul(-aRb, SsL));
          const double dwb = fmul(iwb, -(fmul(iw, iw)));
          SsRb = fadd(SsRb, dwb);
          SsLb = fsub(SsLb, dwb);
          // S*_L = S_M - |b_n| iqL, S*_R = S_M + |b_n| iqR
          SMb = fadd(SMb, fadd(SsLb, SsRb));
          iqLb = fma(-SsLb, abn, iqLb);
          iqRb = fma(SsRb, abn, iqRb);
          bnb = fadd(bnb, neg_if(fma(SsRb, iqR, fmul(-SsLb, iqL)), lt0(bn)));
        }
        // sq = rhos iq, iq = rhos^(-1/2)
        bL.rhos = fma(sqLb, iqL, bL.rhos);
        iqLb = fma(sqLb, tL.rhos, iqLb);
        bR.rhos = fma(sqRb, iqR, bR.rhos);
        iqRb = fma(sqRb, tR.rhos, iqRb);
        bL.rhos = fma(iqLb, (fmul(kmul(RK_MHALF, (fmul(iqL, iqL))), iqL)), bL.rhos);
        bR.rhos = fma(iqRb, (fmul(kmul(RK_MHALF, (fmul(iqR, iqR))), iqR)), bR.rhos);
      }
    }
    if (UCT && !dstar) {  // single-star weights: d^L = S_L (e_L - 1) left of the contact, d^R = S_R (1 - e_R) right
      if (left) {
        SLb = fma(Ib[2], fsub(eL, 1.0), SLb);
        if (!tL.degen) bL.cb = fma(Ib[2], SL, bL.cb);
      } else {
        SRb = fma(Ib[5], fsub(1.0, eR), SRb);
        if (!tR.degen) bR.cb = fma(-Ib[5], SR, bR.cb);
      }
    }
    // ---- F = F_a + S_a (U*_a - U_a) ----
    double Uab[7];
#pragma unroll
    for (int q = 0; q < 7; q++) {
      Sb = fma(Fb[q], (fsub(Us[q], Ua[q])), Sb);
      Usb[q] = fma(Fb[q], S, Usb[q]);
      Uab[q] = fmul(-Fb[q], S);
    }
    // U*_a = (rhos, rhos SM, rhos vs, rhos ws, b1s, b2s, Es)
    ba.rhos = fma(Usb[1], SM, fma(Usb[2], ta.vs, fma(Usb[3], ta.ws, fadd(ba.rhos, Usb[0]))));
    SMb = fma(Usb[1], ta.rhos, SMb);
    ba.vs = fma(Usb[2], ta.rhos, ba.vs);
    ba.ws = fma(Usb[3], ta.rhos, ba.ws);
    ba.b1s = fadd(ba.b1s, Usb[4]);
    ba.b2s = fadd(ba.b2s, Usb[5]);
    Esb = fadd(Esb, Usb[6]);
    // Es = [(sd E_a - pT_a u_a) + (pT* SM + bn (vB_a - vB*))] ism
    const double NEb = fmul(Esb, ta.ism);
    ba.ism = fma(Esb, NE, ba.ism);
    ba.sd = fma(NEb, Ua[6], ba.sd);
    Uab[6] = fma(NEb, ta.sd, Uab[6]);
    double pTab = fmul(-NEb, A.u);
    const double uab = fmul(-NEb, pTa);
    pTsb = fma(NEb, SM, pTsb);
    SMb = fma(NEb, pTs, SMb);
    bnb = fma(NEb, (fsub(vBa, vBs)), bnb);
    const double vBab = fmul(NEb, bn);
    vBsb = fma(-NEb, bn, vBsb);
    // vB* = SM bn + vs b1s + ws b2s
    SMb = fma(vBsb, bn, SMb);
    bnb = fma(vBsb, SM, bnb);
    ba.vs = fma(vBsb, ta.b1s, ba.vs);
    ba.b1s = fma(vBsb, ta.vs, ba.b1s);
    ba.ws = fma(vBsb, ta.b2s, ba.ws);
    ba.b2s = fma(vBsb, ta.ws, ba.b2s);
    // side a: conserved state, flux, v.B
    W7b& Wab = left ? Lb : Rb;
    Wab.u = fadd(Wab.u, uab);
    double B2ab = 0.0;
    side_full_vjp(A, bn, igm1, B2a, pTa, Uab, Fb, vBab, Wab, bnb, bn2b, B2ab, pTab);
    if (left) { B2bL += B2ab; pTbL += pTab; }
    else { B2bR += B2ab; pTbR += pTab; }
    if (left) SLb += Sb;
    else SRb += Sb;
    // star states of both sides
    star_side_vjp<UCT>(L, SM, bn, bn2, tL, bL, Lb, SLb, SMb, bnb, bn2b);
    star_side_vjp<UCT>(R, SM, bn, bn2, tR, bR, Rb, SRb, SMb, bnb, bn2b);
    // pT* = a1 (uR - uL) + (rsR pTL - rsL pTR), times iden; a1 = (rhoL rsR) sdL
    const double Npb = fmul(pTsb, iden);
    double idenb = fmul(pTsb, Np);
    const double a1b = fmul(Npb, (fsub(R.u, L.u)));
    Rb.u = fma(Npb, a1, Rb.u);
    Lb.u = fma(-Npb, a1, Lb.u);
    bR.rs = fma(Npb, ll.pT, bR.rs);
    pTbL = fma(Npb, rsR, pTbL);
    bL.rs = fma(-Npb, lr.pT, bL.rs);
    pTbR = fma(-Npb, rsL, pTbR);
    const double rr = fmul(L.rho, rsR);
    bL.sd = fma(a1b, rr, bL.sd);
    const double rrb = fmul(a1b, sdL);
    Lb.rho = fma(rrb, rsR, Lb.rho);
    bR.rs = fma(rrb, L.rho, bR.rs);
    // SM = [(rsR uR - rsL uL) - pTR + pTL] iden
    const double NMb = fmul(SMb, iden);
    idenb = fma(SMb, NM, idenb);
    bR.rs = fma(NMb, R.u, bR.rs);
    Rb.u = fma(NMb, rsR, Rb.u);
    bL.rs = fma(-NMb, L.u, bL.rs);
    Lb.u = fma(-NMb, rsL, Lb.u);
    pTbR = fsub(pTbR, NMb);
    pTbL = fadd(pTbL, NMb);
    // iden = 1/(rsR - rsL)
    const double d = fmul(idenb, (-(fmul(iden, iden))));
    bR.rs = fadd(bR.rs, d);
    bL.rs = fsub(bL.rs, d);
    // rs = sd rho, sd = S - u
    bL.sd = fma(bL.rs, L.rho, bL.sd);
    Lb.rho = fma(bL.rs, sdL, Lb.rho);
    bR.sd = fma(bR.rs, R.rho, bR.sd);
    Rb.rho = fma(bR.rs, sdR, Rb.rho);
    SLb = fadd(SLb, bL.sd);
    Lb.u = fsub(Lb.u, bL.sd);
    SRb = fadd(SRb, bR.sd);
    Rb.u = fsub(Rb.u, bR.sd);
  }
  double uLb = 0.0, uRb = 0.0, cmaxb = 0.0;
  speeds_vjp(L.u, R.u, cmax, Ih, SLb, SRb, uLb, uRb, cmaxb);
  Lb.u = fadd(Lb.u, uLb);
  Rb.u = fadd(Rb.u, uRb);
  cmax_vjp(L, R, c_right, ll.B2, lr.B2, bn2, gamma, cmaxb, Lb, Rb, B2bL, B2bR, bn2b);
  side_num_vjp(L, B2bL, pTbL, Lb, bn2b);
  side_num_vjp(R, B2bR, pTbR, Rb, bn2b);
  bnb = fma((kmul(RK_2, bn)), bn2b, bnb);
}

}  // namespace mhd
