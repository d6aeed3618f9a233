// Forward-mode multi-tangent numbers for the adjoint: a value and KT tangent
// components.  Instantiating the templated Riemann solvers of mhd_math.cuh
// with D3 gives their exact derivative along KT input directions at once --
// the same operations in the same order as the double path, each branch
// (limiters, wave fan, min/max) taken as the value dictates.
#pragma once
#include "mhd_math.cuh"

namespace mhd {

// The overloads below would hide the double versions for code of this
// namespace that follows them.
using ::fabs;
using ::fma;

constexpr int KT = 3;

struct D3 {
  double v;
  double d[KT];
  __device__ __forceinline__ D3() {}
  __device__ __forceinline__ explicit D3(double x) : v(x) {
#pragma unroll
    for (int k = 0; k < KT; k++) d[k] = 0.0;
  }
};

__device__ __forceinline__ D3 operator+(const D3& a, const D3& b) {
  D3 r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ D3 operator-(const D3& a, const D3& b) {
  D3 r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ D3 operator-(const D3& a) {
  D3 r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = -a.d[k];
  return r;
}
__device__ __forceinline__ D3 operator*(const D3& a, const D3& b) {
  D3 r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = fma(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
__device__ __forceinline__ D3 operator*(double a, const D3& b) {
  D3 r;
  r.v = a * b.v;
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = a * b.d[k];
  return r;
}
__device__ __forceinline__ D3 operator*(const D3& a, double b) { return b * a; }
__device__ __forceinline__ D3 mul_rn(const D3& a, const D3& b) {
  D3 r;
  r.v = __dmul_rn(a.v, b.v);
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = fma(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
// The DFMA forms of the double arithmetic (fmul, fadd, fsub, kmul of
// mhd_math.cuh) are the plain operations on these numbers.
__device__ __forceinline__ D3 fmul(const D3& a, const D3& b) { return a * b; }
__device__ __forceinline__ D3 fadd(const D3& a, const D3& b) { return a + b; }
__device__ __forceinline__ D3 fsub(const D3& a, const D3& b) { return a - b; }
__device__ __forceinline__ D3 kmul(int i, const D3& x) { return rk(i) * x; }
__device__ __forceinline__ D3 fma(const D3& a, const D3& b, const D3& c) {
  D3 r;
  r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = fma(a.d[k], b.v, fma(a.v, b.d[k], c.d[k]));
  return r;
}
__device__ __forceinline__ D3 fma(double a, const D3& b, const D3& c) {
  D3 r;
  r.v = fma(a, b.v, c.v);
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = fma(a, b.d[k], c.d[k]);
  return r;
}
__device__ __forceinline__ D3 rcp(const D3& x) {
  D3 r;
  double q = rcp(x.v);
  r.v = q;
  double dq = -(q * q);
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = dq * x.d[k];
  return r;
}
__device__ __forceinline__ D3 fsqrt(const D3& x) {
  D3 r;
  double s = fsqrt(x.v);
  r.v = s;
  double h = 0.5 * rcp(s);
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = h * x.d[k];
  return r;
}
__device__ __forceinline__ D3 fsqrt0(const D3& x) { return bits(x.v) >= kMinNormalBits ? fsqrt(x) : D3(0.0); }
__device__ __forceinline__ D3 frsqrt(const D3& x) {
  D3 r;
  double y = frsqrt(x.v);
  r.v = y;
  double c = -0.5 * (y * y) * y;
#pragma unroll
  for (int k = 0; k < KT; k++) r.d[k] = c * x.d[k];
  return r;
}
__device__ __forceinline__ D3 fabs(const D3& x) { return lt0(x.v) ? -x : x; }
__device__ __forceinline__ D3 dabs(const D3& x) { return fabs(x); }
__device__ __forceinline__ bool gt0(const D3& x) { return gt0(x.v); }
__device__ __forceinline__ bool lt0(const D3& x) { return lt0(x.v); }
__device__ __forceinline__ bool ge0(const D3& x) { return ge0(x.v); }
__device__ __forceinline__ D3 imin(const D3& a, const D3& b) { return order_key(b.v) < order_key(a.v) ? b : a; }
__device__ __forceinline__ D3 imax(const D3& a, const D3& b) { return order_key(a.v) < order_key(b.v) ? b : a; }
__device__ __forceinline__ D3 imax_pos(const D3& a, const D3& b) { return bits(a.v) < bits(b.v) ? b : a; }
__device__ __forceinline__ bool lt_pos(const D3& a, const D3& b) { return bits(a.v) < bits(b.v); }
__device__ __forceinline__ D3 times_sign(const D3& x, const D3& s) { return gt0(s.v) ? x : -x; }
__device__ __forceinline__ D3 neg_if(const D3& x, bool c) { return c ? -x : x; }
__device__ __forceinline__ bool lt_abs(const D3& x, const D3& y) { return lt_abs(x.v, y.v); }

}  // namespace mhd
