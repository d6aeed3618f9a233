// ORACLE — test infrastructure only (see oracle/mhd_oracle.hpp header).
//
// Scalar types the oracle scheme is instantiated with:
//   double  : the reference result;
//   Counted : a double that counts every floating-point operation it performs,
//             by operation kind and by phase of the time step, to give the
//             algorithmic flop count per cell-update used for the FP64 roofline.
//
// Counting convention: +, -, *, / and sqrt count one each; comparisons, fabs,
// min/max and sign changes count zero.  An expression a*b + c counts two.
#pragma once
#include <cmath>
#include <cstdint>

namespace orc {

enum Phase { PH_GHOST = 0, PH_C2P, PH_RECON, PH_RIEMANN, PH_FLUXDIFF, PH_EMF, PH_CT, PH_RK, PH_CFL, PH_N };
enum OpKind { OP_ADD = 0, OP_MUL, OP_DIV, OP_SQRT, OP_N };

struct FlopCounter {
  int phase = PH_GHOST;
  uint64_t n[PH_N][OP_N] = {};
  void reset() { for (auto& r : n) for (auto& c : r) c = 0; }
};
inline FlopCounter g_flops;

struct Counted {
  double v;
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}
  static void tick(int op) { g_flops.n[g_flops.phase][op]++; }
};
inline Counted operator+(Counted a, Counted b) { Counted::tick(OP_ADD); return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { Counted::tick(OP_ADD); return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { Counted::tick(OP_MUL); return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { Counted::tick(OP_DIV); return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline Counted sqrt(Counted a) { Counted::tick(OP_SQRT); return Counted(std::sqrt(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
inline double value(Counted a) { return a.v; }
inline double value(double a) { return a; }

}  // namespace orc
