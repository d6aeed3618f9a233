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
#include <vector>

namespace orc {

enum Phase { PH_GHOST = 0, PH_C2P, PH_RECON, PH_RIEMANN, PH_FLUXDIFF, PH_EMF, PH_CT, PH_RK, PH_CFL, PH_N };
enum OpKind { OP_ADD = 0, OP_MUL, OP_DIV, OP_SQRT, OP_N };

// Signature of the branch decisions of an evaluation (limiter choices,
// min/max arguments, wave-fan regions, fallbacks): an FNV-1a hash over the
// sequence of decision codes.  Two evaluations with equal signatures took the
// same piecewise-smooth branch of the scheme.
inline uint64_t g_branch_sig = 1469598103934665603ULL;
inline void branch(uint64_t code) { g_branch_sig = (g_branch_sig ^ code) * 1099511628211ULL; }

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

namespace orc {

// ---------------------------------------------------------------------------
// Dual: forward-mode derivative along one direction (value v, tangent d).
// Branches (comparisons, min/max, the limiter and wave-fan choices) follow the
// values, so the tangent is the derivative of the branch taken.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
inline bool operator==(Dual a, Dual b) { return a.v == b.v; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual fabs(Dual a) { return a.v < 0.0 ? Dual(-a.v, -a.d) : a; }
inline double value(Dual a) { return a.v; }

// ---------------------------------------------------------------------------
// Tape: reverse-mode differentiation.  Every operation on tape variables
// appends a node (parents and partial derivatives); backpropagation walks the
// nodes in reverse.  Constants (index -1) record nothing.
// ---------------------------------------------------------------------------
struct TapeNode {
  int a, b;
  double da, db;
};
inline std::vector<TapeNode> g_tape;

// Reverse-mode work recorded on the tape, by phase of the step: the flops of
// the backward sweep over the parent links (adj += w for a partial of +-1: 1;
// adj += d w otherwise: 2) and the flops spent forming partial derivatives
// (1/b and -q/b of a quotient: 2; 1/(2s) of a square root: 1).  Counting
// only; the values are untouched.
struct TapeCounter {
  uint64_t links[PH_N] = {};  // backward-sweep flops
  uint64_t partial_flops[PH_N] = {};
  void reset() {
    for (auto& x : links) x = 0;
    for (auto& x : partial_flops) x = 0;
  }
};
inline TapeCounter g_tape_count;

struct Tape {
  double v;
  int i;
  Tape() : v(0.0), i(-1) {}
  Tape(double x) : v(x), i(-1) {}
  Tape(double x, int idx) : v(x), i(idx) {}
  static Tape variable(double x) {
    g_tape.push_back({-1, -1, 0.0, 0.0});
    return Tape(x, (int)g_tape.size() - 1);
  }
  static Tape node(double x, int a, double da, int b, double db, int partial_flops = 0) {
    if (a < 0 && b < 0) return Tape(x);
    g_tape.push_back({a, b, da, db});
    auto cost = [](int p, double d) -> uint64_t { return p < 0 ? 0 : ((d == 1.0 || d == -1.0) ? 1 : 2); };
    g_tape_count.links[g_flops.phase] += cost(a, da) + cost(b, db);
    g_tape_count.partial_flops[g_flops.phase] += partial_flops;
    return Tape(x, (int)g_tape.size() - 1);
  }
};
inline Tape operator+(Tape a, Tape b) { return Tape::node(a.v + b.v, a.i, 1.0, b.i, 1.0); }
inline Tape operator-(Tape a, Tape b) { return Tape::node(a.v - b.v, a.i, 1.0, b.i, -1.0); }
inline Tape operator*(Tape a, Tape b) { return Tape::node(a.v * b.v, a.i, b.v, b.i, a.v); }
inline Tape operator/(Tape a, Tape b) {
  double q = a.v / b.v;
  return Tape::node(q, a.i, 1.0 / b.v, b.i, -q / b.v, 2);
}
inline Tape operator-(Tape a) { return Tape::node(-a.v, a.i, -1.0, -1, 0.0); }
inline bool operator<(Tape a, Tape b) { return a.v < b.v; }
inline bool operator>(Tape a, Tape b) { return a.v > b.v; }
inline bool operator<=(Tape a, Tape b) { return a.v <= b.v; }
inline bool operator>=(Tape a, Tape b) { return a.v >= b.v; }
inline bool operator==(Tape a, Tape b) { return a.v == b.v; }
inline Tape sqrt(Tape a) {
  double s = std::sqrt(a.v);
  return Tape::node(s, a.i, s > 0.0 ? 0.5 / s : 0.0, -1, 0.0, 1);
}
inline Tape fabs(Tape a) { return a.v < 0.0 ? -a : a; }
inline double value(Tape a) { return a.v; }

// adjoints of every node for d(out)/d(node)
inline std::vector<double> tape_backprop(const Tape& out) {
  std::vector<double> adj(g_tape.size(), 0.0);
  if (out.i < 0) return adj;
  adj[out.i] = 1.0;
  for (long long k = out.i; k >= 0; k--) {
    double w = adj[k];
    if (w == 0.0) continue;
    const TapeNode& n = g_tape[k];
    if (n.a >= 0) adj[n.a] += n.da * w;
    if (n.b >= 0) adj[n.b] += n.db * w;
  }
  return adj;
}

}  // namespace orc
