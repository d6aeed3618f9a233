// ORACLE — test infrastructure only.  C entry points over the templated
// oracle scheme (mhd_oracle.hpp), loaded by the tests through ctypes.
//
// External state layout (no ghosts), x fastest:
//   cell arrays rho, mx, my, mz, E (and the 2D cell Bz): [nz][ny][nx]
//   face Bx: [nz][ny][nx+1], By: [nz][ny+1][nx], Bz (3D): [nz+1][ny][nx]
// On a periodic axis the last face duplicates the first: it is ignored on
// input and written as a copy of the first on output.
#include <cstring>
#include <memory>

#include "glm_oracle.hpp"
#include "mhd_oracle.hpp"

using namespace orc;

namespace {

template <class R> struct Ext {
  // extents of slot q in the external layout
  static void extents(const Sim<R>& s, int q, int e[3]) {
    e[0] = s.n[0]; e[1] = s.n[1]; e[2] = s.n[2];
    for (int d = 0; d < s.ndim; d++)
      if (s.is_face(q, d)) e[d] += 1;
  }
};

template <class R> void load(Sim<R>& s, const double* const* src) {
  for (int q = 0; q < NQ; q++) {
    int e[3];
    Ext<R>::extents(s, q, e);
    const double* p = src[q];
    for (int k = 0; k < e[2]; k++)
      for (int j = 0; j < e[1]; j++)
        for (int i = 0; i < e[0]; i++) s.U0[q](i, j, k) = R(*p++);
  }
}
template <class R> void store(Sim<R>& s, double* const* dst) {
  s.fill_ghosts(s.U0);
  for (int q = 0; q < NQ; q++) {
    int e[3];
    Ext<R>::extents(s, q, e);
    double* p = dst[q];
    for (int k = 0; k < e[2]; k++)
      for (int j = 0; j < e[1]; j++)
        for (int i = 0; i < e[0]; i++) *p++ = value(s.U0[q](i, j, k));
  }
}

}  // namespace

extern "C" {

struct OrcConfig {
  int ndim, nx, ny, nz;
  double x0[3], x1[3];
  double gamma;
  int recon, riemann, rk;
  double cfl;
  int bc[6];
  double p_floor;
  int emf;
};

static Config to_cfg(const OrcConfig* c) {
  Config o{};
  o.ndim = c->ndim; o.nx = c->nx; o.ny = c->ny; o.nz = c->nz;
  for (int d = 0; d < 3; d++) { o.x0[d] = c->x0[d]; o.x1[d] = c->x1[d]; }
  o.gamma = c->gamma; o.recon = c->recon; o.riemann = c->riemann; o.rk = c->rk; o.cfl = c->cfl;
  for (int s = 0; s < 6; s++) o.bc[s] = c->bc[s];
  o.p_floor = c->p_floor;
  o.emf = c->emf;
  return o;
}

void* orc_create(const OrcConfig* c) {
  try {
    return new Sim<double>(to_cfg(c));
  } catch (...) {
    return nullptr;
  }
}
void orc_destroy(void* h) { delete static_cast<Sim<double>*>(h); }

int orc_set_state(void* h, const double* const* arrays) {
  load(*static_cast<Sim<double>*>(h), arrays);
  return 0;
}
int orc_get_state(void* h, double* const* arrays) {
  store(*static_cast<Sim<double>*>(h), arrays);
  return 0;
}
double orc_cfl_dt(void* h) { return static_cast<Sim<double>*>(h)->cfl_dt(); }
int orc_step(void* h, double dt) {
  auto* s = static_cast<Sim<double>*>(h);
  s->step(dt);
  return s->bad ? -4 : 0;
}
double orc_time(void* h) { return static_cast<Sim<double>*>(h)->time; }

// ---- the scheme with GLM divergence cleaning (glm_oracle.hpp) ----
// State: 9 cell arrays [nz][ny][nx]: rho, mx, my, mz, E, Bx, By, Bz, psi.
void* orc_glm_create(const OrcConfig* c, double alpha) {
  try {
    return new GlmSim<double>(to_cfg(c), alpha);
  } catch (...) {
    return nullptr;
  }
}
void orc_glm_destroy(void* h) { delete static_cast<GlmSim<double>*>(h); }
int orc_glm_set_state(void* h, const double* const* arrays) {
  auto* s = static_cast<GlmSim<double>*>(h);
  for (int q = 0; q < NG; q++) {
    const double* p = arrays[q];
    for (int k = 0; k < s->n[2]; k++)
      for (int j = 0; j < s->n[1]; j++)
        for (int i = 0; i < s->n[0]; i++) s->U0[q](i, j, k) = *p++;
  }
  return 0;
}
int orc_glm_get_state(void* h, double* const* arrays) {
  auto* s = static_cast<GlmSim<double>*>(h);
  for (int q = 0; q < NG; q++) {
    double* p = arrays[q];
    for (int k = 0; k < s->n[2]; k++)
      for (int j = 0; j < s->n[1]; j++)
        for (int i = 0; i < s->n[0]; i++) *p++ = s->U0[q](i, j, k);
  }
  return 0;
}
double orc_glm_cfl_dt(void* h) { return static_cast<GlmSim<double>*>(h)->cfl_dt(); }
int orc_glm_step(void* h, double dt) {
  auto* s = static_cast<GlmSim<double>*>(h);
  s->step(dt);
  return s->bad ? -4 : 0;
}
double orc_glm_ch(void* h) { return static_cast<GlmSim<double>*>(h)->ch; }
// Counted-scalar run of the GLM scheme: one CFL evaluation and nsteps steps
// of size dt from the 9 given cell arrays; out[PH_N * OP_N] as orc_count_flops.
int orc_glm_count_flops(const OrcConfig* c, double alpha, const double* const* arrays, int nsteps, double dt,
                        unsigned long long* out) {
  GlmSim<Counted> s(to_cfg(c), alpha);
  for (int q = 0; q < NG; q++) {
    const double* p = arrays[q];
    for (int k = 0; k < s.n[2]; k++)
      for (int j = 0; j < s.n[1]; j++)
        for (int i = 0; i < s.n[0]; i++) s.U0[q](i, j, k) = Counted(*p++);
  }
  g_flops.reset();
  s.cfl_dt();
  for (int t = 0; t < nsteps; t++) s.step(Counted(dt));
  for (int ph = 0; ph < PH_N; ph++)
    for (int op = 0; op < OP_N; op++) out[ph * OP_N + op] = g_flops.n[ph][op];
  return 0;
}
long long orc_glm_fallbacks(void* h) { return static_cast<GlmSim<double>*>(h)->fallbacks; }
long long orc_fallbacks(void* h) { return static_cast<Sim<double>*>(h)->fallbacks; }
long long orc_floors(void* h) { return static_cast<Sim<double>*>(h)->floors; }
int orc_status(void* h, long long* bad_cell) {
  auto* s = static_cast<Sim<double>*>(h);
  if (bad_cell) *bad_cell = s->bad_cell;
  return s->bad ? -4 : 0;
}

// Edge field E_c of the last stage computed, over a-face [0,n_a] x b-face [0,n_b]
// x c-cell [0,n_c-1], written x fastest.
int orc_get_emf(void* h, int cc, double* out) {
  auto* s = static_cast<Sim<double>*>(h);
  int a = (cc + 1) % 3, b = (cc + 2) % 3;
  int ext[3];
  ext[a] = s->n[a] + 1; ext[b] = s->n[b] + 1; ext[cc] = s->n[cc];
  if (s->ndim == 2) { if (cc != 2) return -1; ext[2] = 1; }
  for (int k = 0; k < ext[2]; k++)
    for (int j = 0; j < ext[1]; j++)
      for (int i = 0; i < ext[0]; i++) *out++ = s->E[cc](i, j, k);
  return 0;
}
// Stage increment L(U^n) for the current state with step dt (no state change).
int orc_stage_increment(void* h, double dt, double* const* arrays) {
  auto* s = static_cast<Sim<double>*>(h);
  s->stage_increment(s->U0, dt);
  for (int q = 0; q < NQ; q++) {
    int e[3];
    Ext<double>::extents(*s, q, e);
    double* p = arrays[q];
    for (int k = 0; k < e[2]; k++)
      for (int j = 0; j < e[1]; j++)
        for (int i = 0; i < e[0]; i++) {
          bool upd = true;
          for (int d = 0; d < s->ndim; d++) {
            int idx = d == 0 ? i : (d == 1 ? j : k);
            if (idx >= s->n[d] && !(s->is_face(q, d) && !s->periodic[d])) upd = false;
          }
          *p++ = upd ? s->Lq[q](i, j, k) : 0.0;
        }
  }
  return s->bad ? -4 : 0;
}

// CFL dt of a state given in the external layout, without building the padded
// grid: the same cell-centred field, primitive recovery and per-cell rate as
// Sim::cfl_dt, for grids too large for the full oracle.
double orc_cfl_dt_state(const OrcConfig* cfg, const double* const* a) {
  Config c = to_cfg(cfg);
  int nd = c.ndim;
  int n[3] = {c.nx, c.ny, nd == 3 ? c.nz : 1};
  double idx[3];
  for (int d = 0; d < 3; d++) {
    double x0 = d < nd ? c.x0[d] : 0.0, x1 = d < nd ? c.x1[d] : 1.0;
    double dx = (x1 - x0) / n[d];
    idx[d] = 1.0 / dx;
  }
  long long sx1 = n[0] + 1, sy1 = n[1] + 1;
  double lmax = 0.0;
  for (int k = 0; k < n[2]; k++)
    for (int j = 0; j < n[1]; j++)
      for (int i = 0; i < n[0]; i++) {
        long long cc = ((long long)k * n[1] + j) * n[0] + i;
        double bx0 = a[5][((long long)k * n[1] + j) * sx1 + i], bx1 = a[5][((long long)k * n[1] + j) * sx1 + i + 1];
        double by0 = a[6][((long long)k * sy1 + j) * n[0] + i], by1 = a[6][((long long)k * sy1 + j + 1) * n[0] + i];
        double bx = 0.5 * (bx0 + bx1);
        double by = 0.5 * (by0 + by1);
        double bz;
        if (nd == 3) {
          double bz0 = a[7][cc], bz1 = a[7][cc + (long long)n[0] * n[1]];
          bz = 0.5 * (bz0 + bz1);
        } else {
          bz = a[7][cc];
        }
        double V[NP];
        cons_to_prim<double>(a[0][cc], a[1][cc], a[2][cc], a[3][cc], a[4][cc], bx, by, bz, c.gamma, V);
        if (V[P_PR] < c.p_floor) V[P_PR] = c.p_floor;
        double lam = cfl_rate<double>(V, idx, nd, c.gamma);
        if (lmax < lam) lmax = lam;
      }
  return c.cfl / lmax;
}

// ---- pointwise pieces ----
// solver: RS_HLL, RS_HLLD, or 2 = HLLD with the UCT-HLLD ingredients; ing has NI entries.
void orc_riemann(int solver, const double* wl, const double* wr, double bn, double gamma, double* F, double* ing) {
  if (solver == RS_HLLD || solver == 2) riemann_hlld<double>(wl, wr, bn, gamma, F, ing, solver == 2);
  else riemann_hll<double>(wl, wr, bn, gamma, F, ing);
}
void orc_side_flux(const double* w, double bn, double gamma, double* F, double* U) {
  SideState<double> s = side_state<double>(w, bn, gamma);
  for (int q = 0; q < NW; q++) { F[q] = s.F[q]; U[q] = s.U[q]; }
}
void orc_recon(int method, const double* s5, double* plus, double* minus) {
  if (method == RECON_PLM) recon_plm<double>(s5, *plus, *minus);
  else if (method == RECON_WENOZ) recon_wenoz<double>(s5, *plus, *minus);
  else recon_ppm<double>(s5, *plus, *minus);
}
void orc_c2p(const double* u8, double gamma, double* V) {
  cons_to_prim<double>(u8[0], u8[1], u8[2], u8[3], u8[4], u8[5], u8[6], u8[7], gamma, V);
}
double orc_fast_speed(double rho, double p, double B2, double bn, double gamma) {
  return fast_speed<double>(rho, p, B2, bn, gamma);
}

// ---- algorithmic flop count: nsteps steps of size dt with the Counted scalar ----
// out[ph * OP_N + op] for phases PH_* and kinds OP_*; also counts the CFL once.
int orc_count_flops(const OrcConfig* c, const double* const* arrays, int nsteps, double dt,
                    unsigned long long* out) {
  Sim<Counted> s(to_cfg(c));
  load(s, arrays);
  g_flops.reset();
  s.cfl_dt();
  for (int t = 0; t < nsteps; t++) s.step(Counted(dt));
  for (int ph = 0; ph < PH_N; ph++)
    for (int op = 0; op < OP_N; op++) out[ph * OP_N + op] = g_flops.n[ph][op];
  return 0;
}

// Flops of the face-independent part of one WENO-Z face value (wenoz_shared:
// the three indicators, tau5, the ratios and 1 + ratio^2) on the stencil a[5],
// counted with the Counted scalar: the part a per-cell implementation forms
// once for both faces of a cell.
unsigned long long orc_count_wenoz_shared(const double* a) {
  g_flops.reset();
  g_flops.phase = PH_RECON;
  Counted h0, h1, h2;
  wenoz_shared<Counted>(Counted(a[0]), Counted(a[1]), Counted(a[2]), Counted(a[3]), Counted(a[4]), h0, h1, h2);
  unsigned long long n = 0;
  for (int op = 0; op < OP_N; op++) n += g_flops.n[PH_RECON][op];
  g_flops.reset();
  return n;
}

// Reverse-mode work of nsteps steps of size dt from the given state, every
// state element (cells and faces) a tape variable: out_links[PH_N] flops of
// the backward sweep and out_pflops[PH_N] partial-derivative flops per phase.
int orc_count_tape(const OrcConfig* c, const double* const* arrays, int nsteps, double dt,
                   unsigned long long* out_links, unsigned long long* out_pflops) {
  Sim<double> d(to_cfg(c));
  load(d, arrays);
  Sim<Tape> s(to_cfg(c));
  g_tape.clear();
  for (int q = 0; q < NQ; q++) {
    auto& src = d.U0[q];
    auto& dst = s.U0[q];
    for (size_t i = 0; i < src.a.size(); i++) dst.a[i] = Tape::variable(src.a[i]);
  }
  g_tape_count.reset();
  for (int t = 0; t < nsteps; t++) s.step(Tape(dt));
  for (int ph = 0; ph < PH_N; ph++) {
    out_links[ph] = g_tape_count.links[ph];
    out_pflops[ph] = g_tape_count.partial_flops[ph];
  }
  g_tape.clear();
  g_tape.shrink_to_fit();
  return s.bad ? -4 : 0;
}

// ---- final-state functional and its derivatives w.r.t. the initial rho, v ----
// prim[0..4] = rho, vx, vy, vz, p (cell arrays); B[0..2] as in the state layout;
// dts[nsteps] the frozen step sizes; which = 0 magnetic energy, 1 misfit to
// target[0..4 (2D: 5)] (cell arrays of rho, mx, my, mz, E (, Bz)).
static size_t ncells(const Config& c) { return (size_t)c.nx * c.ny * (c.ndim == 3 ? c.nz : 1); }

// The initial conserved state set_from_prims builds from prim[0..4] = rho, vx,
// vy, vz, p and the fields B[0..2], written to out[0..7] in the state layout.
int orc_state_from_prims(const OrcConfig* oc, const double* const* prim, const double* const* B,
                         double* const* out) {
  Sim<double> s(to_cfg(oc));
  set_from_prims(s, prim[0], prim[1], prim[2], prim[3], prim[4], B);
  store(s, out);
  return 0;
}

int orc_functional_prim(const OrcConfig* oc, const double* const* prim, const double* const* B, const double* dts,
                        int nsteps, int which, const double* const* target, double* J, unsigned long long* sig) {
  Config c = to_cfg(oc);
  int bad = 0;
  g_branch_sig = 1469598103934665603ULL;
  *J = run_functional<double>(c, prim[0], prim[1], prim[2], prim[3], prim[4], B, dts, nsteps, which, target, &bad);
  if (sig) *sig = g_branch_sig;
  return bad ? -4 : 0;
}

int orc_jvp_prim(const OrcConfig* oc, const double* const* prim, const double* const* B, const double* dts,
                 int nsteps, int which, const double* const* target, const double* const* tangent, double* J,
                 double* dJ) {
  Config c = to_cfg(oc);
  size_t N = ncells(c);
  std::vector<Dual> in[4];
  for (int q = 0; q < 4; q++) {
    in[q].resize(N);
    for (size_t i = 0; i < N; i++) in[q][i] = Dual(prim[q][i], tangent[q][i]);
  }
  int bad = 0;
  Dual r = run_functional<Dual>(c, in[0].data(), in[1].data(), in[2].data(), in[3].data(), prim[4], B, dts, nsteps,
                                which, target, &bad);
  *J = r.v;
  *dJ = r.d;
  return bad ? -4 : 0;
}

int orc_grad_prim(const OrcConfig* oc, const double* const* prim, const double* const* B, const double* dts,
                  int nsteps, int which, const double* const* target, double* J, double* const* grad) {
  Config c = to_cfg(oc);
  size_t N = ncells(c);
  g_tape.clear();
  std::vector<Tape> in[4];
  for (int q = 0; q < 4; q++) {
    in[q].resize(N);
    for (size_t i = 0; i < N; i++) in[q][i] = Tape::variable(prim[q][i]);
  }
  int bad = 0;
  Tape r = run_functional<Tape>(c, in[0].data(), in[1].data(), in[2].data(), in[3].data(), prim[4], B, dts, nsteps,
                                which, target, &bad);
  *J = r.v;
  std::vector<double> adj = tape_backprop(r);
  for (int q = 0; q < 4; q++)
    for (size_t i = 0; i < N; i++) grad[q][i] = in[q][i].i >= 0 ? adj[in[q][i].i] : 0.0;
  g_tape.clear();
  g_tape.shrink_to_fit();
  return bad ? -4 : 0;
}

// The same functional's reverse-mode gradient with respect to every element
// of the initial state in the layout of orc_state_from_prims (cells rho, mx,
// my, mz, E and the face fields): state[8] in, grad[8] out.  On a periodic
// axis the face at n is the ghost copy of face 0, so its entry is 0.
int orc_grad_conserved(const OrcConfig* oc, const double* const* state, const double* dts, int nsteps, int which,
                       const double* const* target, double* J, double* const* grad) {
  Config c = to_cfg(oc);
  g_tape.clear();
  Sim<Tape> s(c);
  std::vector<std::vector<int>> ids(NQ);
  for (int q = 0; q < NQ; q++) {
    int e[3];
    Ext<Tape>::extents(s, q, e);
    const double* p = state[q];
    for (int k = 0; k < e[2]; k++)
      for (int j = 0; j < e[1]; j++)
        for (int i = 0; i < e[0]; i++) {
          Tape v = Tape::variable(*p++);
          ids[q].push_back(v.i);
          s.U0[q](i, j, k) = v;
        }
  }
  for (int t = 0; t < nsteps; t++) s.step(Tape(dts[t]));
  Tape r = functional(s, which, target);
  *J = r.v;
  std::vector<double> adj = tape_backprop(r);
  for (int q = 0; q < NQ; q++)
    for (size_t m = 0; m < ids[q].size(); m++) grad[q][m] = adj[ids[q][m]];
  g_tape.clear();
  g_tape.shrink_to_fit();
  return s.bad ? -4 : 0;
}

// One first RK stage, U* = U + L(U) with step dt: J = <w, U*> over the
// evolved cells and faces (w in the state layout, its other entries unused),
// and its reverse-mode gradient with respect to every element of U.
int orc_stage_vjp(const OrcConfig* oc, const double* const* state, double dt, const double* const* w, double* J,
                  double* const* grad) {
  Config c = to_cfg(oc);
  g_tape.clear();
  Sim<Tape> s(c);
  std::vector<std::vector<int>> ids(NQ);
  int ext[NQ][3];
  for (int q = 0; q < NQ; q++) {
    Ext<Tape>::extents(s, q, ext[q]);
    const double* p = state[q];
    for (int k = 0; k < ext[q][2]; k++)
      for (int j = 0; j < ext[q][1]; j++)
        for (int i = 0; i < ext[q][0]; i++) {
          Tape v = Tape::variable(*p++);
          ids[q].push_back(v.i);
          s.U0[q](i, j, k) = v;
        }
  }
  s.stage_increment(s.U0, Tape(dt));
  Tape r(0.0);
  s.each_updated([&](int q, int i, int j, int k) {
    const double wq = w[q][((size_t)k * ext[q][1] + j) * ext[q][0] + i];
    r = r + Tape(wq) * (s.U0[q](i, j, k) + s.Lq[q](i, j, k));
  });
  *J = r.v;
  std::vector<double> adj = tape_backprop(r);
  for (int q = 0; q < NQ; q++)
    for (size_t m = 0; m < ids[q].size(); m++) grad[q][m] = adj[ids[q][m]];
  g_tape.clear();
  g_tape.shrink_to_fit();
  return s.bad ? -4 : 0;
}

}  // extern "C"
