"""ORACLE — test infrastructure only.

Plain FP64 CPU implementation of the ideal-MHD finite-volume step (paper §2),
loaded through ctypes.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package; the product path never does.

State dictionaries use the external layout of the C library (no ghosts, x
fastest): keys rho, mx, my, mz, E and b0, b1, b2, where b0/b1/b2 are the face
fields Bx [nz][ny][nx+1], By [nz][ny+1][nx], Bz [nz+1][ny][nx] in 3D, and in
2D Bx [ny][nx+1], By [ny+1][nx] and the cell-centred Bz [ny][nx].
"""
import ctypes
import os

import numpy as np

from . import build as _build

RECON = {"plm": 0, "wenoz": 1, "ppm": 2}
RIEMANN = {"hll": 0, "hlld": 1}
BC = {"periodic": 0, "outflow": 1}
EMF = {"uct_hll": 0, "uct_hlld": 1}
KEYS = ("rho", "mx", "my", "mz", "E", "b0", "b1", "b2")
PHASES = ("ghost", "c2p", "recon", "riemann", "fluxdiff", "emf", "ct", "rk", "cfl")
OPS = ("add", "mul", "div", "sqrt")


class OrcConfig(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("x1", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("recon", ctypes.c_int), ("riemann", ctypes.c_int), ("rk", ctypes.c_int),
                ("cfl", ctypes.c_double), ("bc", ctypes.c_int * 6), ("p_floor", ctypes.c_double),
                ("emf", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        so = _build.build()
        L = ctypes.CDLL(so)
        P = ctypes.c_void_p
        D = ctypes.c_double
        DP = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = P
        L.orc_create.argtypes = [ctypes.POINTER(OrcConfig)]
        L.orc_destroy.argtypes = [P]
        L.orc_set_state.argtypes = [P, ctypes.POINTER(DP)]
        L.orc_get_state.argtypes = [P, ctypes.POINTER(DP)]
        L.orc_cfl_dt.restype = D
        L.orc_cfl_dt.argtypes = [P]
        L.orc_step.argtypes = [P, D]
        L.orc_time.restype = D
        L.orc_time.argtypes = [P]
        L.orc_fallbacks.restype = ctypes.c_longlong
        L.orc_fallbacks.argtypes = [P]
        L.orc_floors.restype = ctypes.c_longlong
        L.orc_floors.argtypes = [P]
        L.orc_status.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
        L.orc_get_emf.argtypes = [P, ctypes.c_int, DP]
        L.orc_stage_increment.argtypes = [P, D, ctypes.POINTER(DP)]
        L.orc_riemann.argtypes = [ctypes.c_int, DP, DP, D, D, DP, DP]
        L.orc_side_flux.argtypes = [DP, D, D, DP, DP]
        L.orc_recon.argtypes = [ctypes.c_int, DP, DP, DP]
        L.orc_c2p.argtypes = [DP, D, DP]
        L.orc_fast_speed.restype = D
        L.orc_fast_speed.argtypes = [D, D, D, D, D]
        L.orc_cfl_dt_state.restype = D
        L.orc_cfl_dt_state.argtypes = [ctypes.POINTER(OrcConfig), ctypes.POINTER(DP)]
        PP = ctypes.POINTER(DP)
        L.orc_functional_prim.argtypes = [ctypes.POINTER(OrcConfig), PP, PP, DP, ctypes.c_int, ctypes.c_int, PP, DP,
                                          ctypes.POINTER(ctypes.c_ulonglong)]
        L.orc_jvp_prim.argtypes = [ctypes.POINTER(OrcConfig), PP, PP, DP, ctypes.c_int, ctypes.c_int, PP, PP, DP, DP]
        L.orc_grad_prim.argtypes = [ctypes.POINTER(OrcConfig), PP, PP, DP, ctypes.c_int, ctypes.c_int, PP, DP, PP]
        L.orc_grad_conserved.argtypes = [ctypes.POINTER(OrcConfig), PP, DP, ctypes.c_int, ctypes.c_int, PP, DP, PP]
        L.orc_stage_vjp.argtypes = [ctypes.POINTER(OrcConfig), PP, D, PP, DP, PP]
        L.orc_count_flops.argtypes = [ctypes.POINTER(OrcConfig), ctypes.POINTER(DP), ctypes.c_int, D,
                                      ctypes.POINTER(ctypes.c_ulonglong)]
        L.orc_glm_create.restype = P
        L.orc_glm_create.argtypes = [ctypes.POINTER(OrcConfig), D]
        L.orc_glm_destroy.argtypes = [P]
        L.orc_glm_set_state.argtypes = [P, ctypes.POINTER(DP)]
        L.orc_glm_get_state.argtypes = [P, ctypes.POINTER(DP)]
        L.orc_glm_cfl_dt.restype = D
        L.orc_glm_cfl_dt.argtypes = [P]
        L.orc_glm_step.argtypes = [P, D]
        L.orc_glm_ch.restype = D
        L.orc_glm_ch.argtypes = [P]
        L.orc_glm_count_flops.argtypes = [ctypes.POINTER(OrcConfig), D, ctypes.POINTER(DP), ctypes.c_int, D,
                                          ctypes.POINTER(ctypes.c_ulonglong)]
        L.orc_glm_fallbacks.restype = ctypes.c_longlong
        L.orc_glm_fallbacks.argtypes = [P]
        L.orc_count_tape.argtypes = [ctypes.POINTER(OrcConfig), ctypes.POINTER(DP), ctypes.c_int, D,
                                     ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]
        L.orc_count_wenoz_shared.restype = ctypes.c_ulonglong
        L.orc_count_wenoz_shared.argtypes = [DP]
        L.orc_state_from_prims.argtypes = [ctypes.POINTER(OrcConfig), PP, PP, ctypes.POINTER(DP)]
        _lib = L
    return _lib


def make_config(cfg):
    """cfg: dict with ndim, n (tuple), x0, x1, gamma, recon, riemann, rk, cfl, bc (6 names)."""
    c = OrcConfig()
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    c.ndim = cfg["ndim"]
    c.nx, c.ny, c.nz = n[0], n[1], n[2] if cfg["ndim"] == 3 else 1
    x0 = list(cfg["x0"]) + [0.0] * (3 - len(cfg["x0"]))
    x1 = list(cfg["x1"]) + [1.0] * (3 - len(cfg["x1"]))
    for d in range(3):
        c.x0[d] = x0[d]
        c.x1[d] = x1[d]
    c.gamma = cfg["gamma"]
    c.recon = RECON[cfg["recon"]]
    c.riemann = RIEMANN[cfg["riemann"]]
    c.rk = cfg["rk"]
    c.cfl = cfg["cfl"]
    for s in range(6):
        c.bc[s] = BC[cfg["bc"][s]]
    c.p_floor = cfg.get("p_floor", 0.0)
    c.emf = EMF[cfg.get("emf", "uct_hll")]
    return c


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptrs(arrays):
    arrays = list(arrays)
    arr = (ctypes.POINTER(ctypes.c_double) * max(8, len(arrays)))()
    for q, a in enumerate(arrays):
        arr[q] = _dp(a)
    return arr


def state_shapes(cfg):
    nd = cfg["ndim"]
    nx, ny = cfg["n"][0], cfg["n"][1]
    nz = cfg["n"][2] if nd == 3 else 1
    cell = (nz, ny, nx)
    if nd == 3:
        faces = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    else:
        faces = [(1, ny, nx + 1), (1, ny + 1, nx), (1, ny, nx)]
    return [cell] * 5 + faces


class OracleSim:
    """One grid advanced by the oracle scheme."""

    def __init__(self, cfg, state=None):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.h = lib().orc_create(ctypes.byref(self._c))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.shapes = state_shapes(cfg)
        if state is not None:
            self.set_state(state)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_state(self, state):
        arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(s))
                for k, s in zip(KEYS, self.shapes)]
        lib().orc_set_state(self.h, _ptrs(arrs))

    def get_state(self):
        arrs = [np.zeros(s) for s in self.shapes]
        lib().orc_get_state(self.h, _ptrs(arrs))
        return dict(zip(KEYS, arrs))

    def cfl_dt(self):
        return lib().orc_cfl_dt(self.h)

    def step(self, dt):
        rc = lib().orc_step(self.h, float(dt))
        if rc != 0:
            raise FloatingPointError("oracle met a non-positive density or pressure")

    def advance(self, nsteps, record_dt=False):
        dts = []
        for _ in range(nsteps):
            dt = self.cfl_dt()
            self.step(dt)
            dts.append(dt)
        return dts if record_dt else None

    @property
    def time(self):
        return lib().orc_time(self.h)

    @property
    def fallbacks(self):
        return lib().orc_fallbacks(self.h)

    @property
    def floors(self):
        return lib().orc_floors(self.h)

    def emf(self, comp):
        nd = self.cfg["ndim"]
        n = list(self.cfg["n"]) + [1]
        nx, ny, nz = n[0], n[1], (n[2] if nd == 3 else 1)
        ext = {0: (nz + 1, ny + 1, nx), 1: (nz + 1, ny, nx + 1), 2: (nz, ny + 1, nx + 1)}[comp]
        out = np.zeros(ext)
        if lib().orc_get_emf(self.h, comp, _dp(out)) != 0:
            raise ValueError("no such edge field")
        return out

    def stage_increment(self, dt):
        arrs = [np.zeros(s) for s in self.shapes]
        lib().orc_stage_increment(self.h, float(dt), _ptrs(arrs))
        return dict(zip(KEYS, arrs))


GLM_KEYS = ("rho", "mx", "my", "mz", "E", "bx", "by", "bz", "psi")


class OracleGlm:
    """One grid advanced by the oracle scheme with GLM divergence cleaning
    (glm_oracle.hpp): 9 cell-centred variables, GLM_KEYS."""

    def __init__(self, cfg, state=None, alpha=0.1):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.h = lib().orc_glm_create(ctypes.byref(self._c), float(alpha))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.shape = state_shapes(cfg)[0]
        if state is not None:
            self.set_state(state)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_glm_destroy(self.h)
            self.h = None

    def set_state(self, state):
        arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(self.shape)) for k in GLM_KEYS]
        lib().orc_glm_set_state(self.h, _ptrs(arrs))

    def get_state(self):
        arrs = [np.zeros(self.shape) for _ in GLM_KEYS]
        lib().orc_glm_get_state(self.h, _ptrs(arrs))
        return dict(zip(GLM_KEYS, arrs))

    def cfl_dt(self):
        return lib().orc_glm_cfl_dt(self.h)

    def step(self, dt):
        if lib().orc_glm_step(self.h, float(dt)) != 0:
            raise FloatingPointError("oracle met a non-positive density or pressure")

    def advance(self, nsteps, record_dt=False):
        dts = []
        for _ in range(nsteps):
            dt = self.cfl_dt()
            self.step(dt)
            dts.append(dt)
        return dts if record_dt else None

    @property
    def ch(self):
        return lib().orc_glm_ch(self.h)

    def count_flops(self, nsteps, dt, alpha=0.1):
        """Counted-scalar run from the current state: dict phase -> dict op -> count."""
        arrs = [np.ascontiguousarray(a) for a in self.get_state().values()]
        out = (ctypes.c_ulonglong * (len(PHASES) * len(OPS)))()
        lib().orc_glm_count_flops(ctypes.byref(self._c), float(alpha), _ptrs(arrs), int(nsteps), float(dt), out)
        return {ph: {op: int(out[i * len(OPS) + j]) for j, op in enumerate(OPS)} for i, ph in enumerate(PHASES)}

    @property
    def fallbacks(self):
        return lib().orc_glm_fallbacks(self.h)


def riemann(solver, wl, wr, bn, gamma, emf="uct_hll"):
    """Riemann flux (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) and UCT ingredients
    (a^L, a^R, d^L, uL, uR, d^R); emf="uct_hlld" (HLLD only) gives the HLLD
    solver's own weights instead of the HLL ones."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    F = np.zeros(7)
    ing = np.zeros(6)
    code = RIEMANN[solver]
    if emf == "uct_hlld":
        if solver != "hlld":
            raise ValueError("UCT-HLLD ingredients need the HLLD solver")
        code = 2
    lib().orc_riemann(code, _dp(wl), _dp(wr), float(bn), float(gamma), _dp(F), _dp(ing))
    return F, ing


def side_flux(w, bn, gamma):
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(7)
    U = np.zeros(7)
    lib().orc_side_flux(_dp(w), float(bn), float(gamma), _dp(F), _dp(U))
    return F, U


def recon(method, s5):
    s5 = np.ascontiguousarray(s5, dtype=np.float64)
    p = ctypes.c_double()
    m = ctypes.c_double()
    lib().orc_recon(RECON[method], _dp(s5), ctypes.byref(p), ctypes.byref(m))
    return p.value, m.value


def c2p(u8, gamma):
    u8 = np.ascontiguousarray(u8, dtype=np.float64)
    V = np.zeros(8)
    lib().orc_c2p(_dp(u8), float(gamma), _dp(V))
    return V


def fast_speed(rho, p, B2, bn, gamma):
    return lib().orc_fast_speed(rho, p, B2, bn, gamma)


def cfl_dt_state(cfg, state):
    """CFL dt of a state (external layout) without building the padded grid."""
    c = make_config(cfg)
    arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(s))
            for k, s in zip(KEYS, state_shapes(cfg))]
    return lib().orc_cfl_dt_state(ctypes.byref(c), _ptrs(arrs))


def count_wenoz_shared(stencil=(0.3, -1.2, 0.7, 2.1, -0.4)):
    """Counted flops of the face-independent part of one WENO-Z face value
    (indicators, tau5, ratios, 1 + ratio^2), which is the same for both faces
    of a cell; the count does not depend on the stencil's values."""
    a = np.ascontiguousarray(stencil, dtype=np.float64)
    return int(lib().orc_count_wenoz_shared(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def count_flops(cfg, state, nsteps, dt):
    """Counted-scalar run: dict phase -> dict op -> count (one CFL + nsteps steps)."""
    c = make_config(cfg)
    shapes = state_shapes(cfg)
    arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(s)) for k, s in zip(KEYS, shapes)]
    out = (ctypes.c_ulonglong * (len(PHASES) * len(OPS)))()
    lib().orc_count_flops(ctypes.byref(c), _ptrs(arrs), int(nsteps), float(dt), out)
    res = {}
    for i, ph in enumerate(PHASES):
        res[ph] = {op: int(out[i * len(OPS) + j]) for j, op in enumerate(OPS)}
    return res


def count_tape(cfg, state, nsteps, dt):
    """Reverse-mode work of nsteps steps (every state element a tape
    variable): dict phase -> (backward-sweep flops, partial-derivative flops)."""
    c = make_config(cfg)
    shapes = state_shapes(cfg)
    arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(s)) for k, s in zip(KEYS, shapes)]
    links = (ctypes.c_ulonglong * len(PHASES))()
    pfl = (ctypes.c_ulonglong * len(PHASES))()
    lib().orc_count_tape(ctypes.byref(c), _ptrs(arrs), int(nsteps), float(dt), links, pfl)
    return {ph: (int(links[i]), int(pfl[i])) for i, ph in enumerate(PHASES)}


FUNCTIONALS = {"magnetic_energy": 0, "misfit": 1}


def _parr(arrs):
    out = (ctypes.POINTER(ctypes.c_double) * len(arrs))()
    for i, a in enumerate(arrs):
        out[i] = _dp(a)
    return out


def _prim_args(cfg, prim, B, dts, target):
    """prim: dict rho, vx, vy, vz, p (cell arrays); B: (b0, b1, b2) in the state layout."""
    shapes = state_shapes(cfg)
    P = [np.ascontiguousarray(np.asarray(prim[k], dtype=np.float64).reshape(shapes[0]))
         for k in ("rho", "vx", "vy", "vz", "p")]
    Bs = [np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(s)) for b, s in zip(B, shapes[5:])]
    d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    T = None
    if target is not None:
        T = [np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(shapes[0])) for t in target]
    keep = (P, Bs, d, T)
    return keep, _parr(P), _parr(Bs), _dp(d), (_parr(T) if T is not None else None)


def state_from_prims(cfg, prim, B):
    """The conserved state (dict of KEYS) that the functional's initial map
    builds from primitives rho, vx, vy, vz, p and the field B (Eq. Energy)."""
    keep, P, Bp, d, T = _prim_args(cfg, prim, B, [], None)
    arrs = [np.zeros(s) for s in state_shapes(cfg)]
    lib().orc_state_from_prims(ctypes.byref(make_config(cfg)), P, Bp, _ptrs(arrs))
    return dict(zip(KEYS, arrs))


def functional_prim(cfg, prim, B, dts, which="magnetic_energy", target=None, signature=False):
    """J after len(dts) steps of the given sizes from initial primitives (p and B
    fixed); with signature=True also the hash of every branch decision taken."""
    keep, P, Bp, d, T = _prim_args(cfg, prim, B, dts, target)
    J = ctypes.c_double()
    sig = ctypes.c_ulonglong()
    rc = lib().orc_functional_prim(ctypes.byref(make_config(cfg)), P, Bp, d, len(dts), FUNCTIONALS[which], T,
                                   ctypes.byref(J), ctypes.byref(sig))
    if rc:
        raise FloatingPointError("non-positive density or pressure")
    return (J.value, sig.value) if signature else J.value


def jvp_prim(cfg, prim, B, dts, tangent, which="magnetic_energy", target=None):
    """(J, dJ): forward-mode derivative of J along tangent = dict rho, vx, vy, vz."""
    keep, P, Bp, d, T = _prim_args(cfg, prim, B, dts, target)
    tg = [np.ascontiguousarray(np.asarray(tangent[k], dtype=np.float64).reshape(keep[0][0].shape))
          for k in ("rho", "vx", "vy", "vz")]
    J, dJ = ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_jvp_prim(ctypes.byref(make_config(cfg)), P, Bp, d, len(dts), FUNCTIONALS[which], T, _parr(tg),
                            ctypes.byref(J), ctypes.byref(dJ))
    if rc:
        raise FloatingPointError("non-positive density or pressure")
    return J.value, dJ.value


def grad_prim(cfg, prim, B, dts, which="magnetic_energy", target=None):
    """(J, grad): reverse-mode gradient of J w.r.t. the initial rho, vx, vy, vz."""
    keep, P, Bp, d, T = _prim_args(cfg, prim, B, dts, target)
    g = [np.zeros(keep[0][0].shape) for _ in range(4)]
    J = ctypes.c_double()
    rc = lib().orc_grad_prim(ctypes.byref(make_config(cfg)), P, Bp, d, len(dts), FUNCTIONALS[which], T,
                             ctypes.byref(J), _parr(g))
    if rc:
        raise FloatingPointError("non-positive density or pressure")
    return J.value, dict(zip(("rho", "vx", "vy", "vz"), g))


def grad_conserved(cfg, state, dts, which="magnetic_energy", target=None):
    """(J, grad): reverse-mode gradient of J w.r.t. every element of the initial
    conserved state (dict of KEYS; on a periodic axis the face at n is the
    ghost copy of face 0 and its entry is 0)."""
    shapes = state_shapes(cfg)
    arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(sh)) for k, sh in zip(KEYS, shapes)]
    d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    T = None
    if target is not None:
        T = [np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(shapes[0])) for t in target]
    g = [np.zeros(sh) for sh in shapes]
    J = ctypes.c_double()
    rc = lib().orc_grad_conserved(ctypes.byref(make_config(cfg)), _ptrs(arrs), _dp(d), len(dts), FUNCTIONALS[which],
                                  _parr(T) if T is not None else None, ctypes.byref(J), _parr(g))
    if rc:
        raise FloatingPointError("non-positive density or pressure")
    return J.value, dict(zip(KEYS, g))


def stage_vjp(cfg, state, dt, w):
    """(J, grad): J = <w, U + L(U)> over the evolved cells and faces after one
    first RK stage of size dt from state U, and its reverse-mode gradient
    with respect to every element of U (dicts of KEYS)."""
    shapes = state_shapes(cfg)
    arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(sh)) for k, sh in zip(KEYS, shapes)]
    ws = [np.ascontiguousarray(np.asarray(w[k], dtype=np.float64).reshape(sh)) for k, sh in zip(KEYS, shapes)]
    g = [np.zeros(sh) for sh in shapes]
    J = ctypes.c_double()
    rc = lib().orc_stage_vjp(ctypes.byref(make_config(cfg)), _ptrs(arrs), float(dt), _ptrs(ws), ctypes.byref(J),
                             _parr(g))
    if rc:
        raise FloatingPointError("non-positive density or pressure")
    return J.value, dict(zip(KEYS, g))
