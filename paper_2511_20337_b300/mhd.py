"""Thin ctypes binding of libmhd (include/mhd.h): argument marshalling only.

Every step of the method runs in the CUDA library.  There is no fallback: if
libmhd.so is missing or cannot be loaded, every call raises.

State dictionaries use the library's external layout (see include/mhd.h):
keys rho, mx, my, mz, E, b0, b1, b2 with b0/b1 the face fields Bx/By and b2
the face Bz (3D) or the cell-centred Bz (2D).  Values may be numpy arrays
(host memory) or CUDA torch tensors (device memory).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libmhd.so")

MHD_OK = 0
ERRORS = {-1: "MHD_ERR_ARG", -2: "MHD_ERR_CUDA", -3: "MHD_ERR_OOM", -4: "MHD_ERR_UNPHYSICAL",
          -5: "MHD_ERR_TIMEOUT", -6: "MHD_ERR_STATE", -7: "MHD_ERR_TOO_LARGE", -8: "MHD_ERR_DIVB",
          -9: "MHD_ERR_GUARD"}
RECON = {"plm": 0, "wenoz": 1, "ppm": 2}
RIEMANN = {"hll": 0, "hlld": 1}
BC = {"periodic": 0, "outflow": 1}
MEM_HOST, MEM_DEVICE = 0, 1
KEYS = ("rho", "mx", "my", "mz", "E", "b0", "b1", "b2")
DIVB = {"ct": 0, "glm": 1}
EMF = {"uct_hll": 0, "uct_hlld": 1}
# divergence cleaning: cell-centred field and psi
GLM_KEYS = ("rho", "mx", "my", "mz", "E", "bx", "by", "bz", "psi")

# every exported entry point of include/mhd.h
EXPORTS = ("mhd_create", "mhd_destroy", "mhd_set_conserved", "mhd_set_prim", "mhd_get_conserved",
           "mhd_set_boundaries", "mhd_cfl_dt", "mhd_step", "mhd_advance", "mhd_get_time", "mhd_last_dt",
           "mhd_status", "mhd_launch_count", "mhd_strerror", "mhd_counters", "mhd_profile_steps", "mhd_probe_fp64",
           "mhd_step_noalloc", "mhd_batch_create", "mhd_batch_destroy", "mhd_batch_set_conserved",
           "mhd_batch_get_conserved", "mhd_batch_step", "mhd_batch_autotune", "mhd_batch_set_seglen",
           "mhd_batch_get_times", "mhd_batch_status", "mhd_batch_launch_count", "mhd_batch_profile_steps",
           "mhd_adjoint_run", "mhd_adjoint_grad_conserved", "mhd_adjoint_grad_prim", "mhd_adjoint_profile", "mhd_probe_riemann_vjp",
           "mhd_probe_riemann_vjp_emf", "mhd_probe_ghost_vjp",
           "mhd_probe_stage_vjp",
           "mhd_set_divb_check", "mhd_divb",
           "mhd_set_seglen", "mhd_autotune", "mhd_set_psi", "mhd_get_psi", "mhd_probe_cfl_rate", "mhd_get_seglen",
           "mhd_batch_get_conserved_async", "mhd_batch_synchronize", "mhd_batch_packed_size",
           "mhd_batch_set_conserved_packed", "mhd_batch_get_conserved_packed", "mhd_set_time",
           "mhd_probe_riemann", "mhd_probe_fp64_forms",
           "mhd_domain_brick", "mhd_domain_halo", "mhd_domain_create", "mhd_domain_destroy",
           "mhd_domain_set_conserved", "mhd_domain_get_conserved", "mhd_domain_cfl_dt", "mhd_domain_step",
           "mhd_domain_advance", "mhd_domain_get_time", "mhd_domain_status", "mhd_domain_counters",
           "mhd_domain_set_seglen", "mhd_domain_launch_count", "mhd_domain_halo_bytes",
           "mhd_set_fused", "mhd_get_fused", "mhd_set_wait_limit", "mhd_inject_skip_arrive", "mhd_fused_waits",
           "mhd_check_guards", "mhd_guard_layout", "mhd_inject_guard_write", "mhd_batch_check_guards",
           "mhd_domain_check_guards")
# field of mhd_domain_check_guards: a brick's region of the halo send / receive buffer
GUARD_SEND, GUARD_RECV = -2, -3
FUNCTIONALS = {"magnetic_energy": 0, "misfit": 1}
KCLASSES = ("ghost", "prim", "sweep_x", "sweep_y", "sweep_z", "emf", "ct_rk", "other")
AKCLASSES = KCLASSES + ("adj_combine", "adj_edge", "adj_riemann", "adj_recon", "adj_c2p", "adj_ghost")


class MhdError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({lib().mhd_strerror(code).decode()})")
        self.code = code


class mhd_halo_box(ctypes.Structure):
    _fields_ = [("peer", ctypes.c_int), ("dir", ctypes.c_int * 3), ("lo", ctypes.c_int * 3),
                ("ext", ctypes.c_int * 3), ("offset", ctypes.c_longlong)]


class mhd_config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("x1", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("recon", ctypes.c_int), ("riemann", ctypes.c_int), ("rk", ctypes.c_int),
                ("cfl", ctypes.c_double), ("bc", ctypes.c_int * 6), ("p_floor", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("divb", ctypes.c_int), ("glm_alpha", ctypes.c_double),
                ("emf", ctypes.c_int)]


_lib = None


def lib():
    """Load libmhd.so (built in-tree by paper_2511_20337_b300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO):
            raise ImportError(f"libmhd.so not built ({SO}); run python -m paper_2511_20337_b300.build")
        L = ctypes.CDLL(SO)
        P = ctypes.c_void_p
        DPP = ctypes.POINTER(ctypes.c_void_p)
        I, D = ctypes.c_int, ctypes.c_double
        sig = {
            "mhd_create": (I, [ctypes.POINTER(mhd_config), ctypes.POINTER(P)]),
            "mhd_destroy": (I, [P]),
            "mhd_set_conserved": (I, [P, I, DPP, DPP]),
            "mhd_set_prim": (I, [P, I, P, DPP, P, DPP]),
            "mhd_get_conserved": (I, [P, I, DPP, DPP]),
            "mhd_set_boundaries": (I, [P, ctypes.POINTER(I)]),
            "mhd_cfl_dt": (I, [P, ctypes.POINTER(D)]),
            "mhd_step": (I, [P, D]),
            "mhd_advance": (I, [P, I]),
            "mhd_get_time": (I, [P, ctypes.POINTER(D)]),
            "mhd_last_dt": (I, [P, ctypes.POINTER(D)]),
            "mhd_status": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_launch_count": (ctypes.c_longlong, [P]),
            "mhd_counters": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_strerror": (ctypes.c_char_p, [I]),
            "mhd_profile_steps": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(I)]),
            "mhd_probe_fp64": (I, [ctypes.POINTER(D)]),
            "mhd_probe_fp64_forms": (I, [P]),
            "mhd_step_noalloc": (I, [ctypes.POINTER(mhd_config), DPP, DPP, D]),
            "mhd_batch_create": (I, [I, ctypes.POINTER(mhd_config), ctypes.POINTER(P)]),
            "mhd_batch_destroy": (I, [P]),
            "mhd_batch_set_conserved": (I, [P, I, I, DPP, DPP]),
            "mhd_batch_get_conserved": (I, [P, I, I, DPP, DPP]),
            "mhd_batch_get_conserved_async": (I, [P, I, I, DPP, DPP]),
            "mhd_batch_synchronize": (I, [P]),
            "mhd_batch_packed_size": (ctypes.c_longlong, [P]),
            "mhd_set_time": (I, [P, D]),
            "mhd_batch_set_conserved_packed": (I, [P, I, P]),
            "mhd_batch_get_conserved_packed": (I, [P, I, P]),
            "mhd_batch_step": (I, [P, I]),
            "mhd_batch_autotune": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "mhd_batch_set_seglen": (I, [P, I, I]),
            "mhd_batch_get_times": (I, [P, ctypes.POINTER(D)]),
            "mhd_batch_status": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_batch_launch_count": (ctypes.c_longlong, [P]),
            "mhd_batch_profile_steps": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(I)]),
            "mhd_adjoint_run": (I, [P, I, ctypes.POINTER(D), I, I, I, DPP, ctypes.POINTER(D), ctypes.POINTER(D)]),
            "mhd_adjoint_grad_conserved": (I, [P, I, DPP, DPP]),
            "mhd_adjoint_grad_prim": (I, [P, I, P, DPP]),
            "mhd_adjoint_profile": (I, [P, I, ctypes.POINTER(D), I, ctypes.POINTER(D), ctypes.POINTER(D)]),
            "mhd_probe_riemann_vjp": (I, [I, I, D, P, P, P, P]),
            "mhd_probe_riemann_vjp_emf": (I, [I, I, I, D, P, P, P, P]),
            "mhd_probe_ghost_vjp": (I, [P, P, P, P, P]),
            "mhd_probe_stage_vjp": (I, [P, DPP, D, DPP, DPP]),
            "mhd_set_seglen": (I, [P, I]),
            "mhd_autotune": (I, [P, ctypes.POINTER(I)]),
            "mhd_set_psi": (I, [P, I, P]),
            "mhd_get_psi": (I, [P, I, P]),
            "mhd_probe_cfl_rate": (I, [I, D, P, I, P, P, P]),
            "mhd_probe_riemann": (I, [I, I, I, D, P, P, P]),
            "mhd_get_seglen": (I, [P, ctypes.POINTER(I)]),
            "mhd_set_divb_check": (I, [P, D]),
            "mhd_divb": (I, [P, ctypes.POINTER(D)]),
            "mhd_domain_brick": (I, [ctypes.POINTER(mhd_config), ctypes.POINTER(I), I, ctypes.POINTER(I),
                                     ctypes.POINTER(I)]),
            "mhd_domain_halo": (I, [ctypes.POINTER(mhd_config), ctypes.POINTER(I), I, I,
                                    ctypes.POINTER(mhd_halo_box), I, ctypes.POINTER(I)]),
            "mhd_domain_create": (I, [ctypes.POINTER(mhd_config), ctypes.POINTER(I), ctypes.POINTER(P)]),
            "mhd_domain_destroy": (I, [P]),
            "mhd_domain_set_conserved": (I, [P, I, DPP, DPP]),
            "mhd_domain_get_conserved": (I, [P, I, DPP, DPP]),
            "mhd_domain_cfl_dt": (I, [P, ctypes.POINTER(D)]),
            "mhd_domain_step": (I, [P, D]),
            "mhd_domain_advance": (I, [P, I]),
            "mhd_domain_get_time": (I, [P, ctypes.POINTER(D)]),
            "mhd_domain_status": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_domain_counters": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_domain_set_seglen": (I, [P, I]),
            "mhd_domain_launch_count": (ctypes.c_longlong, [P]),
            "mhd_domain_halo_bytes": (ctypes.c_longlong, [P]),
            "mhd_set_fused": (I, [P, I]),
            "mhd_get_fused": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "mhd_set_wait_limit": (I, [P, D]),
            "mhd_inject_skip_arrive": (I, [P, I, I]),
            "mhd_fused_waits": (I, [P, ctypes.POINTER(I)]),
            "mhd_check_guards": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_guard_layout": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_inject_guard_write": (I, [P, I, ctypes.c_longlong]),
            "mhd_batch_check_guards": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I),
                                           ctypes.POINTER(ctypes.c_longlong)]),
            "mhd_domain_check_guards": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I),
                                            ctypes.POINTER(ctypes.c_longlong)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, what):
    if rc != MHD_OK:
        raise MhdError(rc, what)


def make_config(cfg, stream=None):
    c = mhd_config()
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    c.ndim = cfg["ndim"]
    c.nx, c.ny = n[0], n[1]
    c.nz = n[2] if cfg["ndim"] == 3 else 1
    x0 = list(cfg["x0"]) + [0.0] * (3 - len(cfg["x0"]))
    x1 = list(cfg["x1"]) + [1.0] * (3 - len(cfg["x1"]))
    for d in range(3):
        c.x0[d], c.x1[d] = x0[d], x1[d]
    c.gamma = cfg["gamma"]
    c.recon = RECON[cfg["recon"]]
    c.riemann = RIEMANN[cfg["riemann"]]
    c.rk = cfg["rk"]
    c.cfl = cfg["cfl"]
    for s in range(6):
        c.bc[s] = BC[cfg["bc"][s]]
    c.p_floor = cfg.get("p_floor", 0.0)
    c.stream = stream
    c.divb = DIVB[cfg.get("divb", "ct")]
    c.glm_alpha = cfg.get("glm_alpha", 0.1)
    c.emf = EMF[cfg.get("emf", "uct_hll")]
    return c


def state_shapes(cfg):
    nd = cfg["ndim"]
    nx, ny = cfg["n"][0], cfg["n"][1]
    nz = cfg["n"][2] if nd == 3 else 1
    cell = (nz, ny, nx)
    if cfg.get("divb", "ct") == "glm":
        return [cell] * 8
    faces = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx) if nd == 3 else (1, ny, nx)]
    return [cell] * 5 + faces


def _is_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a):
    if hasattr(a, "data_ptr"):
        if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise ValueError("arrays must be C-contiguous float64")
    return ctypes.c_void_p(a.ctypes.data)


def _host_arrays(arrs, shapes):
    """Host arrays as the library reads them: C-contiguous float64 of the slot
    shapes.  Contiguous float64 CPU tensors of the right size are passed as
    they are (no conversion); anything else goes through numpy."""
    out = []
    for a, s in zip(arrs, shapes):
        if hasattr(a, "data_ptr") and str(a.dtype) == "torch.float64" and a.is_contiguous() \
                and a.numel() == int(np.prod(s)):
            out.append(a)
        else:
            out.append(np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(s)))
    return out


def _ptr_array(arrs):
    out = (ctypes.c_void_p * len(arrs))()
    for i, a in enumerate(arrs):
        out[i] = _ptr(a)
    return out


class Sim:
    """One grid in device memory, advanced by libmhd on one GPU."""

    def __init__(self, cfg, state=None, stream=None):
        self.cfg = dict(cfg)
        self.shapes = state_shapes(cfg)
        self._c = make_config(cfg, stream)
        h = ctypes.c_void_p()
        _check(lib().mhd_create(ctypes.byref(self._c), ctypes.byref(h)), "mhd_create")
        self.h = h
        if state is not None:
            self.set_conserved(state)

    def close(self):
        if getattr(self, "h", None):
            lib().mhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def glm(self):
        return self.cfg.get("divb", "ct") == "glm"

    @property
    def keys(self):
        """State keys: KEYS (CT: face fields b0, b1, b2) or GLM_KEYS (cell field and psi)."""
        return GLM_KEYS if self.glm else KEYS

    def set_conserved(self, state):
        """Set the state from a dict of self.keys (GLM: psi optional, default 0)."""
        keys = self.keys[:8]
        arrs = [state[k] for k in keys]
        dev = _is_device(arrs[0])
        if not dev:
            arrs = _host_arrays(arrs, self.shapes)
        self._keep = arrs
        U = _ptr_array(arrs[:5])
        B = _ptr_array(arrs[5:])
        _check(lib().mhd_set_conserved(self.h, MEM_DEVICE if dev else MEM_HOST, U, B), "mhd_set_conserved")
        if self.glm and state.get("psi") is not None:
            self.set_psi(state["psi"])

    def set_psi(self, psi):
        dev = _is_device(psi)
        if not dev:
            psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float64).reshape(self.shapes[0]))
        self._keep_psi = psi
        _check(lib().mhd_set_psi(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr(psi)), "mhd_set_psi")

    def get_psi(self, out=None):
        if out is None:
            out = np.zeros(self.shapes[0])
        _check(lib().mhd_get_psi(self.h, MEM_DEVICE if _is_device(out) else MEM_HOST, _ptr(out)), "mhd_get_psi")
        return out

    def set_prim(self, rho, v, p, B):
        dev = _is_device(rho)
        arrs = [rho, *v, p, *B]
        if not dev:
            arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in arrs]
        self._keep = arrs
        _check(lib().mhd_set_prim(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr(arrs[0]), _ptr_array(arrs[1:4]),
                                  _ptr(arrs[4]), _ptr_array(arrs[5:8])), "mhd_set_prim")

    def get_conserved(self, out=None):
        """Copy the state out: into `out` (dict of numpy arrays or CUDA tensors) or new numpy arrays;
        keys self.keys (GLM: psi included)."""
        keys = self.keys[:8]
        if out is None:
            out = {k: np.zeros(s) for k, s in zip(keys, self.shapes)}
        arrs = [out[k] for k in keys]
        dev = _is_device(arrs[0])
        _check(lib().mhd_get_conserved(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr_array(arrs[:5]),
                                       _ptr_array(arrs[5:])), "mhd_get_conserved")
        if self.glm:
            if "psi" not in out:
                out["psi"] = np.zeros(self.shapes[0])
            self.get_psi(out["psi"])
        return out

    def cfl_dt(self):
        dt = ctypes.c_double()
        _check(lib().mhd_cfl_dt(self.h, ctypes.byref(dt)), "mhd_cfl_dt")
        return dt.value

    def step(self, dt):
        _check(lib().mhd_step(self.h, float(dt)), "mhd_step")

    def advance(self, nsteps):
        _check(lib().mhd_advance(self.h, int(nsteps)), "mhd_advance")

    def status(self):
        bad = ctypes.c_longlong()
        rc = lib().mhd_status(self.h, ctypes.byref(bad))
        return rc, bad.value

    def set_seglen(self, seglen):
        _check(lib().mhd_set_seglen(self.h, int(seglen)), "mhd_set_seglen")

    @property
    def seglen(self):
        s = ctypes.c_int()
        _check(lib().mhd_get_seglen(self.h, ctypes.byref(s)), "mhd_get_seglen")
        return s.value

    def autotune(self):
        """Pick the sweep segment length by timing (state restored); returns it."""
        s = ctypes.c_int()
        _check(lib().mhd_autotune(self.h, ctypes.byref(s)), "mhd_autotune")
        return s.value

    def set_fused(self, on):
        """One cooperative launch per RK stage (2D CT grids that qualify) or one per phase."""
        _check(lib().mhd_set_fused(self.h, 1 if on else 0), "mhd_set_fused")

    @property
    def fused(self):
        """(on, blocks): whether the fused stage is on and its launch's block count (0: not eligible)."""
        on, blocks = ctypes.c_int(), ctypes.c_int()
        _check(lib().mhd_get_fused(self.h, ctypes.byref(on), ctypes.byref(blocks)), "mhd_get_fused")
        return bool(on.value), blocks.value

    def set_wait_limit(self, seconds):
        """Bound of every grid-barrier wait of the fused stage."""
        _check(lib().mhd_set_wait_limit(self.h, float(seconds)), "mhd_set_wait_limit")

    def inject_skip_arrive(self, block, barrier):
        """Fault injection: block `block` skips its arrival at barrier `barrier` of each stage (-1: off)."""
        _check(lib().mhd_inject_skip_arrive(self.h, int(block), int(barrier)), "mhd_inject_skip_arrive")

    def fused_waits(self):
        """Barriers per stage of the last fused launch."""
        n = ctypes.c_int()
        _check(lib().mhd_fused_waits(self.h, ctypes.byref(n)), "mhd_fused_waits")
        return n.value

    def check_guards(self):
        """None when every guard word of the pool is intact, else (field, word) of the
        first damaged one (word < 0: before field 0; word >= 0: past the field's end)."""
        f, w = ctypes.c_int(), ctypes.c_longlong()
        rc = lib().mhd_check_guards(self.h, ctypes.byref(f), ctypes.byref(w))
        if rc == -9:
            return f.value, w.value
        _check(rc, "mhd_check_guards")
        return None

    @property
    def guard_layout(self):
        """(fields in the pool, elements each uses, guard words after each)."""
        n, u, a = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().mhd_guard_layout(self.h, ctypes.byref(n), ctypes.byref(u), ctypes.byref(a)), "mhd_guard_layout")
        return n.value, u.value, a.value

    def inject_guard_write(self, field, word):
        """For tests: write 0.0 into a guard word from the host, as an out-of-bounds store would."""
        _check(lib().mhd_inject_guard_write(self.h, int(field), int(word)), "mhd_inject_guard_write")

    def set_divb_check(self, tol):
        """Check max |div B| h / max |B_c| at the end of every step (tol > 0; 0 = off)."""
        _check(lib().mhd_set_divb_check(self.h, float(tol)), "mhd_set_divb_check")

    def divb(self):
        """max |div B| h / max |B_c| of the current state."""
        r = ctypes.c_double()
        _check(lib().mhd_divb(self.h, ctypes.byref(r)), "mhd_divb")
        return r.value

    def set_boundaries(self, bc):
        arr = (ctypes.c_int * 6)(*[BC[b] for b in bc])
        _check(lib().mhd_set_boundaries(self.h, arr), "mhd_set_boundaries")

    @property
    def time(self):
        t = ctypes.c_double()
        _check(lib().mhd_get_time(self.h, ctypes.byref(t)), "mhd_get_time")
        return t.value

    @time.setter
    def time(self, t):
        _check(lib().mhd_set_time(self.h, float(t)), "mhd_set_time")

    @property
    def last_dt(self):
        t = ctypes.c_double()
        _check(lib().mhd_last_dt(self.h, ctypes.byref(t)), "mhd_last_dt")
        return t.value

    def counters(self):
        """(reconstruction fallbacks, pressure floors) since the last state set."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().mhd_counters(self.h, ctypes.byref(a), ctypes.byref(b)), "mhd_counters")
        return a.value, b.value

    @property
    def launches(self):
        return lib().mhd_launch_count(self.h)

    def profile_steps(self, nsteps):
        """Advance nsteps CFL steps with an event after each kernel: per-class
        device milliseconds and launch counts."""
        ms = (ctypes.c_double * len(KCLASSES))()
        cnt = (ctypes.c_int * len(KCLASSES))()
        _check(lib().mhd_profile_steps(self.h, int(nsteps), ms, cnt), "mhd_profile_steps")
        return {k: ms[i] for i, k in enumerate(KCLASSES)}, {k: cnt[i] for i, k in enumerate(KCLASSES)}


    def adjoint(self, nsteps, dts=None, ckpt_every=20, functional="magnetic_energy", target=None):
        """Run nsteps steps from the current state and take the gradient of the
        final-state functional J (magnetic_energy, or misfit to `target`, a
        list of 5 (3D) or 6 (2D) cell arrays rho, mx, my, mz, E[, b2]) with
        respect to the initial state, the step sizes frozen (given `dts`, else
        the CFL steps of this run).  Returns (J, dts used); the gradient is
        read with grad_prim / grad_conserved."""
        nsteps = int(nsteps)
        d = None
        if dts is not None:
            dts = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
            if dts.shape != (nsteps,):
                raise ValueError("dts must hold nsteps step sizes")
            d = dts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        T, mem = None, MEM_HOST
        if target is not None:
            tg = list(target)
            mem = MEM_DEVICE if _is_device(tg[0]) else MEM_HOST
            if mem == MEM_HOST:
                tg = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(self.shapes[0])) for a in tg]
            self._keep_target = tg
            T = _ptr_array(tg)
        J = ctypes.c_double()
        out = np.zeros(nsteps)
        _check(lib().mhd_adjoint_run(self.h, nsteps, d, int(ckpt_every), FUNCTIONALS[functional], mem, T,
                                     ctypes.byref(J), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "mhd_adjoint_run")
        return J.value, out

    def adjoint_profile(self, nsteps, dts=None, ckpt_every=20):
        """Adjoint run of the magnetic energy with device times: (phase ms
        {forward, recompute, reverse}, reverse-pass ms per kernel class)."""
        nsteps = int(nsteps)
        d = None
        if dts is not None:
            dts = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
            d = dts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        ph = (ctypes.c_double * 3)()
        cl = (ctypes.c_double * len(AKCLASSES))()
        _check(lib().mhd_adjoint_profile(self.h, nsteps, d, int(ckpt_every), ph, cl), "mhd_adjoint_profile")
        return dict(zip(("forward", "recompute", "reverse"), ph)), {k: cl[i] for i, k in enumerate(AKCLASSES)}

    def grad_prim(self, out=None):
        """Gradient of the last adjoint run w.r.t. the initial rho, vx, vy, vz
        (p and B held): dict of cell arrays, numpy or the given CUDA tensors."""
        keys = ("rho", "vx", "vy", "vz")
        if out is None:
            out = {k: np.zeros(self.shapes[0]) for k in keys}
        arrs = [out[k] for k in keys]
        dev = _is_device(arrs[0])
        _check(lib().mhd_adjoint_grad_prim(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr(arrs[0]),
                                           _ptr_array(arrs[1:])), "mhd_adjoint_grad_prim")
        return out

    def grad_conserved(self, out=None):
        """Gradient of the last adjoint run w.r.t. the initial conserved state
        (keys of KEYS; the duplicate last face of a periodic axis carries 0)."""
        if out is None:
            out = {k: np.zeros(s) for k, s in zip(KEYS, self.shapes)}
        arrs = [out[k] for k in KEYS]
        dev = _is_device(arrs[0])
        _check(lib().mhd_adjoint_grad_conserved(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr_array(arrs[:5]),
                                                _ptr_array(arrs[5:])), "mhd_adjoint_grad_conserved")
        return out


def probe_riemann_vjp(solver, inputs, cotangents, gamma, emf=None):
    """The Riemann solver's vector-Jacobian product on the GPU by forward-mode
    numbers and by the hand-written reverse: inputs (n, 15), cotangents (n, 12)
    -> (dual, hand), each (n, 15).  With emf ("uct_hll" or "uct_hlld") the
    cotangents are (n, 13): 7 flux and 6 ingredient (a^L, a^R, d^L, u_L, u_R, d^R)."""
    x = np.ascontiguousarray(np.asarray(inputs, dtype=np.float64))
    c = np.ascontiguousarray(np.asarray(cotangents, dtype=np.float64))
    n = x.shape[0]
    dual, hand = np.zeros((n, 15)), np.zeros((n, 15))
    if emf is None:
        _check(lib().mhd_probe_riemann_vjp(RIEMANN[solver], n, float(gamma), _ptr(x), _ptr(c), _ptr(dual),
                                           _ptr(hand)), "mhd_probe_riemann_vjp")
    else:
        _check(lib().mhd_probe_riemann_vjp_emf(RIEMANN[solver], EMF[emf], n, float(gamma), _ptr(x), _ptr(c),
                                               _ptr(dual), _ptr(hand)), "mhd_probe_riemann_vjp_emf")
    return dual, hand


def probe_ghost_vjp(sim, x, abar):
    """The ghost fill of sim's grid on whole padded fields x (8, E) and its
    transpose on abar (8, E): returns (fill(x), fill^T(abar))."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(abar, dtype=np.float64))
    fx, xb = np.zeros_like(x), np.zeros_like(a)
    _check(lib().mhd_probe_ghost_vjp(sim.h, _ptr(x), _ptr(a), _ptr(fx), _ptr(xb)), "mhd_probe_ghost_vjp")
    return fx, xb


def probe_stage_vjp(sim, state, dt, w):
    """One first RK stage U* = U + L(U) of sim's scheme from state (dict of
    KEYS) with step dt, transposed: returns J^T w (J the Jacobian of U* with
    respect to U) as a dict of KEYS."""
    shapes = sim.shapes
    arrs = [np.ascontiguousarray(np.asarray(state[k], dtype=np.float64).reshape(s)) for k, s in zip(KEYS, shapes)]
    ws = [np.ascontiguousarray(np.asarray(w[k], dtype=np.float64).reshape(s)) for k, s in zip(KEYS, shapes)]
    out = [np.zeros(s) for s in shapes]
    _check(lib().mhd_probe_stage_vjp(sim.h, _ptr_array(arrs), float(dt), _ptr_array(ws), _ptr_array(out)),
           "mhd_probe_stage_vjp")
    return dict(zip(KEYS, out))


def probe_riemann(solver, inputs, gamma, emf="uct_hll"):
    """The sweeps' Riemann solver on the GPU at faces inputs (n, 15) = left
    (rho, u, v, w, b1, b2, p), right (same), b_n -> (F (n, 7), ingredients
    (n, 6) = a^L, a^R, d^L, u_L, u_R, d^R); emf="uct_hlld" gives the HLLD
    weights (HLLD only)."""
    x = np.ascontiguousarray(np.asarray(inputs, dtype=np.float64))
    n = x.shape[0]
    F, ing = np.zeros((n, 7)), np.zeros((n, 6))
    _check(lib().mhd_probe_riemann(RIEMANN[solver], EMF[emf], n, float(gamma), _ptr(x), _ptr(F), _ptr(ing)),
           "mhd_probe_riemann")
    return F, ing


def probe_cfl_rate(ndim, gamma, dx, prim):
    """Both CFL rates of the device for primitive states prim (n, 8) =
    (rho, vx, vy, vz, bx, by, bz, p): (candidate-pass rate, IEEE rate)."""
    x = np.ascontiguousarray(np.asarray(prim, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(dx, dtype=np.float64))
    n = x.shape[0]
    near, ieee = np.zeros(n), np.zeros(n)
    _check(lib().mhd_probe_cfl_rate(int(ndim), float(gamma), _ptr(d), n, _ptr(x), _ptr(near), _ptr(ieee)),
           "mhd_probe_cfl_rate")
    return near, ieee


def probe_fp64_gflops():
    """Measured FP64 FMA throughput of the current device (GFLOP/s, 2 per DFMA)."""
    g = ctypes.c_double()
    _check(lib().mhd_probe_fp64(ctypes.byref(g)), "mhd_probe_fp64")
    return g.value


FP64_FORMS = ("dfma", "dfma_constant_operand", "dfma_distinct_addends", "dmul", "dadd")


def probe_fp64_forms():
    """Issue rates of the FP64 pipe by instruction form, as GFLOP/s
    equivalents (2 per instruction): dict over FP64_FORMS."""
    r = np.zeros(len(FP64_FORMS))
    _check(lib().mhd_probe_fp64_forms(_ptr(r)), "mhd_probe_fp64_forms")
    return dict(zip(FP64_FORMS, r.tolist()))


def step_noalloc(cfg, state, dt, stream=None):
    """One step of size dt, in place, on a state held in CUDA tensors (dict with
    the keys of KEYS), through the allocation-free entry point mhd_step_noalloc:
    no context and no device allocation; the library's fixed scratch array is
    used instead (grids beyond it raise MhdError with MHD_ERR_TOO_LARGE)."""
    arrs = [state[k] for k in KEYS]
    if not all(_is_device(a) for a in arrs):
        raise ValueError("mhd_step_noalloc works on device memory: pass CUDA tensors")
    c = make_config(cfg, stream)
    _check(lib().mhd_step_noalloc(ctypes.byref(c), _ptr_array(arrs[:5]), _ptr_array(arrs[5:]), float(dt)),
           "mhd_step_noalloc")


class Batch:
    """An ensemble of independent grids of one scheme advanced together by
    libmhd's batched entry points (one launch per kernel over all runs)."""

    def __init__(self, cfgs, states=None, stream=None):
        self.cfgs = [dict(c) for c in cfgs]
        self.shapes = [state_shapes(c) for c in cfgs]
        arr = (mhd_config * len(cfgs))()
        for i, c in enumerate(cfgs):
            arr[i] = make_config(c, stream if i == 0 else None)
        h = ctypes.c_void_p()
        _check(lib().mhd_batch_create(len(cfgs), arr, ctypes.byref(h)), "mhd_batch_create")
        self.h = h
        self._keep = {}
        self._pending = []  # destinations of queued read-outs, kept alive until synchronize()
        if states is not None:
            for r, st in enumerate(states):
                self.set_conserved(r, st)

    def close(self):
        if getattr(self, "h", None):
            lib().mhd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_conserved(self, run, state):
        arrs = [state[k] for k in KEYS]
        dev = _is_device(arrs[0])
        if not dev:
            arrs = _host_arrays(arrs, self.shapes[run])
        self._keep[run] = arrs
        _check(lib().mhd_batch_set_conserved(self.h, run, MEM_DEVICE if dev else MEM_HOST, _ptr_array(arrs[:5]),
                                             _ptr_array(arrs[5:])), "mhd_batch_set_conserved")

    def get_conserved(self, run, out=None, wait=True):
        """Copy run's state out (dict of numpy arrays or CUDA tensors, or new
        numpy arrays).  wait=False queues the copies only (out must be pinned
        host memory or device memory, and is complete after synchronize())."""
        if out is None:
            out = {k: np.zeros(s) for k, s in zip(KEYS, self.shapes[run])}
        arrs = [out[k] for k in KEYS]
        dev = _is_device(arrs[0])
        fn = lib().mhd_batch_get_conserved if wait else lib().mhd_batch_get_conserved_async
        _check(fn(self.h, run, MEM_DEVICE if dev else MEM_HOST, _ptr_array(arrs[:5]), _ptr_array(arrs[5:])),
               "mhd_batch_get_conserved")
        if not wait:
            self._pending.append(arrs)
        return out

    def synchronize(self):
        """Wait for the queued work and copies (get_conserved(wait=False), the packed calls)."""
        _check(lib().mhd_batch_synchronize(self.h), "mhd_batch_synchronize")
        self._pending = []

    # ---- packed state I/O: every run's 8 slots in one contiguous array ----
    def packed_size(self):
        return int(lib().mhd_batch_packed_size(self.h))

    def pack(self, states, out=None):
        """The packed array of a list of per-run states (KEYS layout): numpy,
        or written into `out` (e.g. a pinned CPU tensor)."""
        out = np.empty(self.packed_size()) if out is None else out
        flat = out if isinstance(out, np.ndarray) else out.numpy()
        o = 0
        for st, shapes in zip(states, self.shapes):
            for k, s in zip(KEYS, shapes):
                n = int(np.prod(s))
                flat[o:o + n] = np.asarray(st[k], dtype=np.float64).reshape(-1)
                o += n
        return out

    def unpack(self, packed):
        """Per-run state dicts (numpy views) of a packed array."""
        flat = np.asarray(packed.cpu() if hasattr(packed, "cpu") else packed).reshape(-1)
        out, o = [], 0
        for shapes in self.shapes:
            d = {}
            for k, s in zip(KEYS, shapes):
                n = int(np.prod(s))
                d[k] = flat[o:o + n].reshape(s)
                o += n
            out.append(d)
        return out

    def set_conserved_packed(self, packed):
        """Set every run's state from one packed array (numpy, CPU tensor --
        pinned for an overlapped copy -- or CUDA tensor).  Async: keep it
        unchanged until synchronize()."""
        if int(np.prod(packed.shape)) != self.packed_size():
            raise ValueError("packed array of the wrong size")
        dev = _is_device(packed)
        self._keep["packed"] = packed
        _check(lib().mhd_batch_set_conserved_packed(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr(packed)),
               "mhd_batch_set_conserved_packed")

    def get_conserved_packed(self, out=None, wait=True):
        """Every run's state into one packed array (new numpy array, or `out`:
        a pinned CPU tensor or a CUDA tensor for wait=False)."""
        if out is None:
            out = np.empty(self.packed_size())
        if int(np.prod(out.shape)) != self.packed_size():
            raise ValueError("packed array of the wrong size")
        dev = _is_device(out)
        _check(lib().mhd_batch_get_conserved_packed(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr(out)),
               "mhd_batch_get_conserved_packed")
        if wait:
            self.synchronize()
        else:
            self._pending.append(out)
        return out

    def step(self, nsteps):
        _check(lib().mhd_batch_step(self.h, int(nsteps)), "mhd_batch_step")

    def autotune(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().mhd_batch_autotune(self.h, ctypes.byref(a), ctypes.byref(b)), "mhd_batch_autotune")
        return a.value, b.value

    def set_seglen(self, small, large):
        _check(lib().mhd_batch_set_seglen(self.h, int(small), int(large)), "mhd_batch_set_seglen")

    def times(self):
        t = (ctypes.c_double * len(self.cfgs))()
        _check(lib().mhd_batch_get_times(self.h, t), "mhd_batch_get_times")
        return list(t)

    def status(self):
        r, c = ctypes.c_int(), ctypes.c_longlong()
        rc = lib().mhd_batch_status(self.h, ctypes.byref(r), ctypes.byref(c))
        return rc, r.value, c.value

    def check_guards(self):
        """None when every run's guard words are intact, else (run, field, word) of the first damaged one."""
        r, f, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        rc = lib().mhd_batch_check_guards(self.h, ctypes.byref(r), ctypes.byref(f), ctypes.byref(w))
        if rc == -9:
            return r.value, f.value, w.value
        _check(rc, "mhd_batch_check_guards")
        return None

    @property
    def launches(self):
        return lib().mhd_batch_launch_count(self.h)

    def profile_steps(self, nsteps):
        ms = (ctypes.c_double * len(KCLASSES))()
        cnt = (ctypes.c_int * len(KCLASSES))()
        _check(lib().mhd_batch_profile_steps(self.h, int(nsteps), ms, cnt), "mhd_batch_profile_steps")
        return {k: ms[i] for i, k in enumerate(KCLASSES)}, {k: cnt[i] for i, k in enumerate(KCLASSES)}


def final_functional(cfg, rho, vx, vy, vz, p, B, nsteps, dts=None, ckpt_every=20, functional="magnetic_energy",
                     target=None):
    """J(final state) as a differentiable function of the initial rho and v
    (CUDA float64 tensors of the cell shape; p and the face fields B held
    fixed), through torch.autograd: the forward runs libmhd's adjoint (the
    step sizes frozen to `dts`, or to the CFL steps of this run), so backward
    only scales the stored gradient."""
    import torch

    class _Final(torch.autograd.Function):
        @staticmethod
        def forward(ctx, rho_, vx_, vy_, vz_):
            sim = Sim(cfg)
            try:
                sim.set_prim(rho_.contiguous(), [vx_.contiguous(), vy_.contiguous(), vz_.contiguous()],
                             p.contiguous(), [b.contiguous() for b in B])
                J, used = sim.adjoint(nsteps, dts, ckpt_every, functional, target)
                g = {k: torch.empty_like(rho_) for k in ("rho", "vx", "vy", "vz")}
                sim.grad_prim(g)
                torch.cuda.synchronize(rho_.device)
            finally:
                sim.close()
            ctx.save_for_backward(g["rho"], g["vx"], g["vy"], g["vz"])
            ctx.dts = used
            return torch.tensor(J, dtype=torch.float64, device=rho_.device)

        @staticmethod
        def backward(ctx, gJ):
            return tuple(gJ * t for t in ctx.saved_tensors)

    return _Final.apply(rho, vx, vy, vz)


# ---------------------------------------------------------------------------
# domain decomposition: bricks with a halo exchange per stage
# ---------------------------------------------------------------------------
def _parts(parts):
    parts = list(parts) + [1] * (3 - len(parts))
    return (ctypes.c_int * 3)(*parts)


def domain_brick(cfg, parts, brick):
    """(lo, n): first global cell and cells per axis (3 each) of a brick."""
    lo, n = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    _check(lib().mhd_domain_brick(ctypes.byref(make_config(cfg)), _parts(parts), int(brick), lo, n),
           "mhd_domain_brick")
    return tuple(lo), tuple(n)


def domain_halo(cfg, parts, brick, send):
    """The brick's send (send=True) or receive boxes: list of dicts peer, dir,
    lo, ext, offset (see mhd_halo_box in include/mhd.h)."""
    boxes = (mhd_halo_box * 26)()
    nb = ctypes.c_int()
    _check(lib().mhd_domain_halo(ctypes.byref(make_config(cfg)), _parts(parts), int(brick), int(bool(send)), boxes,
                                 26, ctypes.byref(nb)), "mhd_domain_halo")
    return [{"peer": b.peer, "dir": tuple(b.dir), "lo": tuple(b.lo), "ext": tuple(b.ext), "offset": b.offset}
            for b in boxes[:nb.value]]


class Domain:
    """One grid split into bricks (parts = bricks per axis), advanced together
    with a halo exchange per RK stage on one GPU; the state, dt and time are
    the undivided grid's to the bit."""

    def __init__(self, cfg, parts, state=None, stream=None):
        self.cfg = dict(cfg)
        self.parts = tuple(list(parts) + [1] * (3 - len(parts)))
        self.shapes = state_shapes(cfg)
        self._c = make_config(cfg, stream)
        h = ctypes.c_void_p()
        _check(lib().mhd_domain_create(ctypes.byref(self._c), _parts(parts), ctypes.byref(h)), "mhd_domain_create")
        self.h = h
        if state is not None:
            self.set_conserved(state)

    def close(self):
        if getattr(self, "h", None):
            lib().mhd_domain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_conserved(self, state):
        arrs = [state[k] for k in KEYS]
        dev = _is_device(arrs[0])
        if not dev:
            arrs = _host_arrays(arrs, self.shapes)
        self._keep = arrs
        _check(lib().mhd_domain_set_conserved(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr_array(arrs[:5]),
                                              _ptr_array(arrs[5:])), "mhd_domain_set_conserved")

    def get_conserved(self, out=None):
        if out is None:
            out = {k: np.zeros(s) for k, s in zip(KEYS, self.shapes)}
        arrs = [out[k] for k in KEYS]
        dev = _is_device(arrs[0])
        _check(lib().mhd_domain_get_conserved(self.h, MEM_DEVICE if dev else MEM_HOST, _ptr_array(arrs[:5]),
                                              _ptr_array(arrs[5:])), "mhd_domain_get_conserved")
        return out

    def cfl_dt(self):
        dt = ctypes.c_double()
        _check(lib().mhd_domain_cfl_dt(self.h, ctypes.byref(dt)), "mhd_domain_cfl_dt")
        return dt.value

    def step(self, dt):
        _check(lib().mhd_domain_step(self.h, float(dt)), "mhd_domain_step")

    def advance(self, nsteps):
        _check(lib().mhd_domain_advance(self.h, int(nsteps)), "mhd_domain_advance")

    @property
    def time(self):
        t = ctypes.c_double()
        _check(lib().mhd_domain_get_time(self.h, ctypes.byref(t)), "mhd_domain_get_time")
        return t.value

    def status(self):
        bad = ctypes.c_longlong()
        rc = lib().mhd_domain_status(self.h, ctypes.byref(bad))
        return rc, bad.value

    def check_guards(self):
        """None when the bricks' pools and halo buffer regions are intact, else (brick, field, word):
        field >= 0 is a field of the brick's pool, GUARD_SEND / GUARD_RECV its halo buffer region."""
        b, f, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        rc = lib().mhd_domain_check_guards(self.h, ctypes.byref(b), ctypes.byref(f), ctypes.byref(w))
        if rc == -9:
            return b.value, f.value, w.value
        _check(rc, "mhd_domain_check_guards")
        return None

    def counters(self):
        f, p = ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().mhd_domain_counters(self.h, ctypes.byref(f), ctypes.byref(p)), "mhd_domain_counters")
        return f.value, p.value

    def set_seglen(self, seglen):
        _check(lib().mhd_domain_set_seglen(self.h, int(seglen)), "mhd_domain_set_seglen")

    @property
    def launches(self):
        return lib().mhd_domain_launch_count(self.h)

    @property
    def halo_bytes(self):
        return lib().mhd_domain_halo_bytes(self.h)
