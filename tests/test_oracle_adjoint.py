"""Oracle pins for the derivative of a final-state functional w.r.t. the
initial density and velocity (step sizes frozen): the reverse-mode (tape)
gradient, the forward-mode (dual) directional derivative, and central finite
differences must agree (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W

KEYS4 = ("rho", "vx", "vy", "vz")


def prims_of(cfg, st):
    """Primitive arrays and face fields of a conserved state (for the tests)."""
    bx, by, bz = W.cell_field(cfg, st["b0"], st["b1"], st["b2"])
    rho = st["rho"]
    v = [st["mx"] / rho, st["my"] / rho, st["mz"] / rho]
    g = cfg["gamma"]
    p = (g - 1) * (st["E"] - 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) - 0.5 * (bx ** 2 + by ** 2 + bz ** 2))
    return {"rho": rho, "vx": v[0], "vy": v[1], "vz": v[2], "p": p}, (st["b0"], st["b1"], st["b2"])


def frozen_dts(cfg, st, nsteps):
    return oracle.OracleSim(cfg, st).advance(nsteps, record_dt=True)


CASES = {
    "adjoint2d-12-hlld": lambda: W.adjoint_2d(12),
    "adjoint2d-10x8-hll": lambda: (lambda c: (c, W.random_state(c, 51, v=0.2, bamp=0.2)))(
        W.base_cfg(2, (10, 8), (0, 0), (1.0, 0.8), riemann="hll")),
    "random3d-5x4x3-hlld": lambda: (lambda c: (c, W.random_state(c, 52, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (5, 4, 3), (0, 0, 0), (1, 1, 1))),
    "wenoz2d-8x7-hlld-rk3": lambda: (lambda c: (c, W.random_state(c, 54, v=0.2, bamp=0.2)))(
        W.base_cfg(2, (8, 7), (0, 0), (1.0, 0.9), recon="wenoz", rk=3)),
    "ppm2d-7x8-hll": lambda: (lambda c: (c, W.random_state(c, 55, v=0.2, bamp=0.2)))(
        W.base_cfg(2, (7, 8), (0, 0), (0.9, 1.0), recon="ppm", riemann="hll")),
    "wenoz2d-8x8-hlld-rk3-ucthlld": lambda: (lambda c: (c, W.random_state(c, 56, v=0.2, bamp=0.2)))(
        W.base_cfg(2, (8, 8), (0, 0), (1.0, 1.0), recon="wenoz", rk=3, emf="uct_hlld")),
    "plm2d-6x7-hlld-outflow": lambda: (lambda c: (c, W.random_state(c, 57, v=0.2, bamp=0.2)))(
        W.base_cfg(2, (6, 7), (0, 0), (0.6, 0.7), bc="outflow")),
    "plm3d-5x4x5-hll-outflow-z": lambda: (lambda c: (c, W.random_state(c, 58, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (5, 4, 5), (0, 0, 0), (1, 1, 1), riemann="hll",
                   bc=["periodic", "periodic", "periodic", "periodic", "outflow", "outflow"])),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("which", ["magnetic_energy", "misfit"])
def test_tape_gradient_matches_dual_directional_derivative(case, which):
    cfg, st = CASES[case]()
    prim, B = prims_of(cfg, st)
    dts = frozen_dts(cfg, st, 3)
    target = None
    if which == "misfit":
        rng = np.random.default_rng(3)
        keys = ["rho", "mx", "my", "mz", "E"] + (["b2"] if cfg["ndim"] == 2 else [])
        target = [st[k] * (1 + 0.1 * rng.standard_normal(st[k].shape)) for k in keys]
    J, g = oracle.grad_prim(cfg, prim, B, dts, which, target)
    rng = np.random.default_rng(7)
    for _ in range(3):
        tan = {k: rng.standard_normal(prim[k].shape) for k in KEYS4}
        J2, dJ = oracle.jvp_prim(cfg, prim, B, dts, tan, which, target)
        assert J2 == J
        dot = sum(np.sum(g[k] * tan[k]) for k in KEYS4)
        assert abs(dot - dJ) <= 1e-12 * max(abs(dJ), np.sqrt(sum(np.sum(g[k] ** 2) for k in KEYS4)))


def test_tape_gradient_equals_every_unit_jvp():
    """Brute force on a tiny grid: each gradient entry equals the directional
    derivative along that single input."""
    cfg = W.base_cfg(2, (4, 3), (0, 0), (1.0, 0.75))
    st = W.random_state(cfg, 53, v=0.2, bamp=0.2)
    prim, B = prims_of(cfg, st)
    dts = frozen_dts(cfg, st, 2)
    J, g = oracle.grad_prim(cfg, prim, B, dts)
    scale = max(np.max(np.abs(g[k])) for k in KEYS4)
    for k in KEYS4:
        for idx in np.ndindex(prim[k].shape):
            tan = {q: np.zeros(prim[q].shape) for q in KEYS4}
            tan[k][idx] = 1.0
            _, dJ = oracle.jvp_prim(cfg, prim, B, dts, tan)
            assert abs(dJ - g[k][idx]) <= 1e-13 * scale, (k, idx)


def smooth_state(n=16, seed=5):
    cfg, st, prim = W.smooth_2d(n, seed=seed)
    return cfg, st, prim, (st["b0"], st["b1"], st["b2"])


@pytest.mark.parametrize("recon,emf", [("plm", "uct_hll"), ("wenoz", "uct_hll"), ("ppm", "uct_hll"),
                                       ("wenoz", "uct_hlld")])
def test_gradient_matches_central_differences_on_smooth_run(recon, emf):
    """Smooth 16^2 state, 4 steps, misfit to a shifted target so that dJ is of
    the order of J.  Central differences along random directions agree with
    the gradient to 1e-5.  A step size counts only if the branch signature
    (every limiter, min/max and wave-fan decision) is the same at x - h, x and
    x + h; samples that switch a branch are excluded, not passed."""
    cfg, st, prim, B = smooth_state()
    cfg = dict(cfg, recon=recon, emf=emf)
    dts = frozen_dts(cfg, st, 4)
    keys = ["rho", "mx", "my", "mz", "E", "b2"]
    target = [np.roll(st[k], 3, axis=2) * 1.05 for k in keys]
    J, g = oracle.grad_prim(cfg, prim, B, dts, "misfit", target)
    _, sig0 = oracle.functional_prim(cfg, prim, B, dts, "misfit", target, signature=True)
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(4):
        tan = {k: rng.standard_normal(prim[k].shape) for k in KEYS4}
        dot = sum(np.sum(g[k] * tan[k]) for k in KEYS4)
        errs = {}
        for h in (1e-5, 1e-6, 1e-7, 1e-8):
            pp = dict(prim, **{k: prim[k] + h * tan[k] for k in KEYS4})
            pm = dict(prim, **{k: prim[k] - h * tan[k] for k in KEYS4})
            jp, sp = oracle.functional_prim(cfg, pp, B, dts, "misfit", target, signature=True)
            jm, sm = oracle.functional_prim(cfg, pm, B, dts, "misfit", target, signature=True)
            if sp == sig0 and sm == sig0:
                errs[h] = abs((jp - jm) / (2 * h) - dot) / abs(dot)
        if errs:
            checked += 1
            assert min(errs.values()) <= 1e-5, errs
    assert checked >= 3


@pytest.mark.parametrize("case", ["adjoint2d-12-hlld", "random3d-5x4x3-hlld", "plm2d-6x7-hlld-outflow",
                                  "wenoz2d-8x8-hlld-rk3-ucthlld"])
def test_conserved_gradient_reduces_to_the_primitive_one(case):
    """The tape gradient with respect to every conserved element, mapped through
    the initial map U(rho, v; p, B) of Eq. Energy, is the gradient with
    respect to rho and v: d/drho = A_rho + v.A_m + |v|^2/2 A_E and
    d/dv = rho (A_m + v A_E) (p and B held)."""
    cfg, st = CASES[case]()
    prim, B = prims_of(cfg, st)
    U = oracle.state_from_prims(cfg, prim, B)
    dts = frozen_dts(cfg, st, 2)
    J1, gp = oracle.grad_prim(cfg, prim, B, dts)
    J2, gc = oracle.grad_conserved(cfg, U, dts)
    assert J1 == J2
    v = [prim["vx"], prim["vy"], prim["vz"]]
    am = [gc["mx"], gc["my"], gc["mz"]]
    drho = gc["rho"] + sum(vi * ai for vi, ai in zip(v, am)) + 0.5 * sum(vi * vi for vi in v) * gc["E"]
    scale = max(np.max(np.abs(gp[k])) for k in KEYS4)
    assert np.max(np.abs(drho - gp["rho"])) <= 1e-12 * scale
    for k, vi, ai in zip(("vx", "vy", "vz"), v, am):
        assert np.max(np.abs(prim["rho"] * (ai + vi * gc["E"]) - gp[k])) <= 1e-12 * scale, k


def divfree_direction(cfg, rng):
    """A random direction of every cell value and a divergence-free one of the
    face fields (the curl of a random edge potential A_z, periodic on periodic
    axes so that face n repeats face 0): constrained transport keeps div B,
    and a perturbation that breaks it can cross the limiter decisions that a
    divergence-free state puts exactly at zero in the ghost extrapolation."""
    nx, ny = cfg["n"][0], cfg["n"][1]
    d = {k: rng.standard_normal((1, ny, nx)) for k in ("rho", "mx", "my", "mz", "E", "b2")}
    A = rng.standard_normal((ny + 1, nx + 1))
    per = [b == "periodic" for b in cfg["bc"][::2]]
    if per[0]:
        A[:, nx] = A[:, 0]
    if per[1]:
        A[ny, :] = A[0, :]
    d["b0"] = (A[1:, :] - A[:-1, :])[None]
    d["b1"] = -(A[:, 1:] - A[:, :-1])[None]
    return d


def test_conserved_gradient_matches_central_differences():
    """Smooth 16^2 state with a non-uniform face field, 3 steps: <dJ/dU, d>
    against central differences of J along random directions of every cell
    value and divergence-free directions of the faces."""
    cfg, st, _ = W.smooth_2d(16, bpert=0.1)
    dts = frozen_dts(cfg, st, 3)
    J, g = oracle.grad_conserved(cfg, st, dts)
    rng = np.random.default_rng(13)
    for _ in range(3):
        d = divfree_direction(cfg, rng)
        dot = sum(np.sum(g[k] * d[k]) for k in g)
        # a limiter decision within h of switching changes one one-sided
        # difference only: the better side of each step size counts
        errs = []
        for h in (1e-6, 1e-7):
            jp = oracle.grad_conserved(cfg, {k: st[k] + h * d[k] for k in st}, dts)[0]
            jm = oracle.grad_conserved(cfg, {k: st[k] - h * d[k] for k in st}, dts)[0]
            errs += [abs((jp - J) / h - dot) / abs(dot), abs((J - jm) / h - dot) / abs(dot)]
        assert min(errs) <= 2e-5, errs


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_stage_gradient_matches_central_differences(bc):
    """One first RK stage: <grad, d> against central differences of J = <w, U*>
    along random directions.  The outflow case has a strong normal field, so
    the second ghost layer's recovered pressure is negative and raised to the
    floor (0), where J does not depend on it."""
    cfg = W.base_cfg(2, (9, 8), (0, 0), (0.9, 0.8), bc=bc)
    st = W.random_state(cfg, 71, v=0.3, bamp=0.3)
    rng = np.random.default_rng(17)
    w = {k: rng.standard_normal(v.shape) for k, v in st.items()}
    dt = 2e-3
    J, g = oracle.stage_vjp(cfg, st, dt, w)
    for _ in range(3):
        d = divfree_direction(cfg, rng)
        dot = sum(np.sum(g[k] * d[k]) for k in g)
        h = 1e-6
        jp = oracle.stage_vjp(cfg, {k: st[k] + h * d[k] for k in st}, dt, w)[0]
        jm = oracle.stage_vjp(cfg, {k: st[k] - h * d[k] for k in st}, dt, w)[0]
        assert abs((jp - jm) / (2 * h) - dot) <= 1e-7 * max(1.0, abs(dot))
