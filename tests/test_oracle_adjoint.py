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
