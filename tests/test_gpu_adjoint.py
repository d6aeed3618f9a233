"""GPU adjoint (reverse pass of the step, step sizes frozen) against the
oracle's reverse-mode (tape) gradient of the same functional, plus properties
that hold at any size: independence of the checkpoint interval, agreement
with central differences of the GPU's own forward run, and the autograd
wrapper."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import mhd
from paper_2511_20337_b300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS4 = ("rho", "vx", "vy", "vz")
CKEYS = ("rho", "mx", "my", "mz", "E")


def prims_of(cfg, st):
    bx, by, bz = W.cell_field(cfg, st["b0"], st["b1"], st["b2"])
    rho = st["rho"]
    v = [st["mx"] / rho, st["my"] / rho, st["mz"] / rho]
    g = cfg["gamma"]
    p = (g - 1) * (st["E"] - 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) - 0.5 * (bx ** 2 + by ** 2 + bz ** 2))
    return {"rho": rho, "vx": v[0], "vy": v[1], "vz": v[2], "p": p}, (st["b0"], st["b1"], st["b2"])


def misfit_target(cfg, st):
    keys = list(CKEYS) + (["b2"] if cfg["ndim"] == 2 else [])
    return [np.ascontiguousarray(np.roll(st[k], 2, axis=2) * 1.03) for k in keys]


CASES = {
    "2d-12-hlld-rk2": lambda: W.adjoint_2d(12),
    "2d-10x8-hll-rk3": lambda: (lambda c: (c, W.random_state(c, 61, v=0.2, bamp=0.2)))(
        W.base_cfg(2, (10, 8), (0, 0), (1.0, 0.8), riemann="hll", rk=3)),
    "2d-9x7-hlld-rk2-random": lambda: (lambda c: (c, W.random_state(c, 62, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (9, 7), (0, 0), (0.9, 0.7))),
    "3d-6x5x5-hlld-rk2": lambda: (lambda c: (c, W.random_state(c, 63, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (6, 5, 5), (0, 0, 0), (1.2, 1.0, 1.0))),
    "3d-5x6x5-hll-rk3": lambda: (lambda c: (c, W.random_state(c, 64, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (5, 6, 5), (0, 0, 0), (1.0, 1.2, 1.0), riemann="hll", rk=3)),
    # the five-cell reconstructions (at least 2G+1 = 7 cells per axis)
    "2d-12-wenoz-hlld-rk3": lambda: W.adjoint_2d(12, recon="wenoz", rk=3),
    "2d-9x8-wenoz-hll-rk2-random": lambda: (lambda c: (c, W.random_state(c, 65, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (9, 8), (0, 0), (0.9, 0.8), recon="wenoz", riemann="hll")),
    "2d-11x7-ppm-hlld-rk2-random": lambda: (lambda c: (c, W.random_state(c, 66, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (11, 7), (0, 0), (1.1, 0.7), recon="ppm")),
    "2d-10-ppm-hll-rk3": lambda: W.adjoint_2d(10, recon="ppm", riemann="hll", rk=3, seed=7),
    "3d-7x8x7-wenoz-hlld-rk2": lambda: (lambda c: (c, W.random_state(c, 67, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (7, 8, 7), (0, 0, 0), (1.0, 1.1, 1.0), recon="wenoz")),
    "3d-7x7x8-ppm-hlld-rk3": lambda: (lambda c: (c, W.random_state(c, 68, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (7, 7, 8), (0, 0, 0), (1.0, 1.0, 1.1), recon="ppm", rk=3)),
    # UCT-HLLD edge fields, and the paper's scheme (WENO-Z + HLLD + RK3 + UCT-HLLD)
    "2d-10x9-plm-hlld-rk2-ucthlld": lambda: (lambda c: (c, W.random_state(c, 69, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (10, 9), (0, 0), (1.0, 0.9), emf="uct_hlld")),
    "2d-12-wenoz-hlld-rk3-ucthlld": lambda: W.adjoint_2d(12, recon="wenoz", rk=3, emf="uct_hlld"),
    "3d-7x8x7-wenoz-hlld-rk3-ucthlld": lambda: (lambda c: (c, W.random_state(c, 70, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (7, 8, 7), (0, 0, 0), (1.0, 1.1, 1.0), recon="wenoz", rk=3, emf="uct_hlld")),
    # outflow axes: every axis, one axis, and the blast's scheme
    "2d-9x8-plm-hlld-rk2-outflow": lambda: (lambda c: (c, W.random_state(c, 71, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (9, 8), (0, 0), (0.9, 0.8), bc="outflow")),
    "2d-8x10-wenoz-hll-rk3-outflow-x": lambda: (lambda c: (c, W.random_state(c, 72, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (8, 10), (0, 0), (0.8, 1.0), recon="wenoz", riemann="hll", rk=3,
                   bc=["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"])),
    "2d-10x9-ppm-hlld-rk2-outflow-y-ucthlld": lambda: (lambda c: (c, W.random_state(c, 73, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (10, 9), (0, 0), (1.0, 0.9), recon="ppm", emf="uct_hlld",
                   bc=["periodic", "periodic", "outflow", "outflow", "periodic", "periodic"])),
    "3d-7x7x8-wenoz-hlld-rk3-outflow": lambda: (lambda c: (c, W.random_state(c, 74, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (7, 7, 8), (0, 0, 0), (1.0, 1.0, 1.1), recon="wenoz", rk=3, bc="outflow")),
    "3d-5x6x7-plm-hll-rk2-outflow-yz": lambda: (lambda c: (c, W.random_state(c, 75, v=0.2, bamp=0.2)))(
        W.base_cfg(3, (5, 6, 7), (0, 0, 0), (1.0, 1.2, 1.4), riemann="hll",
                   bc=["periodic", "periodic", "outflow", "outflow", "outflow", "outflow"])),
}


def oracle_dts(cfg, st, nsteps):
    return oracle.OracleSim(cfg, st).advance(nsteps, record_dt=True)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("which", ["magnetic_energy", "misfit"])
def test_gradient_matches_oracle_tape(case, which):
    """Gradient w.r.t. the initial rho and v (p, B held) and J after 5 steps of
    the oracle's frozen step sizes, checkpoints every 2 steps."""
    cfg, st = CASES[case]()
    nsteps = 5
    dts = oracle_dts(cfg, st, nsteps)
    prim, B = prims_of(cfg, st)
    target = misfit_target(cfg, st) if which == "misfit" else None
    J0, g0 = oracle.grad_prim(cfg, prim, B, dts, which, target)
    sim = mhd.Sim(cfg, st)
    J, used = sim.adjoint(nsteps, dts, ckpt_every=2, functional=which, target=target)
    g = sim.grad_prim()
    assert np.array_equal(used, dts)
    assert abs(J - J0) <= 1e-12 * abs(J0)
    scale = max(np.max(np.abs(g0[k])) for k in KEYS4)
    for k in KEYS4:
        err = np.max(np.abs(g[k] - g0[k]))
        assert err <= 1e-10 * scale, (k, err, scale)


@pytest.mark.parametrize("recon", ["plm", "wenoz", "ppm"])
def test_checkpoint_interval_does_not_change_the_gradient(recon):
    """Recomputation from checkpoints reproduces the forward bit for bit, so
    any interval gives the same gradient, bitwise."""
    cfg, st = W.adjoint_2d(16, recon=recon)
    nsteps = 7
    grads = []
    for k in (1, 3, 7, 100):
        sim = mhd.Sim(cfg, st)
        J, dts = sim.adjoint(nsteps, None, ckpt_every=k)
        grads.append((J, dts, sim.grad_conserved(), sim.grad_prim()))
    for J, dts, gc, gp in grads[1:]:
        assert J == grads[0][0]
        assert np.array_equal(dts, grads[0][1])
        for key in mhd.KEYS:
            assert np.array_equal(gc[key], grads[0][2][key]), key
        for key in KEYS4:
            assert np.array_equal(gp[key], grads[0][3][key]), key


def test_cfl_steps_are_recorded_and_the_state_advances():
    """With dts=None the forward takes its own CFL steps; they are returned,
    the context ends at the final state of those steps, and its time is their
    sum."""
    cfg, st = W.adjoint_2d(16)
    nsteps = 6
    sim = mhd.Sim(cfg, st)
    J, dts = sim.adjoint(nsteps, None, ckpt_every=4)
    ref = mhd.Sim(cfg, st)
    ref_dts = []
    for _ in range(nsteps):
        ref_dts.append(ref.cfl_dt())
        ref.step(ref_dts[-1])
    assert np.array_equal(dts, np.array(ref_dts))
    a, b = sim.get_conserved(), ref.get_conserved()
    for k in mhd.KEYS:
        assert np.array_equal(a[k], b[k]), k
    assert sim.time == pytest.approx(sum(ref_dts), rel=1e-15)
    bx, by, bz = W.cell_field(cfg, b["b0"], b["b1"], b["b2"])
    dV = (1.0 / 16) ** 2
    assert J == pytest.approx(0.5 * dV * np.sum(bx ** 2 + by ** 2 + bz ** 2), rel=1e-13)


def _gpu_J(cfg, st, dts, which="magnetic_energy", target=None):
    sim = mhd.Sim(cfg, st)
    J, _ = sim.adjoint(len(dts), dts, ckpt_every=len(dts), functional=which, target=target)
    return J


@pytest.mark.parametrize("recon", ["plm", "wenoz"])
def test_conserved_gradient_matches_central_differences(recon):
    """<dJ/dU0, d> against (J(U0 + h d) - J(U0 - h d)) / 2h of the GPU forward,
    along smooth directions d of every conserved cell variable and face field
    (face perturbations from a potential, so div B stays zero).  The initial
    face field is non-uniform: on a uniform one the edge reconstruction sits
    at minmod(0, 0), where J is only directionally differentiable in B.
    WENO-Z's weights are smooth functions of the window, so its gradient
    meets the same bound."""
    cfg, st, _ = W.smooth_2d(32, bpert=0.1)
    cfg = dict(cfg, recon=recon)
    nsteps = 8
    sim = mhd.Sim(cfg, st)
    _, dts = sim.adjoint(nsteps, None, ckpt_every=3)
    g = sim.grad_conserved()
    X, Y, _ = W.cell_centres(cfg)
    tp = 2 * np.pi
    rng = np.random.default_rng(21)
    for trial in range(3):
        ph = rng.uniform(0, tp, 8)
        d = {"rho": 0.1 * np.sin(tp * X + ph[0]) * np.cos(tp * Y + ph[1]),
             "mx": 0.05 * np.cos(tp * (X + Y) + ph[2]), "my": 0.05 * np.sin(tp * (X - 2 * Y) + ph[3]),
             "mz": 0.02 * np.sin(tp * Y + ph[4]), "E": 0.1 * np.cos(tp * (2 * X + Y) + ph[5]),
             "b2": 0.02 * np.cos(tp * X + ph[6])}
        # face perturbation from an edge potential A_z (periodic): bx = dA/dy, by = -dA/dx
        n = 32
        xe = np.arange(n + 1) / n
        Az = 0.01 * np.sin(tp * xe[None, :] + ph[7])[None] * np.cos(tp * xe[:, None])[None]
        d["b0"] = (Az[:, 1:, :] - Az[:, :-1, :]) * n
        d["b1"] = -(Az[:, :, 1:] - Az[:, :, :-1]) * n
        d["b0"][:, :, -1] = d["b0"][:, :, 0]
        d["b1"][:, -1, :] = d["b1"][:, 0, :]
        dot = sum(np.sum(g[k] * d[k]) for k in mhd.KEYS)
        errs = []
        for h in (1e-5, 1e-6):
            sp = {k: st[k] + h * d[k] for k in mhd.KEYS}
            sm = {k: st[k] - h * d[k] for k in mhd.KEYS}
            fd = (_gpu_J(cfg, sp, dts) - _gpu_J(cfg, sm, dts)) / (2 * h)
            errs.append(abs(fd - dot) / abs(dot))
        assert min(errs) <= 1e-5, (trial, errs)


def test_autograd_function_gives_the_library_gradient():
    torch = pytest.importorskip("torch")
    cfg, st = W.adjoint_2d(16)
    prim, B = prims_of(cfg, st)
    dev = torch.device("cuda:0")
    t = {k: torch.tensor(prim[k], dtype=torch.float64, device=dev) for k in ("rho", "vx", "vy", "vz", "p")}
    Bt = [torch.tensor(b, dtype=torch.float64, device=dev) for b in B]
    leaves = {k: t[k].clone().requires_grad_(True) for k in KEYS4}
    J = mhd.final_functional(cfg, leaves["rho"], leaves["vx"], leaves["vy"], leaves["vz"], t["p"], Bt, 6,
                             ckpt_every=4)
    (3.0 * J).backward()
    sim = mhd.Sim(cfg)
    sim.set_prim(prim["rho"], [prim["vx"], prim["vy"], prim["vz"]], prim["p"], list(B))
    J2, _ = sim.adjoint(6, None, ckpt_every=4)
    g = sim.grad_prim()
    assert float(J.detach()) == J2
    for k in KEYS4:
        assert np.array_equal(leaves[k].grad.cpu().numpy(), 3.0 * g[k]), k


def test_unsupported_schemes_are_rejected():
    cfg, st = W.adjoint_2d(12)
    gcfg, gst = W.to_glm(cfg, st)
    sim = mhd.Sim(gcfg, gst)
    with pytest.raises(mhd.MhdError) as e:
        sim.adjoint(2, None)
    assert e.value.code == -1
    # fewer than 2G + 1 cells on an axis: 4 for PLM, 6 for WENO-Z (G = 3)
    for small_cfg, small_st in (W.adjoint_2d(4), W.adjoint_2d(6, recon="wenoz"),
                                W.adjoint_2d(4, bc="outflow")):
        sim = mhd.Sim(small_cfg, small_st)
        with pytest.raises(mhd.MhdError):
            sim.adjoint(2, None)
    sim = mhd.Sim(cfg, st)
    with pytest.raises(mhd.MhdError) as e:
        sim.grad_prim()
    assert e.value.code == -6


# Cases for the full conserved gradient and the stage transposes: every
# reconstruction, both solvers, both edge-field forms, periodic / outflow /
# mixed axes.  The outflow cases with a strong normal field put a negative
# recovered pressure in the second ghost layer, which the forward raises to
# the floor (0): the stage transpose must pass no pressure cotangent there.
O, P = "outflow", "periodic"


def off_divfree(cfg, st, seed):
    """The state with 1e-3 random noise on the face fields (face n of a
    periodic axis kept equal to face 0).  A divergence-free field puts some
    limiter arguments of the outflow ghost extrapolation exactly at zero,
    where J has kinks and the GPU and the oracle, rounding differently, may
    take different one-sided derivatives; off the divergence-free set the
    derivative is unique."""
    rng = np.random.default_rng(seed)
    out = {k: v.copy() for k, v in st.items()}
    for d, k in enumerate(("b0", "b1", "b2")):
        if d >= cfg["ndim"]:
            continue
        out[k] = out[k] + 1e-3 * rng.standard_normal(out[k].shape)
        if cfg["bc"][2 * d] == P:
            first = [slice(None)] * 3
            last = [slice(None)] * 3
            first[2 - d], last[2 - d] = 0, -1
            out[k][tuple(last)] = out[k][tuple(first)]
    return out


FULL_CASES = {
    "2d-9x8-plm-hlld-rk2-outflow-y-strong-bn": lambda: (lambda c: (c, W.random_state(c, 71, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (9, 8), (0, 0), (0.9, 0.8), bc=[P, P, O, O, P, P])),
    "2d-9x8-plm-hll-rk3-outflow": lambda: (lambda c: (c, W.random_state(c, 75, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (9, 8), (0, 0), (0.9, 0.8), riemann="hll", rk=3, bc=O)),
    "2d-10x9-wenoz-hlld-rk2-outflow-x-ucthlld": lambda: (lambda c: (c, W.random_state(c, 74, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (10, 9), (0, 0), (1.0, 0.9), recon="wenoz", emf="uct_hlld", bc=[O, O, P, P, P, P])),
    "2d-11x7-ppm-hlld-rk3-periodic": lambda: (lambda c: (c, W.random_state(c, 66, v=0.3, bamp=0.3)))(
        W.base_cfg(2, (11, 7), (0, 0), (1.1, 0.7), recon="ppm", rk=3)),
    "3d-7x7x8-wenoz-hlld-rk2-outflow-z": lambda: (lambda c: (c, W.random_state(c, 76, v=0.2, bamp=0.3)))(
        W.base_cfg(3, (7, 7, 8), (0, 0, 0), (1.0, 1.0, 1.1), recon="wenoz", bc=[P, P, P, P, O, O])),
    "3d-5x6x5-plm-hll-rk3-outflow": lambda: (lambda c: (c, W.random_state(c, 77, v=0.2, bamp=0.3)))(
        W.base_cfg(3, (5, 6, 5), (0, 0, 0), (1.0, 1.2, 1.0), riemann="hll", rk=3, bc=O)),
}


@pytest.mark.parametrize("case", list(FULL_CASES))
def test_conserved_gradient_matches_oracle_tape(case):
    """dJ/dU^0 with respect to every cell value and face field (the gradient
    with respect to rho and v with p held fixed does not see errors along the
    pressure), against the oracle's tape with every state element a variable."""
    cfg, st = FULL_CASES[case]()
    st = off_divfree(cfg, st, 8)
    nsteps = 3
    dts = oracle_dts(cfg, st, nsteps)
    J0, g0 = oracle.grad_conserved(cfg, st, dts)
    sim = mhd.Sim(cfg, st)
    J, _ = sim.adjoint(nsteps, dts, ckpt_every=2)
    g = sim.grad_conserved()
    assert abs(J - J0) <= 1e-12 * abs(J0)
    scale = max(np.max(np.abs(g0[k])) for k in g0)
    for k in g0:
        err = np.max(np.abs(g[k] - g0[k]))
        assert err <= 1e-10 * scale, (k, err, scale)


@pytest.mark.parametrize("case", list(FULL_CASES))
def test_stage_transpose_matches_oracle(case):
    """One first RK stage and its transpose on the GPU (mhd_probe_stage_vjp)
    against the oracle's tape of the same stage, for a random cotangent."""
    cfg, st = FULL_CASES[case]()
    st = off_divfree(cfg, st, 9)
    rng = np.random.default_rng(3)
    w = {k: rng.standard_normal(v.shape) for k, v in st.items()}
    dt = 0.5 * oracle.OracleSim(cfg, st).cfl_dt()
    _, g0 = oracle.stage_vjp(cfg, st, dt, w)
    sim = mhd.Sim(cfg, st)
    g = mhd.probe_stage_vjp(sim, st, dt, w)
    scale = max(np.max(np.abs(g0[k])) for k in g0)
    for k in g0:
        err = np.max(np.abs(g[k] - g0[k]))
        assert err <= 1e-12 * scale, (k, err, scale)


@pytest.mark.parametrize("bc", [P, O, [O, O, P, P, P, P], [P, P, O, O, P, P], [O, O, P, P, O, O]])
@pytest.mark.parametrize("recon", ["plm", "wenoz"])
def test_ghost_fill_transpose_is_its_adjoint(bc, recon):
    """<fill(x), a> = <x, fill^T(a)> on random whole padded fields: the ghost
    transposes (one shell gather, or the per-axis periodic, copy and
    normal-field passes backwards) are the exact transpose of the ghost fill."""
    nd = 3 if isinstance(bc, list) and bc[4] == O else 2
    n = (7, 8, 7) if nd == 3 else (9, 8)  # periodic axes need 2G + 1 = 7 cells (one image per cell)
    cfg = W.base_cfg(nd, n, (0,) * nd, (1,) * nd, recon=recon, bc=bc)
    sim = mhd.Sim(cfg, W.random_state(cfg, 3))
    G = 3 if recon == "wenoz" else 2
    E = int(np.prod([m + 2 * G + 1 for m in n]))
    rng = np.random.default_rng(5)
    x, a = rng.standard_normal((8, E)), rng.standard_normal((8, E))
    fx, xb = mhd.probe_ghost_vjp(sim, x, a)
    lhs, rhs = float(np.sum(fx * a)), float(np.sum(x * xb))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), float(np.sum(np.abs(fx * a))))
