"""Oracle pins, whole scheme: conservation, discrete div B, invariance of
uniform states, rotation / mirror symmetry, the CFL formula's closed form,
the UCT field's closed forms, the Sod exact solution in the hydro limit and
convergence orders on linear and circularly polarised Alfven waves (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W
from conftest import relerr

KEYS = oracle.KEYS


def div_b(cfg, st):
    nd = cfg["ndim"]
    n = cfg["n"]
    dx = [(cfg["x1"][d] - cfg["x0"][d]) / n[d] for d in range(nd)]
    b0, b1 = st["b0"], st["b1"]
    div = (b0[..., 1:] - b0[..., :-1]) / dx[0] + (b1[:, 1:, :] - b1[:, :-1, :]) / dx[1]
    if nd == 3:
        div = div + (st["b2"][1:] - st["b2"][:-1]) / dx[2]
    bmax = max(np.abs(b0).max(), np.abs(b1).max(), np.abs(st["b2"]).max())
    return np.abs(div).max(), bmax / min(dx)


def totals(cfg, st):
    out = {}
    for k in ("rho", "mx", "my", "mz", "E"):
        out[k] = (st[k].sum(), np.abs(st[k]).sum())
    if cfg["ndim"] == 2:
        out["bz"] = (st["b2"].sum(), np.abs(st["b2"]).sum())
    # periodic faces: drop the duplicate last face
    out["bx"] = (st["b0"][..., :-1].sum(), np.abs(st["b0"][..., :-1]).sum())
    out["by"] = (st["b1"][:, :-1, :].sum(), np.abs(st["b1"][:, :-1, :]).sum())
    if cfg["ndim"] == 3:
        out["bzf"] = (st["b2"][:-1].sum(), np.abs(st["b2"][:-1]).sum())
    return out


CASES = {
    "ot2d-plm-hlld-rk2": lambda: W.orszag_tang_2d(32),
    "rand2d-wenoz-hll-rk3": lambda: (lambda c: (c, W.random_state(c, 3)))(
        W.base_cfg(2, (12, 10), (0, 0), (1.2, 1.0), recon="wenoz", riemann="hll", rk=3)),
    "rand3d-plm-hlld-rk2": lambda: (lambda c: (c, W.random_state(c, 4)))(
        W.base_cfg(3, (6, 7, 5), (0, 0, 0), (1.2, 1.4, 1.0))),
    "rand3d-ppm-hlld-rk3": lambda: (lambda c: (c, W.random_state(c, 5)))(
        W.base_cfg(3, (6, 6, 6), (0, 0, 0), (1, 1, 1), recon="ppm", rk=3)),
    "turb3d-plm-hlld-rk2": lambda: W.turbulent_3d(12, seed=9),
}


@pytest.mark.parametrize("case", list(CASES))
def test_conservation_on_periodic_grids(case):
    """Eq. FV in flux form and CT conserve the totals of rho, m, E and every
    field component to round-off on a periodic grid."""
    cfg, st = CASES[case]()
    s = oracle.OracleSim(cfg, st)
    s.advance(4)
    out = s.get_state()
    t0, t1 = totals(cfg, st), totals(cfg, out)
    for k in t0:
        assert abs(t1[k][0] - t0[k][0]) <= 1e-13 * max(t0[k][1], t1[k][1], 1e-300), k


@pytest.mark.parametrize("case", list(CASES))
def test_div_b_stays_at_roundoff(case):
    cfg, st = CASES[case]()
    s = oracle.OracleSim(cfg, st)
    s.advance(4)
    div, scale = div_b(cfg, s.get_state())
    assert div <= 1e-12 * scale


def test_div_b_blast_outflow():
    cfg, st = W.blast_3d(10)
    s = oracle.OracleSim(cfg, st)
    s.advance(3)
    div, scale = div_b(cfg, s.get_state())
    assert div <= 1e-12 * scale


@pytest.mark.parametrize("ndim,recon,rk,bc", [(2, "plm", 2, "periodic"), (2, "wenoz", 3, "outflow"),
                                              (3, "ppm", 3, "outflow"), (3, "plm", 2, "periodic")])
def test_uniform_state_is_steady_bitwise(ndim, recon, rk, bc):
    n = (7, 5) if ndim == 2 else (5, 4, 6)
    cfg = W.base_cfg(ndim, n, (0,) * ndim, (1,) * ndim, recon=recon, rk=rk, bc=bc)
    shape = (n[2] if ndim == 3 else 1, n[1], n[0])
    one = np.ones(shape)
    bx, by, bz = W.uniform_faces(cfg, (0.3, -0.7, 0.45))
    st = W.assemble(cfg, 1.3 * one, 0.2 * one, -0.1 * one, 0.35 * one, 0.8 * one, bx, by, bz)
    s = oracle.OracleSim(cfg, st)
    s.advance(3)
    out = s.get_state()
    for k in KEYS:
        # spatially uniform, bitwise
        assert np.all(out[k] == out[k].flat[0]), k
        if rk == 2:
            # SSP-RK2 combines a constant exactly: (a + a) / 2 = a
            np.testing.assert_array_equal(out[k], st[k], err_msg=k)
        else:
            # the 3/4, 1/4 and 1/3, 2/3 combines of Eq. RK3 round a constant
            np.testing.assert_allclose(out[k], st[k], rtol=4e-16, atol=0, err_msg=k)


def test_uniform_state_emf_is_minus_v_cross_b():
    """Every UCT edge field of a uniform state equals -(v x B) (a+ + a- = 1)."""
    cfg = W.base_cfg(3, (4, 5, 6), (0, 0, 0), (1, 1, 1))
    shape = (6, 5, 4)
    one = np.ones(shape)
    v = np.array([0.2, -0.1, 0.35])
    B = np.array([0.3, -0.7, 0.45])
    bx, by, bz = W.uniform_faces(cfg, B)
    st = W.assemble(cfg, 1.3 * one, *(c * one for c in v), 0.8 * one, bx, by, bz)
    s = oracle.OracleSim(cfg, st)
    s.stage_increment(1e-3)
    E = -np.cross(v, B)
    for c in range(3):
        np.testing.assert_allclose(s.emf(c), E[c], rtol=1e-14, atol=1e-16)


def minmod(a, b):
    return np.where(a * b > 0, np.where(np.abs(b) < np.abs(a), b, a), 0.0)


def test_emf_one_dimensional_reduction():
    """For 2D data uniform in y, E_z at every vertex equals the HLL-upwinded
    -u B_y of the x-face plus the centred v_y B_x:
    E_z = -(a+ u_L By_L + a- u_R By_R) + d (By_R - By_L) + vbar_y Bx."""
    nx, ny = 12, 4
    cfg = W.base_cfg(2, (nx, ny), (0, 0), (1.0, 0.5))
    rng = np.random.default_rng(11)
    row = lambda lo, hi: np.tile(rng.uniform(lo, hi, nx), (ny, 1))[None]  # noqa: E731
    rho, vx, vy, vz, p = row(0.5, 1.5), row(-0.4, 0.4), row(-0.4, 0.4), row(-0.4, 0.4), row(0.5, 1.5)
    bxval = 0.6
    byrow = rng.uniform(-0.5, 0.5, nx)
    bx = np.full((1, ny, nx + 1), bxval)
    by = np.tile(byrow, (ny + 1, 1))[None]
    bz = row(-0.5, 0.5)
    st = W.assemble(cfg, rho, vx, vy, vz, p, bx, by, bz)
    s = oracle.OracleSim(cfg, st)
    s.stage_increment(1e-3)
    Ez = s.emf(2)[0]   # [ny+1][nx+1]
    # expected, from primitive rows (periodic in x)
    g = cfg["gamma"]
    V = {"rho": rho[0, 0], "u": vx[0, 0], "v": vy[0, 0], "w": vz[0, 0], "by": byrow, "bz": bz[0, 0], "p": p[0, 0]}
    P = lambda a, s_: np.roll(a, -s_)  # noqa: E731  value at i+s_
    plus, minus = {}, {}
    for k, a in V.items():
        d = minmod(a - P(a, -1), P(a, 1) - a)
        plus[k], minus[k] = a + 0.5 * d, a - 0.5 * d
    for i in range(nx + 1):
        L = {k: plus[k][(i - 1) % nx] for k in V}
        R = {k: minus[k][i % nx] for k in V}
        wl = [L["rho"], L["u"], L["v"], L["w"], L["by"], L["bz"], L["p"]]
        wr = [R["rho"], R["u"], R["v"], R["w"], R["by"], R["bz"], R["p"]]
        _, ing = oracle.riemann("hlld", wl, wr, bxval, g)
        ap, am, dd = ing[0], ing[1], ing[2]
        vbar = 0.5 * (vy[0, 0][(i - 1) % nx] + vy[0, 0][i % nx])
        expect = -(ap * L["u"] * L["by"] + am * R["u"] * R["by"]) + dd * (R["by"] - L["by"]) + vbar * bxval
        np.testing.assert_allclose(Ez[:, i], expect, rtol=1e-13, atol=1e-14)


def test_cfl_dt_closed_form_for_gas_at_rest():
    """No flow and no field: dt = C / (c_s sum_d 1/dx_d)."""
    for nd, n, L in [(2, (8, 6), (2.0, 1.5)), (3, (4, 6, 5), (1.0, 2.0, 0.5))]:
        cfg = W.base_cfg(nd, n, (0,) * nd, L, cfl=0.37)
        shape = (n[2] if nd == 3 else 1, n[1], n[0])
        one = np.ones(shape)
        bx, by, bz = W.uniform_faces(cfg, (0.0, 0.0, 0.0))
        rho, p = 1.7, 0.6
        st = W.assemble(cfg, rho * one, 0 * one, 0 * one, 0 * one, p * one, bx, by, bz)
        dt = oracle.OracleSim(cfg, st).cfl_dt()
        cs = math.sqrt(cfg["gamma"] * p / rho)
        expect = 0.37 / (cs * sum(n[d] / L[d] for d in range(nd)))
        assert dt == pytest.approx(expect, rel=1e-14)


def test_cfl_dt_uses_fastest_direction_sum():
    """Random state: dt equals C over the max over cells of the per-direction sum
    of |v_d| + cf_d over dx_d, evaluated from the fast-speed closed form."""
    cfg = W.base_cfg(3, (5, 4, 3), (0, 0, 0), (1.0, 0.8, 0.6), cfl=0.4)
    st = W.random_state(cfg, 21)
    dt = oracle.OracleSim(cfg, st).cfl_dt()
    bx, by, bz = W.cell_field(cfg, st["b0"], st["b1"], st["b2"])
    rho = st["rho"]
    v = [st["mx"] / rho, st["my"] / rho, st["mz"] / rho]
    g = cfg["gamma"]
    B2 = bx ** 2 + by ** 2 + bz ** 2
    p = (g - 1) * (st["E"] - 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) - 0.5 * B2)
    lam = 0.0
    for d, bd in enumerate((bx, by, bz)):
        a2 = g * p / rho
        b2 = B2 / rho
        cf = np.sqrt(0.5 * (a2 + b2 + np.sqrt((a2 + b2) ** 2 - 4 * a2 * bd ** 2 / rho)))
        lam = lam + (np.abs(v[d]) + cf) / (0.2 if d == 0 else 0.2)
    assert dt == pytest.approx(0.4 / lam.max(), rel=1e-13)


# ---- symmetry ----

def rot90_2d(st):
    """Rotate a square periodic 2D state by +90 degrees: (x, y) -> (-y, x),
    vectors v' = (-v_y, v_x), B' = (-B_y, B_x)."""
    n = st["rho"].shape[-1]
    s = lambda a: a[0, ::-1, :].T[None]  # noqa: E731  A'[y', x'] = A[n-1-x', y']
    out = {"rho": s(st["rho"]), "mx": -s(st["my"]), "my": s(st["mx"]), "mz": s(st["mz"]), "E": s(st["E"]),
           "b2": s(st["b2"])}
    b0, b1 = st["b0"][0], st["b1"][0]
    ip = np.arange(n + 1)
    jp = np.arange(n)
    # Bx'(face i', row j') = -By(y-face (n - i') mod n, column j')
    out["b0"] = -b1[np.ix_((n - ip) % n, jp)].T[None]
    # By'(column i', y-face j') = Bx(x-face j', row n-1-i')
    out["b1"] = b0[np.ix_(n - 1 - jp, ip)].T[None]
    return out


def rotz90_3d(st):
    """Rotate a 3D state with square x-y section by +90 degrees about z."""
    n = st["rho"].shape[-1]
    s = lambda a: np.transpose(a[:, ::-1, :], (0, 2, 1))  # noqa: E731
    out = {"rho": s(st["rho"]), "mx": -s(st["my"]), "my": s(st["mx"]), "mz": s(st["mz"]), "E": s(st["E"]),
           "b2": s(st["b2"])}
    ip = np.arange(n + 1)
    jp = np.arange(n)
    b0, b1 = st["b0"], st["b1"]
    out["b0"] = -np.transpose(b1[:, (n - ip) % n, :][:, :, jp], (0, 2, 1))
    out["b1"] = np.transpose(b0[:, n - 1 - jp, :][:, :, ip], (0, 2, 1))
    return out


def mirror_x(st, ndim):
    """x -> -x with (v_x, B_x) -> -(v_x, B_x)."""
    f = lambda a: a[..., ::-1]  # noqa: E731
    out = {k: f(st[k]) for k in ("rho", "my", "mz", "E", "b1")}
    out["mx"] = -f(st["mx"])
    out["b0"] = -f(st["b0"])
    out["b2"] = f(st["b2"])
    return out


def _norm_periodic(st):
    """Copy the first face into the duplicate last face on periodic axes."""
    st = {k: np.array(v) for k, v in st.items()}
    st["b0"][..., -1] = st["b0"][..., 0]
    st["b1"][:, -1, :] = st["b1"][:, 0, :]
    if st["b2"].shape[0] > st["rho"].shape[0]:
        st["b2"][-1] = st["b2"][0]
    return st


def _advance(cfg, st, steps, dt):
    s = oracle.OracleSim(cfg, st)
    for _ in range(steps):
        s.step(dt)
    return s.get_state()


@pytest.mark.parametrize("recon,riemann,rk", [("plm", "hlld", 2), ("wenoz", "hlld", 3), ("ppm", "hll", 2)])
def test_rotation_commutes_with_step_2d(recon, riemann, rk):
    cfg = W.base_cfg(2, (8, 8), (0, 0), (1, 1), recon=recon, riemann=riemann, rk=rk)
    st = _norm_periodic(W.random_state(cfg, 31))
    dt = 0.2 * oracle.OracleSim(cfg, st).cfl_dt()
    a = rot90_2d(_advance(cfg, st, 2, dt))
    b = _advance(cfg, rot90_2d(st), 2, dt)
    for k in KEYS:
        assert relerr(b[k], a[k]) < 1e-13, k


@pytest.mark.parametrize("recon", ["plm", "wenoz"])
def test_rotation_commutes_with_step_3d(recon):
    cfg = W.base_cfg(3, (6, 6, 5), (0, 0, 0), (1, 1, 0.8), recon=recon, rk=3 if recon == "wenoz" else 2)
    st = _norm_periodic(W.random_state(cfg, 32))
    dt = 0.2 * oracle.OracleSim(cfg, st).cfl_dt()
    a = rotz90_3d(_advance(cfg, st, 2, dt))
    b = _advance(cfg, rotz90_3d(st), 2, dt)
    for k in KEYS:
        assert relerr(b[k], a[k]) < 1e-13, k


@pytest.mark.parametrize("ndim", [2, 3])
def test_mirror_commutes_with_step(ndim):
    n = (8, 7) if ndim == 2 else (6, 5, 4)
    cfg = W.base_cfg(ndim, n, (0,) * ndim, (1,) * ndim, rk=3, recon="wenoz")
    st = _norm_periodic(W.random_state(cfg, 33))
    dt = 0.2 * oracle.OracleSim(cfg, st).cfl_dt()
    a = mirror_x(_advance(cfg, st, 2, dt), ndim)
    b = _advance(cfg, mirror_x(st, ndim), 2, dt)
    for k in KEYS:
        assert relerr(b[k], a[k]) < 1e-13, k


def test_orszag_tang_keeps_point_symmetry():
    """The 2D OT state is invariant under (x, y) -> (-x, -y), v -> -v, B -> -B;
    the discrete solution must keep that symmetry."""
    cfg, st = W.orszag_tang_2d(32)
    s = oracle.OracleSim(cfg, st)
    s.advance(20)
    out = s.get_state()
    r = lambda a: np.roll(a[0, ::-1, ::-1], 1, axis=(0, 1))  # noqa: E731  cell (i,j) -> (-i-1,-j-1) = (n-1-i, n-1-j)
    for k, sg in (("rho", 1), ("E", 1), ("mx", -1), ("my", -1)):
        a = out[k][0]
        assert relerr(sg * a[::-1, ::-1], a) < 1e-12, k


# ---- exact solutions ----

def sod_exact(x, t, gamma=1.4, x0=0.5, L=(1.0, 0.0, 1.0), R=(0.125, 0.0, 0.1)):
    """Exact Riemann solution of the Euler equations (Toro, ch. 4): Newton
    iteration for p*, then sampling of the wave pattern."""
    rl, ul, pl = L
    rr, ur, pr = R
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)

    def fk(p, rk, pk, ck):
        if p > pk:
            A, B = 2 / ((gamma + 1) * rk), (gamma - 1) / (gamma + 1) * pk
            f = (p - pk) * math.sqrt(A / (p + B))
            df = math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        else:
            f = 2 * ck / (gamma - 1) * ((p / pk) ** ((gamma - 1) / (2 * gamma)) - 1)
            df = 1 / (rk * ck) * (p / pk) ** (-(gamma + 1) / (2 * gamma))
        return f, df

    p = 0.5 * (pl + pr)
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, cl)
        f2, d2 = fk(p, rr, pr, cr)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    f1, _ = fk(p, rl, pl, cl)
    f2, _ = fk(p, rr, pr, cr)
    us = 0.5 * (ul + ur) + 0.5 * (f2 - f1)
    out = np.zeros_like(x)
    g = gamma
    for n_, xi in enumerate((x - x0) / t):
        if xi <= us:  # left of contact
            if p > pl:
                S = ul - cl * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                out[n_] = rl if xi < S else rl * ((p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1))
            else:
                cs = cl * (p / pl) ** ((g - 1) / (2 * g))
                if xi < ul - cl:
                    out[n_] = rl
                elif xi > us - cs:
                    out[n_] = rl * (p / pl) ** (1 / g)
                else:
                    out[n_] = rl * (2 / (g + 1) + (g - 1) / ((g + 1) * cl) * (ul - xi)) ** (2 / (g - 1))
        else:
            if p > pr:
                S = ur + cr * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
                out[n_] = rr if xi > S else rr * ((p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1))
            else:
                cs = cr * (p / pr) ** ((g - 1) / (2 * g))
                if xi > ur + cr:
                    out[n_] = rr
                elif xi < us + cs:
                    out[n_] = rr * (p / pr) ** (1 / g)
                else:
                    out[n_] = rr * (2 / (g + 1) - (g - 1) / ((g + 1) * cr) * (ur - xi)) ** (2 / (g - 1))
    return out


def run_sod(nx, solver, recon="plm", rk=2, t_end=0.2):
    cfg = W.base_cfg(2, (nx, 4), (0, 0), (1.0, 4.0 / nx), gamma=1.4, riemann=solver, recon=recon, rk=rk,
                     bc=["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"])
    X, _, _ = W.cell_centres(cfg)
    left = X < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(X)
    bx, by, bz = W.uniform_faces(cfg, (0.0, 0.0, 0.0))
    s = oracle.OracleSim(cfg, W.assemble(cfg, rho, z, z, z, p, bx, by, bz))
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(s.cfl_dt(), t_end - t)
        s.step(dt)
        t += dt
    out = s.get_state()
    xc = X[0, 0]
    return np.mean(np.abs(out["rho"][0, 0] - sod_exact(xc, t_end))), out


@pytest.mark.parametrize("solver", ["hlld", "hll"])
def test_sod_hydro_limit_converges_to_exact_solution(solver):
    e1, out = run_sod(100, solver)
    e2, _ = run_sod(200, solver)
    assert e1 < 0.02 and e2 < 0.011
    assert e1 / e2 > 1.5            # about first order at discontinuities
    # y-rows identical, no spurious field
    assert np.all(out["rho"][0] == out["rho"][0, :1])
    assert np.all(out["b0"] == 0.0) and np.all(out["b1"] == 0.0) and np.all(out["b2"] == 0.0)


def test_hlld_less_diffusive_than_hll_on_contact():
    e_d, _ = run_sod(100, "hlld")
    e_h, _ = run_sod(100, "hll")
    assert e_d < e_h


def linear_mhd_matrix(rho, u, bx, by, bz, p, gamma):
    """Primitive-variable Jacobian of 1D ideal MHD, W = (rho, u, v, w, By, Bz, p)."""
    A = np.zeros((7, 7))
    A[0] = [u, rho, 0, 0, 0, 0, 0]
    A[1] = [0, u, 0, 0, by / rho, bz / rho, 1 / rho]
    A[2] = [0, 0, u, 0, -bx / rho, 0, 0]
    A[3] = [0, 0, 0, u, 0, -bx / rho, 0]
    A[4] = [0, by, -bx, 0, u, 0, 0]
    A[5] = [0, bz, 0, -bx, 0, u, 0]
    A[6] = [0, gamma * p, 0, 0, 0, 0, u]
    return A


def wave_state_2d(n, wave, amp, t=0.0, recon="plm", rk=2):
    """Oblique small-amplitude wave along k = 2 pi (1, 1) on the unit square.
    Background (frame e1 = k/|k|, e2 in-plane, e3 = z): rho = 1, p = 1/G,
    B = (1, sqrt 2, 1/2).  The eigenvector comes from numpy's eigendecomposition
    of the linearised Jacobian; wave in {'fast', 'alfven', 'slow'} (right-going)."""
    g = 5.0 / 3.0
    rho0, p0 = 1.0, 1.0 / g
    B1, B2, B3 = 1.0, math.sqrt(2.0), 0.5
    A = linear_mhd_matrix(rho0, 0.0, B1, B2, B3, p0, g)
    lam, R = np.linalg.eig(A)
    lam, R = lam.real, R.real
    order = np.argsort(lam)[::-1]   # fast+, alfven+, slow+, entropy, ...
    idx = {"fast": order[0], "alfven": order[1], "slow": order[2]}[wave]
    r = R[:, idx] / np.max(np.abs(R[:, idx]))
    speed = lam[idx]
    cfg = W.base_cfg(2, (n, n), (0, 0), (1, 1), recon=recon, rk=rk)
    kv = 2 * math.pi * np.array([1.0, 1.0])
    kmag = np.linalg.norm(kv)
    e1 = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    e3 = np.array([0.0, 0.0, 1.0])
    e2 = np.cross(e3, e1)
    X, Y, _ = W.cell_centres(cfg)
    ph = kv[0] * X + kv[1] * Y - kmag * speed * t
    c = amp * np.cos(ph)
    rho = rho0 + c * r[0]
    vel = [c * (r[1] * e1[d] + r[2] * e2[d] + r[3] * e3[d]) for d in range(3)]
    p = p0 + c * r[6]
    # field: uniform background + wave part (r4 e2 + r5 e3) amp cos(phi)
    bu = B1 * e1 + B2 * e2 + B3 * e3
    ux, uy, _ = W.uniform_faces(cfg, bu)
    b2amp = amp * r[4]
    bx, by, _ = W.faces_from_potential(
        cfg, Az=lambda x, y, z: -b2amp * np.sin(kv[0] * x + kv[1] * y - kmag * speed * t) / kmag)
    bz = B3 + c * r[5]
    st = W.assemble(cfg, rho, *vel, p, bx + ux, by + uy, bz)
    period = (1.0 / math.sqrt(2.0)) / abs(speed)
    return cfg, st, period


def wave_error(n, wave, recon="plm", rk=2, emf="uct_hll"):
    amp = 1e-6
    cfg, st, T = wave_state_2d(n, wave, amp, recon=recon, rk=rk)
    s = oracle.OracleSim(dict(cfg, emf=emf), st)
    t = 0.0
    while t < T - 1e-14:
        dt = min(s.cfl_dt(), T - t)
        s.step(dt)
        t += dt
    out = s.get_state()
    err = sum(np.mean(np.abs(out[k] - st[k])) for k in ("rho", "mx", "my", "mz", "E", "b2"))
    err += np.mean(np.abs(out["b0"] - st["b0"])) + np.mean(np.abs(out["b1"] - st["b1"]))
    return err / amp


@pytest.mark.slow
@pytest.mark.parametrize("wave", ["fast", "alfven"])
def test_linear_wave_second_order(wave):
    """L1 error over one period falls at about second order (ratio 4 per
    halving; minmod clipping at smooth extrema lowers the ratio at coarse
    resolution, a first-order defect would give about 2)."""
    e = [wave_error(n, wave) for n in (16, 32, 64)]
    assert e[0] / e[1] > 2.5 and e[1] / e[2] > 2.6, e


@pytest.mark.slow
def test_linear_wave_wenoz_rk3_higher_order():
    """WENO-Z + RK3 (Eq. RK3 with the cited SSP weights): second order overall,
    since the CT edge fields use linear reconstructions, with a smaller error
    than PLM + RK2.  With the printed 1/3 weight of L** the error does not
    converge at all."""
    e = [wave_error(n, "fast", recon="wenoz", rk=3) for n in (16, 32, 64)]
    assert e[0] / e[1] > 2.8 and e[1] / e[2] > 2.8, e
    assert e[2] < wave_error(64, "fast")


def cpa_error(n, ndim, t_end, recon="plm", rk=2):
    gen = W.cpa_2d if ndim == 2 else W.cpa_3d
    cfg, st = gen(n, recon=recon, rk=rk)
    _, exact = gen(n, t=t_end, recon=recon, rk=rk)
    s = oracle.OracleSim(cfg, st)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(s.cfl_dt(), t_end - t)
        s.step(dt)
        t += dt
    out = s.get_state()
    return sum(np.mean(np.abs(out[k] - exact[k])) for k in ("rho", "mx", "my", "mz", "E", "b0", "b1", "b2"))


@pytest.mark.slow
def test_cpa_2d_converges_to_exact_translation():
    """The circularly polarised Alfven wave is an exact nonlinear solution
    translating at the Alfven speed (§4.2); PLM + RK2 converges at second order."""
    T = 1.0 / math.sqrt(2.0)
    e = [cpa_error(n, 2, T) for n in (16, 32, 64)]
    assert e[0] / e[1] > 2.4 and e[1] / e[2] > 2.3, e


@pytest.mark.slow
def test_cpa_3d_short_time():
    T = 0.1
    e = [cpa_error(n, 3, T) for n in (8, 16)]
    assert e[0] / e[1] > 3.0, e


def test_pressure_floor_keeps_conservation():
    """The floor acts on the recovered primitives only: on a periodic grid the
    totals stay conserved even while floors are hit (the low-beta blast)."""
    cfg, st = W.blast_3d(20, bc="periodic")
    s = oracle.OracleSim(cfg, st)
    s.advance(15)
    assert s.floors > 0
    out = s.get_state()
    t0, t1 = totals(cfg, st), totals(cfg, out)
    for k in t0:
        assert abs(t1[k][0] - t0[k][0]) <= 1e-13 * max(t0[k][1], t1[k][1], 1e-300), k
    div, scale = div_b(cfg, out)
    assert div <= 1e-12 * scale


def test_without_floor_the_low_beta_blast_fails():
    """The reason for the floor: at beta = 0.002 the recovered pressure turns
    negative within a few steps."""
    cfg, st = W.blast_3d(16, p_floor=0.0)
    s = oracle.OracleSim(cfg, st)
    with pytest.raises(FloatingPointError):
        s.advance(20)
