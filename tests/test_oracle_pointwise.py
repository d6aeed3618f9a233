"""Oracle pins, pointwise pieces: primitive recovery, physical flux, fast speed,
Riemann solvers and reconstructions, each against a closed form or an
independent textbook formula (CPU only)."""
import math

import numpy as np
import pytest

import oracle

G = 5.0 / 3.0


def prim_to_cons_3d(rho, v, B, p, gamma):
    """Eq. Energy and m = rho v, written in vector form."""
    E = p / (gamma - 1) + 0.5 * rho * np.dot(v, v) + 0.5 * np.dot(B, B)
    return np.array([rho, *(rho * v), E])


def test_c2p_inverts_energy_definition():
    rng = np.random.default_rng(1)
    for _ in range(200):
        rho = rng.uniform(0.1, 10)
        v = rng.uniform(-3, 3, 3)
        B = rng.uniform(-3, 3, 3)
        p = rng.uniform(0.01, 10)
        u = prim_to_cons_3d(rho, v, B, p, G)
        V = oracle.c2p(np.concatenate([u, B]), G)
        assert V[0] == rho
        np.testing.assert_allclose(V[1:4], v, rtol=1e-14, atol=1e-14)
        np.testing.assert_array_equal(V[4:7], B)
        assert abs(V[7] - p) <= 1e-12 * (u[4] + 1.0)


def flux_tensor(rho, v, B, p, gamma):
    """Flux tensor T of Eq. mhd as 3x8 (rows: direction; cols: rho, m, B, E)."""
    pt = p + 0.5 * np.dot(B, B)
    E = p / (gamma - 1) + 0.5 * rho * np.dot(v, v) + 0.5 * np.dot(B, B)
    T = np.zeros((3, 8))
    T[:, 0] = rho * v
    T[:, 1:4] = rho * np.outer(v, v) - np.outer(B, B) + pt * np.eye(3)
    T[:, 4:7] = np.outer(v, B) - np.outer(B, v)
    T[:, 7] = (E + pt) * v - np.dot(v, B) * B
    return T


@pytest.mark.parametrize("d", [0, 1, 2])
def test_sweep_flux_matches_flux_tensor(d):
    """The sweep-frame flux (normal d, cyclic transverse) equals row d of T."""
    rng = np.random.default_rng(10 + d)
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    for _ in range(50):
        rho = rng.uniform(0.1, 5)
        v = rng.uniform(-2, 2, 3)
        B = rng.uniform(-2, 2, 3)
        p = rng.uniform(0.1, 5)
        w = [rho, v[d], v[t1], v[t2], B[t1], B[t2], p]
        F, U = oracle.side_flux(w, B[d], G)
        T = flux_tensor(rho, v, B, p, G)[d]
        expect = [T[0], T[1 + d], T[1 + t1], T[1 + t2], T[4 + t1], T[4 + t2], T[7]]
        np.testing.assert_allclose(F, expect, rtol=1e-13, atol=1e-13)
        assert abs(T[4 + d]) < 1e-14  # no flux of the normal field
        cons = prim_to_cons_3d(rho, v, B, p, G)
        np.testing.assert_allclose(U, [cons[0], cons[1 + d], cons[1 + t1], cons[1 + t2], B[t1], B[t2], cons[4]],
                                   rtol=1e-14)


def test_fast_speed_limits():
    rho, p = 1.7, 0.9
    cs = math.sqrt(G * p / rho)
    # no field: sound speed
    assert oracle.fast_speed(rho, p, 0.0, 0.0, G) == pytest.approx(cs, rel=1e-15)
    # field along the normal: max(cs, cA)
    for b in (0.3, 2.5):
        ca = b / math.sqrt(rho)
        assert oracle.fast_speed(rho, p, b * b, b, G) == pytest.approx(max(cs, ca), rel=1e-14)
    # field across the normal: sqrt(cs^2 + cA^2)
    b = 1.3
    assert oracle.fast_speed(rho, p, b * b, 0.0, G) == pytest.approx(math.sqrt(cs * cs + b * b / rho), rel=1e-15)


def random_w(rng):
    return np.array([rng.uniform(0.2, 3), *rng.uniform(-1.5, 1.5, 3), *rng.uniform(-1.5, 1.5, 2), rng.uniform(0.2, 3)])


@pytest.mark.parametrize("solver", ["hll", "hlld"])
def test_riemann_consistency(solver):
    """F(U, U) = F(U)."""
    rng = np.random.default_rng(3)
    for _ in range(300):
        w = random_w(rng)
        bn = rng.uniform(-2, 2)
        F, ing = oracle.riemann(solver, w, w, bn, G)
        Fe, _ = oracle.side_flux(w, bn, G)
        np.testing.assert_allclose(F, Fe, rtol=1e-12, atol=1e-12 * np.max(np.abs(Fe)))
        assert ing[0] + ing[1] == pytest.approx(1.0, abs=1e-15)
        assert ing[2] >= 0.0


@pytest.mark.parametrize("solver", ["hll", "hlld"])
def test_riemann_supersonic_upwind(solver):
    rng = np.random.default_rng(4)
    for sgn in (+1, -1):
        wl = random_w(rng)
        wr = random_w(rng)
        wl[1] = wr[1] = sgn * 50.0
        F, ing = oracle.riemann(solver, wl, wr, 0.7, G)
        Fe, _ = oracle.side_flux(wl if sgn > 0 else wr, 0.7, G)
        np.testing.assert_array_equal(F, Fe)


@pytest.mark.parametrize("u", [0.0, 0.4, -0.3])
def test_hlld_resolves_isolated_contact_exactly(u):
    """A pure density jump moving with the flow (same u, v, w, B, p) is resolved
    without diffusion by HLLD: the flux is F of the upwind state.  HLL is not."""
    wl = np.array([2.0, u, 0.3, -0.2, 0.5, 0.4, 1.0])
    wr = np.array([0.5, u, 0.3, -0.2, 0.5, 0.4, 1.0])
    bn = 0.8
    F, _ = oracle.riemann("hlld", wl, wr, bn, G)
    up = wl if u >= 0 else wr
    Fe, _ = oracle.side_flux(up, bn, G)
    np.testing.assert_allclose(F, Fe, rtol=1e-13, atol=1e-13)
    Fh, _ = oracle.riemann("hll", wl, wr, bn, G)
    assert np.max(np.abs(Fh - Fe)) > 1e-2


@pytest.mark.parametrize("theta", [0.5, 1.7, 3.0])
@pytest.mark.parametrize("direction", [+1, -1])
def test_hlld_resolves_isolated_rotational_discontinuity_exactly(theta, direction):
    """An isolated rotational (Alfven) discontinuity with u = 0, equal rho, p and
    |B_t| on both sides.  Rankine-Hugoniot for the induction and transverse
    momentum equations at speed s = direction * Bn / sqrt(rho) gives
    [v_t] = -(s / Bn) [B_t], satisfied by v_t = -direction * B_t / sqrt(rho).
    A right-going wave leaves U_L at x/t = 0 (flux F(U_L)); a left-going one
    leaves U_R.  HLLD reproduces this exactly; HLL does not."""
    rho, p, bn, b = 1.3, 0.8, 0.9, 0.7
    btl = np.array([b, 0.0])
    btr = b * np.array([math.cos(theta), math.sin(theta)])
    sr = math.sqrt(rho)
    wl = np.array([rho, 0.0, *(-direction * btl / sr), *btl, p])
    wr = np.array([rho, 0.0, *(-direction * btr / sr), *btr, p])
    F, _ = oracle.riemann("hlld", wl, wr, bn, G)
    Fe, _ = oracle.side_flux(wl if direction > 0 else wr, bn, G)
    np.testing.assert_allclose(F, Fe, rtol=1e-13, atol=1e-13)
    Fh, _ = oracle.riemann("hll", wl, wr, bn, G)
    assert np.max(np.abs(Fh - Fe)) > 1e-2


def hllc_flux(wl, wr, gamma, SL, SR):
    """HLLC flux for the Euler equations (Toro, Riemann Solvers, eq. 10.26, 10.37-10.39)."""
    def cons(w):
        rho, u, v, wz, p = w
        return np.array([rho, rho * u, rho * v, rho * wz, p / (gamma - 1) + 0.5 * rho * (u * u + v * v + wz * wz)])

    def flux(w):
        rho, u, v, wz, p = w
        U = cons(w)
        return np.array([rho * u, rho * u * u + p, rho * u * v, rho * u * wz, (U[4] + p) * u])

    rl, ul, pl = wl[0], wl[1], wl[4]
    rr, ur, pr = wr[0], wr[1], wr[4]
    Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (rl * (SL - ul) - rr * (SR - ur))

    def ustar(w, S):
        rho, u, v, wz, p = w
        U = cons(w)
        f = rho * (S - u) / (S - Ss)
        return f * np.array([1.0, Ss, v, wz, U[4] / rho + (Ss - u) * (Ss + p / (rho * (S - u)))])

    if SL >= 0:
        return flux(wl)
    if Ss >= 0:
        return flux(wl) + SL * (ustar(wl, SL) - cons(wl))
    if SR > 0:
        return flux(wr) + SR * (ustar(wr, SR) - cons(wr))
    return flux(wr)


def test_hlld_reduces_to_hllc_without_field():
    rng = np.random.default_rng(7)
    gamma = 1.4
    for _ in range(300):
        wl = np.array([rng.uniform(0.2, 3), *rng.uniform(-1, 1, 3), 0.0, 0.0, rng.uniform(0.2, 3)])
        wr = np.array([rng.uniform(0.2, 3), *rng.uniform(-1, 1, 3), 0.0, 0.0, rng.uniform(0.2, 3)])
        F, _ = oracle.riemann("hlld", wl, wr, 0.0, gamma)
        cl = math.sqrt(gamma * wl[6] / wl[0])
        cr = math.sqrt(gamma * wr[6] / wr[0])
        SL = min(wl[1], wr[1]) - max(cl, cr)
        SR = max(wl[1], wr[1]) + max(cl, cr)
        e = lambda w: np.array([w[0], w[1], w[2], w[3], w[6]])  # noqa: E731
        Fc = hllc_flux(e(wl), e(wr), gamma, SL, SR)
        np.testing.assert_allclose(F[[0, 1, 2, 3, 6]], Fc, rtol=1e-12, atol=1e-12)
        assert F[4] == 0.0 and F[5] == 0.0


def test_hll_matches_two_wave_formula():
    """HLL = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) inside the fan."""
    rng = np.random.default_rng(8)
    for _ in range(100):
        wl, wr = random_w(rng), random_w(rng)
        bn = rng.uniform(-1, 1)
        F, ing = oracle.riemann("hll", wl, wr, bn, G)
        FL, UL = oracle.side_flux(wl, bn, G)
        FR, UR = oracle.side_flux(wr, bn, G)
        BL = bn * bn + wl[4] ** 2 + wl[5] ** 2
        BR = bn * bn + wr[4] ** 2 + wr[5] ** 2
        cf = max(oracle.fast_speed(wl[0], wl[6], BL, bn, G), oracle.fast_speed(wr[0], wr[6], BR, bn, G))
        SL = min(wl[1], wr[1]) - cf
        SR = max(wl[1], wr[1]) + cf
        if SL >= 0:
            expect = FL
        elif SR <= 0:
            expect = FR
        else:
            expect = (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)
        np.testing.assert_allclose(F, expect, rtol=1e-12, atol=1e-12)
        aR, aL = max(0.0, SR), min(0.0, SL)
        d = -aR * aL / (aR - aL)
        np.testing.assert_allclose(ing, [aR / (aR - aL), -aL / (aR - aL), d, wl[1], wr[1], d],
                                   rtol=1e-14, atol=1e-15)


# ---- reconstruction ----

@pytest.mark.parametrize("method", ["plm", "wenoz", "ppm"])
def test_recon_constant_and_linear(method):
    for a, b in [(1.0, 0.0), (0.3, 0.7), (-2.0, -0.25)]:
        s = a + b * np.arange(-2, 3)
        p, m = oracle.recon(method, s)
        assert p == pytest.approx(a + 0.5 * b, abs=1e-14)
        assert m == pytest.approx(a - 0.5 * b, abs=1e-14)


def test_plm_minmod_cases():
    assert oracle.recon("plm", [0, 1.0, 2.0, 1.0, 0]) == (2.0, 2.0)   # extremum: flat
    p, m = oracle.recon("plm", [0, 0.0, 1.0, 1.5, 0])                   # slopes 1, 0.5 -> 0.5
    assert (p, m) == (1.25, 0.75)
    p, m = oracle.recon("plm", [0, 0.0, -1.0, -4.0, 0])                 # slopes -1, -3 -> -1
    assert (p, m) == (-1.5, -0.5)


def cell_avg_poly(coef, i):
    """Average of sum_k c_k x^k over [i - 1/2, i + 1/2]."""
    P = np.polynomial.polynomial.Polynomial(coef).integ()
    return P(i + 0.5) - P(i - 0.5)


def test_wenoz_exact_for_quadratic_averages():
    """All three candidate stencils are exact for cell averages of a quadratic, so
    any convex combination is: V^L_{i+1/2} = q(i + 1/2)."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        c = rng.uniform(-2, 2, 3)
        s = np.array([cell_avg_poly(c, i) for i in range(-2, 3)])
        p, m = oracle.recon("wenoz", s)
        q = np.polynomial.polynomial.Polynomial(c)
        assert p == pytest.approx(q(0.5), abs=1e-12)
        assert m == pytest.approx(q(-0.5), abs=1e-12)


def test_wenoz_fifth_order_on_smooth_data():
    errs = []
    for h in (0.1, 0.05, 0.025):
        x = 0.3 + h * np.arange(-2, 3)
        avg = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h   # averages of sin
        p, m = oracle.recon("wenoz", avg)
        errs.append(max(abs(p - math.sin(0.3 + h / 2)), abs(m - math.sin(0.3 - h / 2))))
    assert errs[0] / errs[1] > 20 and errs[1] / errs[2] > 25


def test_ppm_fourth_order_face_value_on_cubic():
    """The unlimited PPM face value is exact for cell averages of a cubic; on a
    monotone cubic no constraint acts."""
    c = [0.1, 1.0, 0.05, 0.01]   # monotone on [-3, 3]
    s = np.array([cell_avg_poly(c, i) for i in range(-2, 3)])
    p, m = oracle.recon("ppm", s)
    q = np.polynomial.polynomial.Polynomial(c)
    assert p == pytest.approx(q(0.5), abs=1e-13)
    assert m == pytest.approx(q(-0.5), abs=1e-13)


@pytest.mark.parametrize("method", ["plm", "ppm"])
def test_no_new_extrema(method):
    rng = np.random.default_rng(5)
    for _ in range(500):
        s = rng.uniform(-1, 1, 5)
        p, m = oracle.recon(method, s)
        lo, hi = min(s[1:4]), max(s[1:4])
        assert lo - 1e-15 <= p <= hi + 1e-15 and lo - 1e-15 <= m <= hi + 1e-15
    # step data: no overshoot
    for s in ([0, 0, 0, 1, 1], [0, 0, 1, 1, 1], [1, 1, 1, 0, 0]):
        p, m = oracle.recon(method, np.array(s, dtype=float))
        assert 0.0 <= p <= 1.0 and 0.0 <= m <= 1.0
