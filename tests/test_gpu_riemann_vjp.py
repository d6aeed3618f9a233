"""The adjoint's hand-written reverse of the HLL and HLLD solvers against the
forward-mode (multi-tangent) derivative of the same device arithmetic, and
against the oracle's forward-mode directional derivative of its own solver,
on random faces covering every branch of the wave fan."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import mhd

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0


def faces(n, seed):
    """(n, 15) sweep-frame face inputs: W_L, W_R, b_n.  Blocks of subsonic
    random states, supersonic to either side, vanishing normal field, a
    purely normal strong field (degenerate star states), and exactly equal
    left and right states (ties in every min/max)."""
    rng = np.random.default_rng(seed)
    x = np.empty((n, 15))
    for side in (0, 7):
        x[:, side + 0] = rng.uniform(0.3, 2.0, n)       # rho
        x[:, side + 1] = rng.uniform(-0.8, 0.8, n)      # u
        x[:, side + 2] = rng.uniform(-0.8, 0.8, n)      # v
        x[:, side + 3] = rng.uniform(-0.8, 0.8, n)      # w
        x[:, side + 4] = rng.uniform(-1.0, 1.0, n)      # b1
        x[:, side + 5] = rng.uniform(-1.0, 1.0, n)      # b2
        x[:, side + 6] = rng.uniform(0.2, 2.0, n)       # p
    x[:, 14] = rng.uniform(-1.5, 1.5, n)
    k = n // 8
    x[0:k, 1] += 6.0                   # supersonic to the right
    x[0:k, 8] += 6.0
    x[k:2 * k, 1] -= 6.0               # supersonic to the left
    x[k:2 * k, 8] -= 6.0
    x[2 * k:3 * k, 14] = 0.0           # no normal field: no rotational waves
    sl = slice(3 * k, 4 * k)           # field along the normal only, Alfven > sound
    x[sl, [4, 5, 11, 12]] = 0.0
    x[sl, 14] = rng.choice([-1.0, 1.0], k) * rng.uniform(2.0, 3.0, k)
    x[sl, 6] = x[sl, 13] = 0.3
    x[sl, 7] = x[sl, 0]
    x[4 * k:5 * k, 7:14] = x[4 * k:5 * k, 0:7]   # identical sides
    return x


def star_conditioning(x):
    """min over the two sides of |D| / (rho (S - u)(S - S_M)), D = rho (S - u)(S - S_M) - b_n^2:
    the HLLD star-state derivatives carry 1/D^2, so rounding is amplified by
    about this number to the power -2 (numpy estimate of the solver's speeds)."""
    L, R, bn = x[:, 0:7], x[:, 7:14], x[:, 14]

    def lite(W):
        B2 = W[:, 4] ** 2 + W[:, 5] ** 2 + bn ** 2
        gp = GAMMA * W[:, 6]
        s = gp + B2
        disc = np.maximum(s * s - 4 * gp * bn ** 2, 0.0)
        return W[:, 6] + 0.5 * B2, np.sqrt((s + np.sqrt(disc)) / (2 * W[:, 0]))

    pTL, cfL = lite(L)
    pTR, cfR = lite(R)
    cmax = np.maximum(cfL, cfR)
    SL = np.minimum(L[:, 1], R[:, 1]) - cmax
    SR = np.maximum(L[:, 1], R[:, 1]) + cmax
    rsL, rsR = (SL - L[:, 1]) * L[:, 0], (SR - R[:, 1]) * R[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        SM = ((rsR * R[:, 1] - rsL * L[:, 1]) - pTR + pTL) / (rsR - rsL)
        kL = np.abs(1 - bn ** 2 / (rsL * (SL - SM)))
        kR = np.abs(1 - bn ** 2 / (rsR * (SR - SM)))
    k = np.nan_to_num(np.minimum(kL, kR), nan=1.0)
    return np.clip(k, 1e-6, 1.0)


@pytest.mark.parametrize("solver", ["hll", "hlld"])
def test_hand_written_reverse_equals_forward_mode(solver):
    """Both are the exact derivative of the same arithmetic, so they agree to
    rounding: 1e-13 of the face's largest cotangent, times the conditioning
    of near-degenerate HLLD star states."""
    n = 4096
    x = faces(n, 71 if solver == "hll" else 72)
    cot = np.random.default_rng(73).standard_normal((n, 12))
    dual, hand = mhd.probe_riemann_vjp(solver, x, cot, GAMMA)
    assert np.all(np.isfinite(hand))
    scale = np.maximum(np.max(np.abs(dual), axis=1), 1e-300)
    err = np.max(np.abs(hand - dual), axis=1) / scale
    tol = 1e-13 / (star_conditioning(x) ** 2 if solver == "hlld" else 1.0)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, [(int(f), float(err[f]), float(tol[f])) for f in bad[:5]]
    assert np.median(err) <= 1e-15


@pytest.mark.parametrize("solver", ["hll", "hlld"])
def test_reverse_matches_oracle_directional_derivatives(solver):
    """<xbar, t> = <ybar, J t> with J t from central differences of the
    oracle's solver (an independent implementation), on subsonic faces away
    from branch switches: agreement to the difference error."""
    n = 64
    x = faces(8 * n, 74)[5 * n:6 * n]  # the subsonic random block
    rng = np.random.default_rng(75)
    cot = rng.standard_normal((n, 12))
    _, hand = mhd.probe_riemann_vjp(solver, x, cot, GAMMA)
    for f in range(n):
        t = rng.standard_normal(15)
        h = 1e-6

        def out(z):
            F, ing = oracle.riemann(solver, z[0:7], z[7:14], z[14], GAMMA)
            return np.concatenate([F, ing[:5]])  # the UCT-HLL ingredients (d^R repeats d)

        jt = (out(x[f] + h * t) - out(x[f] - h * t)) / (2 * h)
        lhs = float(np.dot(hand[f], t))
        rhs = float(np.dot(cot[f], jt))
        assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(rhs)), (f, lhs, rhs)


def test_uct_hlld_weights_reverse_equals_forward_mode():
    """The UCT-HLLD weights (a^L, a^R, d^L, d^R of the fan region that holds
    x/t = 0) through the hand-written reverse and through forward-mode
    numbers: the same agreement as the flux's, on faces in every region."""
    n = 4096
    x = faces(n, 76)
    cot = np.random.default_rng(77).standard_normal((n, 13))
    dual, hand = mhd.probe_riemann_vjp("hlld", x, cot, GAMMA, emf="uct_hlld")
    assert np.all(np.isfinite(hand))
    scale = np.maximum(np.max(np.abs(dual), axis=1), 1e-300)
    err = np.max(np.abs(hand - dual), axis=1) / scale
    tol = 1e-13 / star_conditioning(x) ** 2
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, [(int(f), float(err[f]), float(tol[f])) for f in bad[:5]]
    assert np.median(err) <= 1e-15
    # with the d^R cotangent zero and UCT-HLL's the same as the old 12-column probe
    c12 = cot[:, :12]
    d_old, h_old = mhd.probe_riemann_vjp("hlld", x, c12, GAMMA)
    c13 = np.concatenate([c12, np.zeros((n, 1))], axis=1)
    d_new, h_new = mhd.probe_riemann_vjp("hlld", x, c13, GAMMA, emf="uct_hll")
    assert np.array_equal(h_old, h_new) and np.array_equal(d_old, d_new)


def test_uct_hlld_reverse_matches_oracle_directional_derivatives():
    """<xbar, t> = <ybar, J t> with J t from central differences of the
    oracle's HLLD solver and its UCT-HLLD weights, on subsonic faces."""
    n = 64
    x = faces(8 * n, 78)[5 * n:6 * n]
    rng = np.random.default_rng(79)
    cot = rng.standard_normal((n, 13))
    _, hand = mhd.probe_riemann_vjp("hlld", x, cot, GAMMA, emf="uct_hlld")
    for f in range(n):
        t = rng.standard_normal(15)
        h = 1e-6

        def out(z):
            F, ing = oracle.riemann("hlld", z[0:7], z[7:14], z[14], GAMMA, emf="uct_hlld")
            return np.concatenate([F, ing])

        jt = (out(x[f] + h * t) - out(x[f] - h * t)) / (2 * h)
        lhs = float(np.dot(hand[f], t))
        rhs = float(np.dot(cot[f], jt))
        assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(rhs)), (f, lhs, rhs)
