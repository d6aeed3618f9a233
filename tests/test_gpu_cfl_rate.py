"""The two CFL rates of the device against each other and against the oracle's
per-cell rate.  The CFL step takes the largest IEEE rate.  Its candidate pass
keeps only the cells whose fast rate lies within 4e-13 of the largest fast
rate.  That is exact as long as the fast rate is within 2e-13 of the IEEE one;
here it must stay within 5e-14.  The IEEE rate must equal the oracle's
bitwise."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import mhd

pytestmark = pytest.mark.gpu


def states(n, seed, gamma):
    """Random primitives over many decades, plus the corner cases of the fast
    speed: zero field, purely normal or purely transverse field, zero normal
    velocity, and gamma p = B_n^2 with no transverse field (the discriminant
    (gamma p - B_n^2)^2 vanishes) or with a tiny one."""
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(-4, 4, n)
    p = 10.0 ** rng.uniform(-8, 4, n)
    v = rng.uniform(-10, 10, (n, 3)) * (10.0 ** rng.uniform(-6, 0, (n, 1)))
    B = rng.standard_normal((n, 3)) * (10.0 ** rng.uniform(-6, 2, (n, 1)))
    X = np.column_stack([rho, v, B, p])
    m = n // 8
    X[0:m, 4:7] = 0.0                                   # no field
    X[m:2 * m, 5:7] = 0.0                               # field along x only
    X[2 * m:3 * m, 4] = 0.0                             # no x field
    X[3 * m:4 * m, 1:4] = 0.0                           # at rest
    a = X[4 * m:5 * m]                                  # gamma p = B_x^2, no transverse field
    a[:, 5:7] = 0.0
    a[:, 4] = np.sqrt(gamma * a[:, 7])
    b = X[5 * m:6 * m]                                  # the same with a tiny transverse field
    b[:, 4] = np.sqrt(gamma * b[:, 7])
    b[:, 5:7] = b[:, 4:5] * 1e-9 * rng.standard_normal((m, 2))
    return X


def oracle_rate(X, ndim, gamma, dx):
    """The oracle's per-cell rate (its cfl_rate, IEEE double in the same order)."""
    out = np.zeros(len(X))
    for t, (rho, vx, vy, vz, bx, by, bz, p) in enumerate(X):
        B2 = (bx * bx + by * by) + bz * bz
        lam = 0.0
        for d, (vd, bd) in enumerate(((vx, bx), (vy, by), (vz, bz))[:ndim]):
            cf = oracle.fast_speed(rho, p, B2, bd, gamma)
            term = (abs(vd) + cf) * (1.0 / dx[d])
            lam = term if d == 0 else lam + term
        out[t] = lam
    return out


@pytest.mark.parametrize("ndim,gamma,dx", [(3, 5.0 / 3.0, (1 / 256, 1 / 256, 1 / 256)),
                                           (3, 1.4, (1 / 704, 1 / 704, 1 / 352)),
                                           (2, 5.0 / 3.0, (2 * np.pi / 128, 2 * np.pi / 128, 1.0))])
def test_fast_rate_within_window_and_ieee_rate_equals_oracle(ndim, gamma, dx):
    X = states(20000, 11 + ndim, gamma)
    near, ieee = mhd.probe_cfl_rate(ndim, gamma, dx, X)
    ref = oracle_rate(X, ndim, gamma, dx)
    bad = np.flatnonzero(ieee != ref)
    assert bad.size == 0, (bad[:5], ieee[bad[:5]], ref[bad[:5]])
    rel = np.abs(near - ieee) / ieee
    assert np.all(ieee > 0)
    assert rel.max() <= 5e-14, (rel.max(), X[np.argmax(rel)])
