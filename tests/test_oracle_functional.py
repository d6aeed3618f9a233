"""Pins of the oracle's adjoint functionals and of its initial map from
primitives (the two pieces the gradient tests all share, so a mistake there
would pass every tape / dual / finite-difference comparison):

  * J_mag = 1/2 sum_c |B_c|^2 dV with B_c the mean of the two faces (2D B_z:
    the cell value) -- uniform fields give 1/2 |B|^2 V exactly, and a
    discrete sine field on the faces gives the closed form
    1/4 A^2 cos^2(pi dx) V, because the mean of two face values of
    A sin(2 pi x) is A sin(2 pi x_c) cos(pi dx);
  * J_misfit = 1/2 sum_c sum_q (U_q - T_q)^2 dV over rho, m, E (2D: and B_z)
    -- a uniform state against a constant offset target gives
    1/2 V sum_q delta_q^2, and against a zero target the hand-computed
    conserved values of a worked example (Eq. Energy);
  * the initial map m = rho v, E = p/(G-1) + rho v^2/2 + B^2/2 (Eq. Energy) is
    undone by the oracle's primitive recovery to round-off, and a uniform
    state keeps J over steps (it is steady)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W


def uniform(cfg, rho, v, p, B):
    shapes = oracle.state_shapes(cfg)
    cell = shapes[0]
    prim = {"rho": np.full(cell, rho), "vx": np.full(cell, v[0]), "vy": np.full(cell, v[1]),
            "vz": np.full(cell, v[2]), "p": np.full(cell, p)}
    Bf = [np.full(s, b) for s, b in zip(shapes[5:], B)]
    return prim, Bf


def volume(cfg):
    nd = cfg["ndim"]
    return math.prod(cfg["x1"][d] - cfg["x0"][d] for d in range(nd))


CASES = [W.base_cfg(3, (5, 4, 3), (0.0, 0.0, 0.0), (1.0, 2.0, 0.5)),
         W.base_cfg(2, (6, 5), (-1.0, 0.0), (1.0, 1.5))]


@pytest.mark.parametrize("cfg", CASES, ids=["3d", "2d"])
def test_magnetic_energy_of_uniform_field(cfg):
    B = (0.75, -1.25, 0.5)
    prim, Bf = uniform(cfg, 1.3, (0.1, -0.2, 0.3), 0.9, B)
    J = oracle.functional_prim(cfg, prim, Bf, [])
    exact = 0.5 * (0.75 ** 2 + 1.25 ** 2 + 0.5 ** 2) * volume(cfg)
    assert J == pytest.approx(exact, rel=1e-14)


def test_magnetic_energy_of_face_sine_field():
    """B_x on the faces x_f = x0 + i dx is A sin(2 pi x_f) (periodic: the last
    face repeats the first); B_y = b uniform, B_z = 0.  The cell means are
    A sin(2 pi x_c) cos(pi dx) and the sum of sin^2 over a full period of nx
    cells is nx/2, so J = 1/4 A^2 cos^2(pi dx) V + 1/2 b^2 V."""
    nx, ny, nz = 8, 3, 2
    cfg = W.base_cfg(3, (nx, ny, nz), (0.0, 0.0, 0.0), (1.0, 0.75, 0.5))
    A, b = 1.7, 0.4
    prim, Bf = uniform(cfg, 1.0, (0.0, 0.0, 0.0), 1.0, (0.0, b, 0.0))
    dx = 1.0 / nx
    xf = np.arange(nx + 1) * dx
    Bf[0] = np.broadcast_to(A * np.sin(2 * np.pi * xf), (nz, ny, nx + 1)).copy()
    J = oracle.functional_prim(cfg, prim, Bf, [])
    V = 1.0 * 0.75 * 0.5
    exact = 0.25 * A * A * math.cos(math.pi * dx) ** 2 * V + 0.5 * b * b * V
    assert J == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("cfg", CASES, ids=["3d", "2d"])
def test_misfit_of_uniform_state_against_offset_target(cfg):
    nd = cfg["ndim"]
    rho, v, p, B = 2.0, (0.5, -1.0, 0.25), 3.0, (1.0, 2.0, -0.5)
    prim, Bf = uniform(cfg, rho, v, p, B)
    U = oracle.state_from_prims(cfg, prim, Bf)
    keys = ["rho", "mx", "my", "mz", "E"] + (["b2"] if nd == 2 else [])
    delta = [0.1, -0.2, 0.3, 0.05, -0.4, 0.7][:len(keys)]
    target = [U[k] - d for k, d in zip(keys, delta)]
    J = oracle.functional_prim(cfg, prim, Bf, [], which="misfit", target=target)
    exact = 0.5 * volume(cfg) * sum(d * d for d in delta)
    assert J == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("cfg", CASES, ids=["3d", "2d"])
def test_misfit_against_zero_target_worked_example(cfg):
    """rho = 2, v = (1/2, -1, 1/4), p = 3, B = (1, 2, -1/2), G = 5/3: by hand,
    m = (1, -2, 1/2) and E = 3/(2/3) + (1/2)(2)(1/4 + 1 + 1/16) + (1/2)(1 + 4 + 1/4)
    = 9/2 + 21/16 + 21/8 = 135/16, so with a zero target
    J = 1/2 V (4 + 1 + 4 + 1/4 + (135/16)^2) (2D: + B_z^2 = 1/4)."""
    nd = cfg["ndim"]
    prim, Bf = uniform(cfg, 2.0, (0.5, -1.0, 0.25), 3.0, (1.0, 2.0, -0.5))
    U = oracle.state_from_prims(cfg, prim, Bf)
    E = Fraction(135, 16)
    assert np.all(U["rho"] == 2.0)
    assert np.all(U["mx"] == 1.0) and np.all(U["my"] == -2.0) and np.all(U["mz"] == 0.5)
    assert np.max(np.abs(U["E"] - float(E))) <= 1e-15 * float(E)
    zeros = [np.zeros_like(U["rho"]) for _ in range(6 if nd == 2 else 5)]
    J = oracle.functional_prim(cfg, prim, Bf, [], which="misfit", target=zeros)
    s = Fraction(4) + 1 + 4 + Fraction(1, 4) + E * E + (Fraction(1, 4) if nd == 2 else 0)
    exact = 0.5 * volume(cfg) * float(s)
    assert J == pytest.approx(exact, rel=1e-14)


@pytest.mark.parametrize("cfg", CASES, ids=["3d", "2d"])
def test_initial_map_round_trips_through_primitive_recovery(cfg):
    nd = cfg["ndim"]
    rng = np.random.default_rng(7)
    shapes = oracle.state_shapes(cfg)
    cell = shapes[0]
    prim = {"rho": rng.uniform(0.5, 2.0, cell), "vx": rng.normal(0, 1, cell), "vy": rng.normal(0, 1, cell),
            "vz": rng.normal(0, 1, cell), "p": rng.uniform(0.3, 3.0, cell)}
    Bf = [rng.normal(0, 1, s) for s in shapes[5:]]
    for d in range(nd):  # periodic layout: the last face of each axis repeats the first
        ax = Bf[d].ndim - 1 - d
        first = np.take(Bf[d], [0], axis=ax)
        idx = [slice(None)] * Bf[d].ndim
        idx[ax] = slice(-1, None)
        Bf[d][tuple(idx)] = first
    U = oracle.state_from_prims(cfg, prim, Bf)
    bx, by, bz = W.cell_field(cfg, U["b0"], U["b1"], U["b2"])
    for q, b in zip(("b0", "b1", "b2"), Bf):
        assert np.array_equal(U[q], b)  # the field is held, not mapped
    for idx in np.ndindex(cell):
        u8 = [U["rho"][idx], U["mx"][idx], U["my"][idx], U["mz"][idx], U["E"][idx], bx[idx], by[idx], bz[idx]]
        V = oracle.c2p(u8, cfg["gamma"])
        assert V[0] == prim["rho"][idx]
        for d, k in enumerate(("vx", "vy", "vz")):
            assert abs(V[1 + d] - prim[k][idx]) <= 1e-14 * max(1.0, abs(prim[k][idx]))
        assert abs(V[7] - prim["p"][idx]) <= 1e-13 * prim["p"][idx]
    assert nd in (2, 3)


def test_uniform_state_keeps_its_functionals_over_steps():
    cfg = W.base_cfg(3, (6, 5, 4), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    prim, Bf = uniform(cfg, 1.1, (0.3, -0.2, 0.1), 0.8, (0.6, 0.4, -0.3))
    U = oracle.state_from_prims(cfg, prim, Bf)
    target = [U[k] * 0.9 for k in ("rho", "mx", "my", "mz", "E")]
    dts = [0.01, 0.012, 0.009]
    for which, tg in (("magnetic_energy", None), ("misfit", target)):
        J0 = oracle.functional_prim(cfg, prim, Bf, [], which=which, target=tg)
        J3 = oracle.functional_prim(cfg, prim, Bf, dts, which=which, target=tg)
        assert J3 == pytest.approx(J0, rel=1e-13)
