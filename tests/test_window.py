"""The sampled-window oracle reproduces the full-grid oracle bitwise (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W
from window import window_step, box, halo_for, blockwise_cfl_dt

CASES = [
    ("rand3d-plm-hlld-rk2", lambda: (lambda c: (c, W.random_state(c, 41)))(W.base_cfg(3, (20, 18, 19), (0, 0, 0), (1, 1, 1)))),
    ("blast3d-wenoz-rk3-outflow", lambda: W.blast_3d(22)),
    ("ot2d-ppm-hll-rk3", lambda: W.orszag_tang_2d(30, recon="ppm", riemann="hll", rk=3)),
    # large enough that the power-of-two windows are true sub-boxes
    ("rand3d-40-windowed", lambda: (lambda c: (c, W.random_state(c, 42)))(W.base_cfg(3, (40, 36, 38), (0, 0, 0), (1, 1, 1)))),
    ("blast3d-40-windowed", lambda: W.blast_3d(40)),
    ("ot2d-80-windowed", lambda: W.orszag_tang_2d(80, recon="wenoz", rk=3)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_window_matches_full_grid(name, make):
    cfg, st = make()
    full = oracle.OracleSim(cfg, st)
    dt = full.cfl_dt()
    full.step(dt)
    ref = full.get_state()
    nd = cfg["ndim"]
    n = cfg["n"]
    rng = np.random.default_rng(7)
    for _ in range(3):
        size = [3] * nd
        lo = [int(rng.integers(0, n[d] - size[d] + 1)) if cfg["bc"][2 * d] == "outflow" else int(rng.integers(0, n[d]))
              for d in range(nd)]
        got = window_step(cfg, st, lo, size, halo_for(cfg), dt)
        for k in oracle.KEYS:
            exp = box(ref[k], lo, size, n)
            np.testing.assert_array_equal(got[k], exp, err_msg=f"{k} lo={lo}")


BLOCK_CASES = [
    ("rand3d-40x36x34-ct", 16, lambda: (lambda c: (c, W.random_state(c, 43)))(W.base_cfg(3, (40, 36, 34), (0, 0, 0), (1, 0.9, 1.1)))),
    ("blast3d-40-outflow-ct", 16, lambda: W.blast_3d(40)),
    ("ot2d-80-ct", 16, lambda: W.orszag_tang_2d(80)),
    ("turbulent3d-32-glm", 8, lambda: W.to_glm(*W.turbulent_3d(32))),
    ("rand3d-24x20x18-glm", 8, lambda: W.to_glm(*(lambda c: (c, W.random_state(c, 44)))(
        W.base_cfg(3, (24, 20, 18), (0, 0, 0), (1, 1, 1))))),
]


@pytest.mark.parametrize("name,block,make", BLOCK_CASES, ids=[c[0] for c in BLOCK_CASES])
def test_blockwise_cfl_equals_full_grid_cfl(name, block, make):
    cfg, st = make()
    glm = cfg.get("divb", "ct") == "glm"
    full = (oracle.OracleGlm(cfg, st) if glm else oracle.OracleSim(cfg, st)).cfl_dt()
    assert blockwise_cfl_dt(cfg, st, block) == full


def test_glm_window_matches_full_grid():
    cfg, st = W.to_glm(*W.orszag_tang_2d(64, recon="wenoz", rk=3), alpha=0.2)
    rng = np.random.default_rng(9)
    st["psi"] = 0.01 * rng.standard_normal(st["rho"].shape)
    full = oracle.OracleGlm(cfg, st, alpha=0.2)
    dt = full.cfl_dt()
    full.step(dt)
    ref = full.get_state()
    for lo in ([0, 0], [61, 3], [30, 62]):
        got = window_step(cfg, st, lo, [3, 3], halo_for(cfg), dt)
        for k in oracle.GLM_KEYS:
            np.testing.assert_array_equal(got[k], box(ref[k], lo, [3, 3], cfg["n"]), err_msg=f"{k} lo={lo}")
