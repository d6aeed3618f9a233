"""The sampled-window oracle reproduces the full-grid oracle bitwise (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W
from window import window_step, box, halo_for

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
