"""The domain-decomposed step (mhd_domain_*: bricks with a halo exchange per
RK stage, the decomposition of paper §3.4, Fig. par_ex) against the undivided
grid and the FP64 oracle, through the C-ABI.

Each brick executes the undivided grid's arithmetic on its cells once its
ghost shell holds the undivided grid's values, so the bar is bitwise: the CFL
step, the state after ten CFL steps (captured graph), a host-dt step, the
time and the pressure-floor count equal those of one context on the whole
grid (the fallback count may exceed it: bricks also reconstruct the cells of
their halo pencils), for periodic, outflow and mixed boundaries, PLM / WENO-Z / PPM,
HLL / HLLD, UCT-HLL / UCT-HLLD, RK2 / RK3, 2D and 3D, with uneven bricks.
One step is also compared with the oracle (1e-12), and a bad cell made on the
host is reported with its index in the whole grid."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W
from conftest import relerr

pytestmark = pytest.mark.gpu

KEYS = oracle.KEYS


@pytest.fixture(scope="module")
def mhd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20337_b300 import mhd as M
    M.lib()
    return M


def rand(ndim, n, seed, **kw):
    cfg = W.base_cfg(ndim, n, (0.0,) * ndim, (1.0,) * ndim, **kw)
    return cfg, W.random_state(cfg, seed)


CASES = {
    "turb3d-24-plm-hlld-rk2-2x2x2": (lambda: W.turbulent_3d(24, seed=11), (2, 2, 2)),
    "blast3d-20-wenoz-rk3-outflow-2x1x2": (lambda: W.blast_3d(20), (2, 1, 2)),
    "ot2d-40-plm-hlld-rk2-3x2": (lambda: W.orszag_tang_2d(40), (3, 2)),
    "ot3d-16-wenoz-rk3-ucthlld-1x2x2": (lambda: W.orszag_tang_3d(16, recon="wenoz", rk=3, emf="uct_hlld"), (1, 2, 2)),
    "rand3d-17x9x10-ppm-hll-rk3-outflow-x-3x1x2": (
        lambda: rand(3, (17, 9, 10), 3, recon="ppm", riemann="hll", rk=3,
                     bc=["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"]), (3, 1, 2)),
    "rand2d-23x19-wenoz-hlld-rk2-outflow-y-1x3": (
        lambda: rand(2, (23, 19), 4, recon="wenoz",
                     bc=["periodic", "periodic", "outflow", "outflow", "periodic", "periodic"]), (1, 3)),
    "rand3d-13x12x11-plm-hlld-rk2-outflow-3x2x2": (lambda: rand(3, (13, 12, 11), 5, bc="outflow"), (3, 2, 2)),
}


def same(a, b, what):
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"{what}: {k}")


@pytest.mark.parametrize("case", list(CASES))
def test_domain_equals_undivided_grid_bitwise(mhd, case):
    gen, parts = CASES[case]
    cfg, st = gen()
    g = mhd.Sim(cfg, st)
    d = mhd.Domain(cfg, parts, st)
    assert d.cfl_dt() == g.cfl_dt()
    same(d.get_conserved(), g.get_conserved(), "initial state")
    g.advance(10)
    d.advance(10)
    same(d.get_conserved(), g.get_conserved(), "10 CFL steps")
    assert d.time == g.time
    (fd, pd), (fg, pg) = d.counters(), g.counters()
    assert pd == pg and fd >= fg   # bricks also reconstruct the cells of their halo pencils
    dt = g.cfl_dt()
    g.step(0.5 * dt)
    d.step(0.5 * dt)
    same(d.get_conserved(), g.get_conserved(), "host-dt step")
    assert d.time == g.time
    assert d.status() == (0, -1)
    assert d.launches > 0 and d.halo_bytes > 0
    d.close()
    g.close()


def test_domain_one_step_against_oracle(mhd):
    cfg, st = W.blast_3d(20)
    o = oracle.OracleSim(cfg, st)
    dt = o.cfl_dt()
    o.step(dt)
    d = mhd.Domain(cfg, (2, 2, 1), st)
    assert d.cfl_dt() == dt
    d.step(dt)
    out, ref = d.get_conserved(), o.get_state()
    for k in KEYS:
        assert relerr(out[k], ref[k]) <= 1e-12, k


def test_domain_device_arrays_and_segment_length(mhd):
    import torch
    cfg, st = W.turbulent_3d(20, seed=3)
    dev = {k: torch.from_numpy(v).cuda() for k, v in st.items()}
    d = mhd.Domain(cfg, (2, 2, 2), dev)
    g = mhd.Sim(cfg, st)
    d.set_seglen(3)
    d.advance(4)
    g.advance(4)
    out = {k: torch.empty_like(v) for k, v in dev.items()}
    d.get_conserved(out)
    ref = g.get_conserved()
    for k in KEYS:
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k], err_msg=k)


def test_domain_reports_a_bad_cell_by_its_whole_grid_index(mhd):
    cfg, st = rand(3, (12, 10, 9), 12)
    st = {k: v.copy() for k, v in st.items()}
    st["E"][6, 7, 9] = -1.0                      # in brick (1, 1, 1) of a 2x2x2 split
    d = mhd.Domain(cfg, (2, 2, 2), st)
    with pytest.raises(mhd.MhdError) as e:
        d.cfl_dt()
    assert e.value.code == -4
    rc, bad = d.status()
    assert rc == -4 and bad == (6 * 10 + 7) * 12 + 9
    assert d.status()[0] == 0                    # cleared


def test_domain_rejects_what_it_cannot_split(mhd):
    cfg, st = W.turbulent_3d(12, seed=1)
    for parts in ((5, 1, 1), (1, 1, 0)):          # bricks below G + 1 cells, no bricks
        with pytest.raises(mhd.MhdError):
            mhd.Domain(cfg, parts)
    with pytest.raises(mhd.MhdError):
        mhd.Domain(W.to_glm(cfg, st)[0], (2, 1, 1))
    d = mhd.Domain(cfg, (2, 1, 1))
    with pytest.raises(mhd.MhdError):
        d.advance(1)                             # no state yet
