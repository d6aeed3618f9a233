"""CUDA library vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (normwise per array: max|gpu - oracle| / max|oracle|):
  1 step: 1e-12, 100 steps: 1e-10; CFL dt: bitwise (both sides use IEEE
  operations in the same order).  The GPU contracts a*b+c into FMAs and forms
  reciprocals by a refined seed, so single operations differ from the oracle
  by an ulp; the limiter and wave-fan branches are continuous, so those
  differences stay at the round-off level.
"""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W
from conftest import relerr

pytestmark = pytest.mark.gpu

KEYS = oracle.KEYS
TOL1 = 1e-12
TOL100 = 1e-10


@pytest.fixture(scope="module")
def mhd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20337_b300 import mhd as M
    M.lib()
    return M


def compare(a, b, tol, where=""):
    errs = {k: relerr(a[k], b[k]) for k in KEYS}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"{where} rel errors above {tol}: {bad}"
    return max(errs.values())


def random_case(ndim, n, recon="plm", riemann="hlld", rk=2, bc="periodic", seed=0, L=None):
    L = L or (1.0,) * ndim
    cfg = W.base_cfg(ndim, n, (0.0,) * ndim, L, recon=recon, riemann=riemann, rk=rk, bc=bc)
    return cfg, W.random_state(cfg, seed)


SMALL = {
    "ot2d-48": lambda: W.orszag_tang_2d(48),
    "rand2d-37x29-plm-hlld-rk2": lambda: random_case(2, (37, 29), seed=1),
    "rand2d-33x17-plm-hll-rk3": lambda: random_case(2, (33, 17), riemann="hll", rk=3, seed=2),
    "rand2d-31x35-wenoz-hlld-rk3": lambda: random_case(2, (31, 35), recon="wenoz", rk=3, seed=3),
    "rand2d-20x21-ppm-hlld-rk2-outflow": lambda: random_case(2, (20, 21), recon="ppm", bc="outflow", seed=4),
    "rand3d-13x11x9-plm-hlld-rk2": lambda: random_case(3, (13, 11, 9), seed=5),
    "rand3d-17x5x7-wenoz-hll-rk3-outflow": lambda: random_case(3, (17, 5, 7), recon="wenoz", riemann="hll", rk=3,
                                                               bc="outflow", seed=6),
    "rand3d-9x10x11-ppm-hlld-rk3": lambda: random_case(3, (9, 10, 11), recon="ppm", rk=3, seed=7),
    "blast3d-20-wenoz-rk3": lambda: W.blast_3d(20),
    "turb3d-24-plm-hlld-rk2": lambda: W.turbulent_3d(24, seed=11),
    "cpa3d-16-wenoz-rk3": lambda: W.cpa_3d(16, recon="wenoz", rk=3),
    "mixed-bc-2d": lambda: (lambda c: (c, W.random_state(c, 8)))(
        W.base_cfg(2, (26, 19), (0, 0), (1.3, 1.0), bc=["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"])),
}


@pytest.mark.parametrize("case", list(SMALL))
def test_cfl_dt_bitwise(mhd, case):
    cfg, st = SMALL[case]()
    dt_o = oracle.OracleSim(cfg, st).cfl_dt()
    dt_g = mhd.Sim(cfg, st).cfl_dt()
    assert dt_g == dt_o, (dt_g, dt_o)


@pytest.mark.parametrize("case", list(SMALL))
def test_one_step(mhd, case):
    cfg, st = SMALL[case]()
    o = oracle.OracleSim(cfg, st)
    dt = o.cfl_dt()
    o.step(dt)
    g = mhd.Sim(cfg, st)
    g.step(dt)
    compare(g.get_conserved(), o.get_state(), TOL1, case)
    assert g.status()[0] == 0


@pytest.mark.parametrize("case", ["rand2d-37x29-plm-hlld-rk2", "rand3d-13x11x9-plm-hlld-rk2",
                                  "rand2d-31x35-wenoz-hlld-rk3", "blast3d-20-wenoz-rk3"])
def test_ten_steps_with_oracle_dt(mhd, case):
    """Ten steps with the oracle's dt sequence stay within the one-step bound
    times the step count."""
    cfg, st = SMALL[case]()
    o = oracle.OracleSim(cfg, st)
    g = mhd.Sim(cfg, st)
    for _ in range(10):
        dt = o.cfl_dt()
        o.step(dt)
        g.step(dt)
    compare(g.get_conserved(), o.get_state(), 10 * TOL1, case)


def test_orszag_tang_2d_128_100_steps(mhd):
    """The 2D Orszag-Tang workload (128^2, PLM + HLLD + RK2 + UCT, CFL 0.4),
    100 CFL steps each side with its own dt: state within 1e-10, time and dt
    sequence equal to round-off."""
    cfg, st = W.orszag_tang_2d(128)
    o = oracle.OracleSim(cfg, st)
    dts = o.advance(100, record_dt=True)
    g = mhd.Sim(cfg, st)
    g.advance(100)
    compare(g.get_conserved(), o.get_state(), TOL100, "OT 100 steps")
    assert abs(g.time - o.time) <= 1e-13 * o.time
    assert abs(g.last_dt - dts[-1]) <= 1e-12 * dts[-1]


@pytest.mark.parametrize("case", ["turb3d-24-plm-hlld-rk2", "ot3d-24-wenoz-hlld-rk3-ucthlld"])
def test_3d_100_steps(mhd, case):
    """3D over 100 CFL steps, each side with its own dt: the turbulent field
    (PLM + HLLD + RK2 + UCT-HLL) and Orszag-Tang (WENO-Z + HLLD + RK3 +
    UCT-HLLD), state within 1e-10 (face fields relative to the largest
    component: the Orszag-Tang B_z starts at zero), time to round-off."""
    if case in SMALL:
        cfg, st = SMALL[case]()
    else:
        cfg, st = W.orszag_tang_3d(24, recon="wenoz", rk=3, emf="uct_hlld")
    o = oracle.OracleSim(cfg, st)
    o.advance(100)
    g = mhd.Sim(cfg, st)
    g.advance(100)
    out, ref = g.get_conserved(), o.get_state()
    bmax = max(np.max(np.abs(ref[k])) for k in ("b0", "b1", "b2"))
    for k in KEYS:
        err = (np.max(np.abs(out[k] - ref[k])) / bmax if k in ("b0", "b1", "b2")
               else relerr(out[k], ref[k]))
        assert err <= TOL100, (case, k, err)
    assert abs(g.time - o.time) <= 1e-13 * o.time


@pytest.mark.parametrize("case", ["blast3d-20-wenoz-rk3", "turb3d-24-plm-hlld-rk2",
                                  "rand2d-20x21-ppm-hlld-rk2-outflow"])
def test_many_steps(mhd, case):
    cfg, st = SMALL[case]()
    o = oracle.OracleSim(cfg, st)
    o.advance(30)
    g = mhd.Sim(cfg, st)
    g.advance(30)
    compare(g.get_conserved(), o.get_state(), TOL100, case)


def test_advance_equals_cfl_step_loop(mhd):
    """mhd_advance (device dt, graph replay) is bitwise the host loop of
    mhd_cfl_dt + mhd_step."""
    cfg, st = W.orszag_tang_2d(40, recon="wenoz", rk=3)
    a = mhd.Sim(cfg, st)
    a.advance(7)
    b = mhd.Sim(cfg, st)
    for _ in range(7):
        b.step(b.cfl_dt())
    sa, sb = a.get_conserved(), b.get_conserved()
    for k in KEYS:
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
    assert a.time == b.time


@pytest.mark.parametrize("n", [(1, 9), (9, 1), (2, 3), (16, 16), (17, 33), (48, 1)])
def test_degenerate_and_ragged_2d_sizes(mhd, n):
    """One-cell and two-cell axes, exact and ragged segment counts."""
    cfg, st = random_case(2, n, seed=sum(n))
    o = oracle.OracleSim(cfg, st)
    dt = o.cfl_dt()
    o.step(dt)
    g = mhd.Sim(cfg, st)
    assert g.cfl_dt() == dt
    g.step(dt)
    compare(g.get_conserved(), o.get_state(), TOL1, str(n))


@pytest.mark.parametrize("n", [(1, 1, 5), (3, 1, 2), (5, 4, 1)])
def test_degenerate_3d_sizes(mhd, n):
    cfg, st = random_case(3, n, recon="wenoz", rk=3, seed=sum(n))
    o = oracle.OracleSim(cfg, st)
    dt = o.cfl_dt()
    o.step(dt)
    g = mhd.Sim(cfg, st)
    g.step(dt)
    compare(g.get_conserved(), o.get_state(), TOL1, str(n))


def test_device_memory_io_matches_host(mhd):
    import torch
    cfg, st = random_case(3, (8, 7, 6), seed=9)
    g = mhd.Sim(cfg, {k: torch.from_numpy(v).cuda() for k, v in st.items()})
    h = mhd.Sim(cfg, st)
    for s in (g, h):
        s.advance(3)
    out_d = g.get_conserved({k: torch.zeros(v.shape, dtype=torch.float64, device="cuda") for k, v in st.items()})
    out_h = h.get_conserved()
    for k in KEYS:
        np.testing.assert_array_equal(out_d[k].cpu().numpy(), out_h[k], err_msg=k)


def test_set_prim_equals_set_conserved(mhd):
    cfg = W.base_cfg(3, (6, 5, 4), (0, 0, 0), (1, 1, 1))
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)
    rho = rng.uniform(0.5, 1.5, shape)
    v = [rng.uniform(-1, 1, shape) for _ in range(3)]
    p = rng.uniform(0.5, 1.5, shape)
    bx, by, bz = W.uniform_faces(cfg, (0.3, 0.2, -0.4))
    st = W.assemble(cfg, rho, *v, p, bx, by, bz)
    a = mhd.Sim(cfg, st)
    b = mhd.Sim(cfg)
    b.set_prim(rho, v, p, [bx, by, bz])
    sa, sb = a.get_conserved(), b.get_conserved()
    for k in KEYS:
        np.testing.assert_allclose(sb[k], sa[k], rtol=1e-15, atol=1e-15, err_msg=k)


def test_unphysical_state_is_reported(mhd):
    """A cell with negative pressure (made on the host) is reported with its
    flat index k*ny*nx + j*nx + i; the context stays usable afterwards."""
    cfg, st = random_case(2, (12, 10), seed=12)
    st = {k: v.copy() for k, v in st.items()}
    st["E"][0, 3, 7] = -1.0
    g = mhd.Sim(cfg, st)
    with pytest.raises(mhd.MhdError) as e:
        g.cfl_dt()              # primitive pass only: exactly that cell is flagged
    assert e.value.code == -4
    rc, bad = g.status()
    assert rc == -4 and bad == 3 * 12 + 7
    assert g.status()[0] == 0   # cleared
    g.step(1e-4)                # later stages may flag its neighbours too
    rc, bad = g.status()
    assert rc == -4 and 0 <= bad <= 3 * 12 + 7
    cfg2, st2 = random_case(2, (12, 10), seed=13)
    g.set_conserved(st2)
    g.step(1e-4)
    assert g.status()[0] == 0


def test_invalid_configs_rejected(mhd):
    base = W.base_cfg(2, (8, 8), (0, 0), (1, 1))
    for bad in ({"ndim": 4}, {"n": (0, 8)}, {"gamma": 1.0}, {"rk": 4}, {"cfl": 0.0},
                {"bc": ["periodic", "outflow", "periodic", "periodic", "periodic", "periodic"]}):
        cfg = dict(base)
        cfg.update(bad)
        with pytest.raises(mhd.MhdError) as e:
            mhd.Sim(cfg)
        assert e.value.code == -1


def test_boundary_switch(mhd):
    """Periodic -> outflow on x through mhd_set_boundaries equals a context
    created with outflow x."""
    cfg, st = random_case(2, (14, 12), seed=14)
    g = mhd.Sim(cfg, st)
    bc = ["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"]
    g.set_boundaries(bc)
    cfg2 = dict(cfg)
    cfg2["bc"] = bc
    h = mhd.Sim(cfg2, st)
    o = oracle.OracleSim(cfg2, st)
    dt = o.cfl_dt()
    for s in (g, h):
        s.step(dt)
    o.step(dt)
    compare(g.get_conserved(), o.get_state(), TOL1)
    sg, sh = g.get_conserved(), h.get_conserved()
    for k in KEYS:
        np.testing.assert_array_equal(sg[k], sh[k])


@pytest.mark.parametrize("recon", ["wenoz", "ppm", "plm"])
def test_low_beta_blast_floors_and_fallbacks_match(mhd, recon):
    """The beta = 0.002 blast with the pressure floor: state within the
    many-step bound, and the counts of floored pressures and first-order
    reconstruction fallbacks equal to the oracle's."""
    cfg, st = W.blast_3d(24, recon=recon, rk=3 if recon != "plm" else 2)
    o = oracle.OracleSim(cfg, st)
    o.advance(12)
    g = mhd.Sim(cfg, st)
    g.advance(12)
    compare(g.get_conserved(), o.get_state(), TOL100, f"blast {recon}")
    fb, fl = g.counters()
    assert (fb, fl) == (o.fallbacks, o.floors)
    assert fl > 0


@pytest.mark.parametrize("case", ["ot2d", "turb3d"])
def test_segment_length_does_not_change_the_result(mhd, case):
    """Each face is solved by the same arithmetic whatever segment marches it,
    so any segment length gives the same state, bitwise."""
    cfg, st = W.orszag_tang_2d(40) if case == "ot2d" else W.turbulent_3d(20)
    out = []
    for seg in (1, 2, 5, 16, 64):
        sim = mhd.Sim(cfg, st)
        sim.set_seglen(seg)
        sim.advance(3)
        out.append(sim.get_conserved())
    for o in out[1:]:
        for k in KEYS:
            assert np.array_equal(o[k], out[0][k]), k


def test_autotune_restores_state_and_time(mhd):
    cfg, st = W.orszag_tang_2d(64)
    sim = mhd.Sim(cfg, st)
    sim.advance(2)
    before, t0 = sim.get_conserved(), sim.time
    seg = sim.autotune()
    F = max(cfg["n"][:cfg["ndim"]]) + 1
    assert seg in {2, 4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64} | {-(-F // k) for k in range(4, 13)}
    after = sim.get_conserved()
    for k in KEYS:
        assert np.array_equal(before[k], after[k]), k
    assert sim.time == t0
    ref = mhd.Sim(cfg, st)
    ref.advance(5)
    sim.advance(3)
    a, b = sim.get_conserved(), ref.get_conserved()
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("n", [(128, 128), (64, 48, 40), (256, 256, 256)])
def test_default_segment_length_and_setter(mhd, n):
    """The default is the longest of 2..64 that leaves about eight waves of
    384-thread SM loads in the sweep with the fewest faces; set/get round-trip."""
    torch = pytest.importorskip("torch")
    nd = len(n)
    cfg = W.base_cfg(nd, n, (0.0,) * nd, (1.0,) * nd)
    sim = mhd.Sim(cfg)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fewest = min((n[d] + 1) * int(np.prod([n[t] + 2 for t in range(nd) if t != d])) for d in range(nd))
    assert sim.seglen == min(64, max(2, fewest // (8 * sms * 384)))
    sim.set_seglen(7)
    assert sim.seglen == 7
    with pytest.raises(mhd.MhdError):
        sim.set_seglen(0)


@pytest.mark.parametrize("divb", ["ct", "glm"])
def test_checkpoint_and_resume_equals_uninterrupted_run(mhd, divb):
    """Save the state and time after 4 CFL steps, resume in a new context and
    take 3 more: the state and time equal those of 7 uninterrupted steps."""
    cfg, st = W.orszag_tang_2d(48, recon="wenoz", rk=3)
    if divb == "glm":
        cfg, st = W.to_glm(cfg, st)
    a = mhd.Sim(cfg, st)
    a.advance(7)
    want, t_want = a.get_conserved(), a.time
    b = mhd.Sim(cfg, st)
    b.advance(4)
    saved, t_saved = b.get_conserved(), b.time
    b.close()
    c = mhd.Sim(cfg, saved)
    c.time = t_saved
    c.advance(3)
    got = c.get_conserved()
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    assert c.time == t_want
    with pytest.raises(mhd.MhdError):
        c.time = float("nan")
