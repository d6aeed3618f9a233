"""The fused stage of 2D constrained-transport grids (one cooperative launch
per RK stage, include/mhd.h "fused stage"): the same state as one launch per
phase, to the bit, and the bounded grid barrier that reports MHD_ERR_TIMEOUT.

The timeout tests make a wait run out without faulting anything: one block is
told (from the host) not to arrive at one barrier, the other blocks' waits end
at their limit, every block returns, and the host reads the status.  The
context stays usable afterwards."""
import numpy as np
import pytest

from paper_2511_20337_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20337_b300 import mhd as M
    M.lib()
    return M


def rand2d(n, seed, **kw):
    cfg = W.base_cfg(2, n, (0.0, 0.0), (1.0, 1.3), **kw)
    return cfg, W.random_state(cfg, seed)


CASES = {
    "ot-64-plm-hlld-rk2": lambda: W.orszag_tang_2d(64),
    "ot-48-wenoz-hlld-rk3-ucthlld": lambda: W.orszag_tang_2d(48, recon="wenoz", rk=3, emf="uct_hlld"),
    "rand-37x23-ppm-hll-rk3-outflow": lambda: rand2d((37, 23), 3, recon="ppm", riemann="hll", rk=3, bc="outflow"),
    "rand-29x31-plm-hll-rk2-mixed": lambda: rand2d(
        (29, 31), 4, bc=["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"]),
    "rand-19x26-wenoz-hlld-rk2-mixed-y": lambda: rand2d(
        (19, 26), 5, recon="wenoz", bc=["periodic", "periodic", "outflow", "outflow", "periodic", "periodic"]),
    "adjoint-256": lambda: W.adjoint_2d(256),
    "blast-like-floor-2d": lambda: rand2d((40, 40), 6, recon="wenoz", rk=3, bc="outflow", p_floor=0.9),
}


def run(M, cfg, st, fused, nsteps, seglen=None, dt=None):
    g = M.Sim(cfg, st)
    g.set_fused(fused)
    if seglen:
        g.set_seglen(seglen)
    if dt is None:
        g.advance(nsteps)
    else:
        for _ in range(nsteps):
            g.step(dt)
    out = g.get_conserved()
    return out, g.time, g.counters(), g.status()


@pytest.mark.parametrize("case", list(CASES))
def test_fused_equals_per_phase_launches(mhd, case):
    cfg, st = CASES[case]()
    g = mhd.Sim(cfg, st)
    on, blocks = g.fused
    assert on and blocks >= 148, (on, blocks)
    ref = run(mhd, cfg, st, False, 12)
    for seglen in (None, 3):
        got = run(mhd, cfg, st, True, 12, seglen=seglen)
        for k in ref[0]:
            np.testing.assert_array_equal(got[0][k], ref[0][k], err_msg=f"{case} {k} seglen {seglen}")
        assert got[1] == ref[1] and got[2] == ref[2] and got[3] == ref[3] == (0, -1)


def test_fused_given_dt_equals_per_phase(mhd):
    cfg, st = W.orszag_tang_2d(40, rk=3)
    ref = run(mhd, cfg, st, False, 5, dt=2e-3)
    got = run(mhd, cfg, st, True, 5, dt=2e-3)
    for k in ref[0]:
        np.testing.assert_array_equal(got[0][k], ref[0][k])
    assert got[1] == ref[1]


def test_fused_eligibility(mhd):
    cfg, st = W.turbulent_3d(12, seed=1)
    g = mhd.Sim(cfg, st)
    assert g.fused == (False, 0)
    with pytest.raises(mhd.MhdError):
        g.set_fused(True)
    gcfg, gst = W.to_glm(*W.orszag_tang_2d(32))
    h = mhd.Sim(gcfg, gst)
    assert h.fused == (False, 0)
    with pytest.raises(mhd.MhdError):
        h.set_fused(True)
    cfg2, st2 = W.orszag_tang_2d(32)
    s = mhd.Sim(cfg2, st2)
    for bad in (0.0, -1.0, 61.0, float("nan")):
        with pytest.raises(mhd.MhdError):
            s.set_wait_limit(bad)
    with pytest.raises(mhd.MhdError):
        s.inject_skip_arrive(s.fused[1], 0)   # no such block
    # above 256^2 cells: eligible, off by default, on when asked
    big_cfg, big_st = W.orszag_tang_2d(300)
    b = mhd.Sim(big_cfg, big_st)
    on, blocks = b.fused
    assert not on and blocks >= 148
    b.set_fused(True)
    assert b.fused == (True, blocks)


def test_autotune_picks_a_form_and_restores_the_state(mhd):
    cfg, st = W.orszag_tang_2d(96)
    g = mhd.Sim(cfg, st)
    g.advance(3)
    before, t = g.get_conserved(), g.time
    seglen = g.autotune()
    assert seglen >= 2 and g.seglen == seglen
    on, blocks = g.fused
    assert blocks >= 148
    after = g.get_conserved()
    for k in before:
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)
    assert g.time == t
    g.advance(2)
    ref = mhd.Sim(cfg, st)
    ref.advance(5)
    want, got = ref.get_conserved(), g.get_conserved()
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_barrier_count_per_stage(mhd):
    cfg, st = W.orszag_tang_2d(32)
    g = mhd.Sim(cfg, st)
    g.advance(1)
    # last stage: primitives, sweeps, edge fields (its ghost zones came with
    # the first stage's output)
    assert g.fused_waits() == 3
    g.step(1e-3)
    assert g.fused_waits() == 3
    ocfg, ost = rand2d((20, 24), 2, bc="outflow")
    h = mhd.Sim(ocfg, ost)
    h.advance(1)
    assert h.fused_waits() == 7            # two outflow axes: copy and normal passes each


@pytest.mark.parametrize("barrier,time_moves", [(1, False), (3, True)])
def test_skipped_arrival_times_out_and_keeps_the_state(mhd, barrier, time_moves):
    cfg, st = W.orszag_tang_2d(64)
    g = mhd.Sim(cfg, st)
    g.advance(2)
    before = g.get_conserved()
    t_before = g.time
    g.set_wait_limit(0.05)
    g.inject_skip_arrive(5, barrier)
    g.advance(3)
    rc, bad = g.status()
    assert (rc, bad) == (-5, -1)
    assert g.status() == (0, -1)           # cleared, barrier re-armed, injection off
    after = g.get_conserved()
    for k in before:
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)
    if time_moves:                          # the first stage's CFL phase completed
        assert g.time > t_before
    else:
        assert g.time == t_before
    # the context keeps working: three more steps equal an uninterrupted run's
    g.time = t_before
    g.advance(3)
    ref = mhd.Sim(cfg, st)
    ref.advance(5)
    want = ref.get_conserved()
    got = g.get_conserved()
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    assert g.status() == (0, -1)


def test_timeout_in_a_single_step_call(mhd):
    cfg, st = W.orszag_tang_2d(32, rk=3)
    g = mhd.Sim(cfg, st)
    before = g.get_conserved()
    g.set_wait_limit(0.02)
    g.inject_skip_arrive(0, 2)
    g.step(1e-3)
    assert g.status()[0] == -5
    after = g.get_conserved()
    for k in before:
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)


def test_two_fused_contexts_side_by_side(mhd):
    """Two contexts on their own streams advance at the same time (no sync
    between them): both cooperative grids complete with no timeout."""
    import torch
    cfg, st = W.orszag_tang_2d(96)
    cfg2, st2 = W.adjoint_2d(128)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = mhd.Sim(cfg, st, stream=s1.cuda_stream)
    b = mhd.Sim(cfg2, st2, stream=s2.cuda_stream)
    for s in (a, b):
        s.set_wait_limit(0.5)
    for _ in range(10):
        a.advance(5)
        b.advance(5)
    assert a.status() == (0, -1) and b.status() == (0, -1)
    ra, rb = mhd.Sim(cfg, st), mhd.Sim(cfg2, st2)
    ra.advance(50)
    rb.advance(50)
    for x, y in ((a, ra), (b, rb)):
        got, want = x.get_conserved(), y.get_conserved()
        for k in want:
            np.testing.assert_array_equal(got[k], want[k], err_msg=k)


ADJ_CASES = {
    "adjoint-48-hlld-rk2": lambda: W.adjoint_2d(48),
    "random-40x36-hll-rk3": lambda: rand2d((40, 36), 9, riemann="hll", rk=3),
    "random-37x29-hlld-rk3-misfit": lambda: rand2d((37, 29), 10, rk=3),
    "random-33x30-wenoz-hlld-rk3": lambda: rand2d((33, 30), 11, recon="wenoz", rk=3),
    "random-31x27-ppm-hll-rk2-misfit": lambda: rand2d((31, 27), 12, recon="ppm", riemann="hll"),
}


def adjoint_of(M, cfg, st, fused, nsteps=10, functional="magnetic_energy"):
    g = M.Sim(cfg, st)
    g.set_fused(fused)
    target = None
    if functional == "misfit":
        target = [np.full(s, 0.5) for s in g.shapes[:5]] + [np.full(g.shapes[0], 0.1)]
    J, dts = g.adjoint(nsteps, None, ckpt_every=4, functional=functional, target=target)
    return J, dts, g.grad_conserved()


@pytest.mark.parametrize("case", list(ADJ_CASES))
def test_adjoint_of_a_fused_context_equals_the_per_launch_one(mhd, case):
    """The adjoint of a fused context (its forward pass one cooperative launch
    per stage) equals that of a per-launch context to the bit."""
    cfg, st = ADJ_CASES[case]()
    functional = "misfit" if "misfit" in case else "magnetic_energy"
    Jf, dtf, gf = adjoint_of(mhd, cfg, st, True, functional=functional)
    Ju, dtu, gu = adjoint_of(mhd, cfg, st, False, functional=functional)
    assert Jf == Ju
    assert np.array_equal(dtf, dtu)
    for k in gu:
        np.testing.assert_array_equal(gf[k], gu[k], err_msg=k)


def test_forward_pass_timeout_in_an_adjoint_run(mhd):
    """A barrier of the adjoint's fused forward pass that runs out: the run
    reports MHD_ERR_TIMEOUT, mhd_status re-arms the barrier, and the next run
    gives the per-launch context's gradient."""
    cfg, st = W.adjoint_2d(32)
    g = mhd.Sim(cfg, st)
    g.set_wait_limit(0.05)
    g.inject_skip_arrive(7, 1)
    with pytest.raises(mhd.MhdError) as err:
        g.adjoint(6, None, ckpt_every=3)
    assert err.value.code == -5
    assert g.status() == (-5, -1)
    assert g.status() == (0, -1)
    g.set_conserved(st)
    J, dts = g.adjoint(6, None, ckpt_every=3)
    got = g.grad_conserved()
    ref = mhd.Sim(cfg, st)
    ref.set_fused(False)
    J2, dts2 = ref.adjoint(6, None, ckpt_every=3)
    want = ref.grad_conserved()
    assert J == J2
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_profiled_adjoint_equals_the_timed_one(mhd):
    """The profiling run keeps one launch per reverse kernel class (and runs the
    recomputes in sequence on the context); the timed run fuses the combine and
    edge transposes into one launch and recomputes beside the reverse pass.
    Both give the same gradient to the bit."""
    cfg, st = W.adjoint_2d(40)
    g = mhd.Sim(cfg, st)
    J, dts = g.adjoint(8, None, ckpt_every=3)
    want = g.grad_conserved()
    h = mhd.Sim(cfg, st)
    phases, classes = h.adjoint_profile(8, dts, ckpt_every=3)
    assert phases["reverse"] > 0.0
    got = h.grad_conserved()
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
