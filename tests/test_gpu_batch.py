"""Batched ensemble (mhd_batch_*) against the single-grid path and the oracle.

Every run of a batch executes the same item bodies as a single-grid context
with its own CFL dt, so after any number of steps each run must equal, bitwise,
the same run advanced alone; the segment length chosen by the autotuner moves
only where a thread's march starts, not any face's arithmetic.
"""
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


def ensemble(sizes, seed=4, **kw):
    members = W.ensemble_members(len(sizes), seed=seed, sizes=(16,))
    cases = []
    for n, m in zip(sizes, members):
        m = dict(m, n=n)
        cases.append(W.ensemble_member_state(m, **kw))
    return cases


def assert_same(a, b, what):
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"{what}: {k}")


def test_batch_equals_single_grid_runs_bitwise(mhd):
    cases = ensemble([12, 16, 33, 20, 48, 7])
    cfgs = [c for c, _ in cases]
    bt = mhd.Batch(cfgs, [s for _, s in cases])
    bt.step(6)
    times = bt.times()
    for r, (cfg, st) in enumerate(cases):
        g = mhd.Sim(cfg, st)
        g.advance(6)
        assert_same(bt.get_conserved(r), g.get_conserved(), f"run {r}")
        assert times[r] == g.time
    assert bt.status()[0] == 0
    # per-run dt: the runs differ in size, beta and Mach, so their times differ
    assert len(set(times)) == len(times)


def test_batch_matches_oracle(mhd):
    cases = ensemble([24, 10])
    bt = mhd.Batch([c for c, _ in cases], [s for _, s in cases])
    bt.step(5)
    for r, (cfg, st) in enumerate(cases):
        o = oracle.OracleSim(cfg, st)
        o.advance(5)
        out, ref = bt.get_conserved(r), o.get_state()
        for k in KEYS:
            assert relerr(out[k], ref[k]) <= 5e-12, (r, k)


def test_autotune_restores_state_and_keeps_results(mhd):
    cases = ensemble([16, 130, 24, 40])   # one run above the small-class size
    cfgs = [c for c, _ in cases]
    bt = mhd.Batch(cfgs, [s for _, s in cases])
    bt.step(2)
    before = [bt.get_conserved(r) for r in range(len(cases))]
    t_before = bt.times()
    small, large = bt.autotune()
    assert small in (8, 16, 32, 64) and large in (8, 16, 32, 64)
    for r in range(len(cases)):
        assert_same(bt.get_conserved(r), before[r], f"run {r} after autotune")
    assert bt.times() == t_before
    bt.step(3)
    for r, (cfg, st) in enumerate(cases):
        g = mhd.Sim(cfg, st)
        g.advance(5)
        assert_same(bt.get_conserved(r), g.get_conserved(), f"run {r}")


@pytest.mark.parametrize("seglen", [(1, 3), (64, 5)])
def test_any_segment_length_gives_the_same_state(mhd, seglen):
    cases = ensemble([17, 31])
    bt = mhd.Batch([c for c, _ in cases], [s for _, s in cases])
    bt.set_seglen(*seglen)
    bt.step(4)
    for r, (cfg, st) in enumerate(cases):
        g = mhd.Sim(cfg, st)
        g.advance(4)
        assert_same(bt.get_conserved(r), g.get_conserved(), f"run {r}")


def test_batch_3d_outflow_wenoz_rk3(mhd):
    cases = [W.blast_3d(12), W.blast_3d((10, 14, 9))]
    bt = mhd.Batch([c for c, _ in cases], [s for _, s in cases])
    bt.step(4)
    for r, (cfg, st) in enumerate(cases):
        g = mhd.Sim(cfg, st)
        g.advance(4)
        assert_same(bt.get_conserved(r), g.get_conserved(), f"run {r}")


def test_batch_rejects_mixed_schemes(mhd):
    a, _ = W.orszag_tang_2d(16)
    b, _ = W.orszag_tang_2d(16, rk=3)
    with pytest.raises(mhd.MhdError) as e:
        mhd.Batch([a, b])
    assert e.value.code == -1


def test_batch_reports_the_bad_run(mhd):
    cases = ensemble([12, 14, 16])
    states = [dict(s) for _, s in cases]
    states[1] = {k: v.copy() for k, v in states[1].items()}
    states[1]["E"][0, 2, 3] = -1.0
    bt = mhd.Batch([c for c, _ in cases], states)
    bt.step(1)
    rc, run, cell = bt.status()
    assert rc == -4 and run == 1 and 0 <= cell <= 2 * 14 + 3


@pytest.mark.parametrize("case", ["plm-hlld", "wenoz-hlld-rk3"])
def test_staged_x_sweep_equals_direct_loads_bitwise(mhd, case):
    """A single 3D grid with at least 2048 x-pencils stages its x sweep
    through shared memory; the batched kernels always load directly.  Both
    execute the same arithmetic, so one run stepped either way agrees to the
    bit, and with the oracle to round-off (face fields relative to the
    largest field component: the Orszag-Tang B_z starts at zero, and its
    round-off scales with |B|)."""
    if case == "plm-hlld":
        cfg, st = W.turbulent_3d(44)                      # 46^2 = 2116 pencils
    else:
        cfg, st = W.orszag_tang_3d((40, 46, 44), recon="wenoz", rk=3)   # 48 x 46 = 2208 pencils
    g = mhd.Sim(cfg, st)
    g.advance(2)
    bt = mhd.Batch([cfg], [st])
    bt.step(2)
    assert_same(bt.get_conserved(0), g.get_conserved(), case)
    o = oracle.OracleSim(cfg, st)
    o.advance(2)
    out, ref = g.get_conserved(), o.get_state()
    bmax = max(np.max(np.abs(ref[k])) for k in ("b0", "b1", "b2"))
    for k in KEYS:
        if k in ("b0", "b1", "b2"):
            assert np.max(np.abs(out[k] - ref[k])) <= 1e-12 * bmax, k
        else:
            assert relerr(out[k], ref[k]) <= 1e-12, k


def test_packed_io_equals_per_run_io(mhd):
    """Packed state I/O (one array for all runs) against the per-run calls,
    host and device arrays, bitwise; a step after a packed set equals a step
    after per-run sets."""
    torch = pytest.importorskip("torch")
    cases = ensemble([12, 16, 20, 14])
    cfgs = [c for c, _ in cases]
    states = [s for _, s in cases]
    a = mhd.Batch(cfgs, states)
    b = mhd.Batch(cfgs)
    packed = b.pack(states)
    assert packed.size == b.packed_size()
    b.set_conserved_packed(packed)
    b.synchronize()
    for r in range(len(cases)):
        got = b.get_conserved(r)
        for k in KEYS:
            assert np.array_equal(got[k], states[r][k]), (r, k)
    a.step(2)
    b.step(2)
    out = b.unpack(b.get_conserved_packed())
    for r in range(len(cases)):
        want = a.get_conserved(r)
        for k in KEYS:
            assert np.array_equal(out[r][k], want[k]), (r, k)
    # device packed arrays, and a pinned host array read without waiting
    d = torch.from_numpy(packed).cuda()
    b.set_conserved_packed(d)
    b.step(2)
    dev_out = torch.empty_like(d)
    b.get_conserved_packed(dev_out, wait=False)
    pin = torch.empty(b.packed_size(), dtype=torch.float64).pin_memory()
    b.get_conserved_packed(pin, wait=False)
    b.synchronize()
    assert np.array_equal(dev_out.cpu().numpy(), pin.numpy())
    assert np.array_equal(pin.numpy(), a.pack([a.get_conserved(r) for r in range(len(cases))]))
    with pytest.raises(ValueError):
        b.set_conserved_packed(np.zeros(3))
