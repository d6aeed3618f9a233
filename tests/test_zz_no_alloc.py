"""The allocation-free entry point mhd_step_noalloc against the context API.

Some callers cannot allocate device memory (their memory belongs to another
allocator or budget, or they may not pay the synchronisation an allocation can
imply); mhd_step_noalloc serves them from a fixed file-scope scratch array.
Its result must equal mhd_step's on the same state and dt, on two calls in a
row; it must accept the grids the header's table lists and refuse one cell
more; a step that meets a non-positive pressure leaves the caller's arrays as
they were; and calls after the first leave the device's free memory
unchanged.  Collected last, so a failure here comes after every other test
has run; it also passes alone.
"""
import numpy as np
import pytest

from paper_2511_20337_b300 import workloads as W
from conftest import relerr

pytestmark = pytest.mark.gpu

KEYS = ("rho", "mx", "my", "mz", "E", "b0", "b1", "b2")
TOL = 1e-12   # the one-step tolerance of the parity tests


@pytest.fixture(scope="module")
def mhd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20337_b300 import mhd as M
    M.lib()
    return M


CASES = {
    "turbulent3d-12x10x8-wenoz-hlld-rk3": lambda: W.turbulent_3d((12, 10, 8), seed=3, recon="wenoz", rk=3),
    "orszag-tang2d-64-plm-hlld-rk2": lambda: W.orszag_tang_2d(64),
    "blast3d-16-outflow-ppm-rk3": lambda: W.blast_3d(16, recon="ppm"),
}


def _reference(mhd, cfg, st, nsteps):
    """States and step sizes of nsteps CFL steps through the context API."""
    sim = mhd.Sim(cfg, st)
    states, dts = [], []
    for _ in range(nsteps):
        dt = sim.cfl_dt()
        sim.step(dt)
        dts.append(dt)
        states.append(sim.get_conserved())
    sim.close()
    return states, dts


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_context_step_twice(mhd, case):
    import torch
    cfg, st = CASES[case]()
    ref, dts = _reference(mhd, cfg, st, 2)
    dev = {k: torch.from_numpy(np.ascontiguousarray(st[k])).cuda() for k in KEYS}
    for n, dt in enumerate(dts):           # two calls in a row on the same arrays
        mhd.step_noalloc(cfg, dev, dt)
        torch.cuda.synchronize()
        for k in KEYS:
            got = dev[k].cpu().numpy()
            assert relerr(got, ref[n][k]) <= TOL, (case, n, k)


def test_noalloc_after_a_different_grid(mhd):
    """The scratch array keeps the previous call's contents; a call on another
    grid shape must not see them."""
    import torch
    a_cfg, a_st = CASES["turbulent3d-12x10x8-wenoz-hlld-rk3"]()
    b_cfg, b_st = CASES["orszag-tang2d-64-plm-hlld-rk2"]()
    ref, dts = _reference(mhd, b_cfg, b_st, 1)
    a_dev = {k: torch.from_numpy(np.ascontiguousarray(a_st[k])).cuda() for k in KEYS}
    mhd.step_noalloc(a_cfg, a_dev, 1e-4)
    b_dev = {k: torch.from_numpy(np.ascontiguousarray(b_st[k])).cuda() for k in KEYS}
    mhd.step_noalloc(b_cfg, b_dev, dts[0])
    for k in KEYS:
        assert relerr(b_dev[k].cpu().numpy(), ref[0][k]) <= TOL, k


def test_noalloc_rejects_grids_beyond_its_scratch(mhd):
    import torch
    cfg = W.base_cfg(3, (64, 64, 64), (0, 0, 0), (1, 1, 1))
    shapes = mhd.state_shapes(cfg)
    dev = {k: torch.ones(s, dtype=torch.float64, device="cuda") for k, s in zip(KEYS, shapes)}
    before = {k: v.clone() for k, v in dev.items()}
    with pytest.raises(mhd.MhdError) as e:
        mhd.step_noalloc(cfg, dev, 1e-3)
    assert e.value.code == -7
    for k in KEYS:
        assert torch.equal(dev[k], before[k])   # nothing was touched


def _uniform(cfg, shapes):
    """A uniform state (steady under the step): rho = 1, v = 0, p = 1, B = (0.3, -0.2, 0.1)."""
    B = (0.3, -0.2, 0.1)
    E = 1.0 / (cfg["gamma"] - 1.0) + 0.5 * sum(b * b for b in B)
    return {k: np.full(s, v) for k, s, v in zip(KEYS, shapes, (1.0, 0.0, 0.0, 0.0, E) + B)}


# largest square / cubic grids that fit the scratch array (the table in include/mhd.h)
LIMITS = [(2, "plm", "uct_hll", 266), (2, "plm", "uct_hlld", 259), (2, "wenoz", "uct_hll", 264),
          (2, "ppm", "uct_hlld", 257), (3, "plm", "uct_hll", 36), (3, "plm", "uct_hlld", 36),
          (3, "wenoz", "uct_hll", 34), (3, "ppm", "uct_hlld", 34)]


@pytest.mark.parametrize("ndim,recon,emf,n", LIMITS, ids=[f"{a}d-{b}-{c}-{d}" for a, b, c, d in LIMITS])
def test_noalloc_documented_limits(mhd, ndim, recon, emf, n):
    import torch
    for m, ok in ((n, True), (n + 1, False)):
        cfg = W.base_cfg(ndim, (m,) * ndim, (0,) * ndim, (1,) * ndim, recon=recon, emf=emf)
        st = _uniform(cfg, mhd.state_shapes(cfg))
        dev = {k: torch.from_numpy(st[k]).cuda() for k in KEYS}
        if ok:
            mhd.step_noalloc(cfg, dev, 1e-3)
            for k in KEYS:   # a uniform state stays uniform
                assert relerr(dev[k].cpu().numpy(), st[k]) <= 1e-14, (m, k)
        else:
            with pytest.raises(mhd.MhdError) as e:
                mhd.step_noalloc(cfg, dev, 1e-3)
            assert e.value.code == -7


def test_noalloc_leaves_the_arrays_alone_on_an_unphysical_step(mhd):
    import torch
    cfg, st = CASES["orszag-tang2d-64-plm-hlld-rk2"]()
    st = {k: np.ascontiguousarray(v).copy() for k, v in st.items()}
    st["E"][0, 20, 30] = -5.0          # a negative pressure, made on the host
    dev = {k: torch.from_numpy(st[k]).cuda() for k in KEYS}
    with pytest.raises(mhd.MhdError) as e:
        mhd.step_noalloc(cfg, dev, 1e-3)
    assert e.value.code == -4
    for k in KEYS:
        np.testing.assert_array_equal(dev[k].cpu().numpy(), st[k], err_msg=k)


def test_noalloc_allocates_no_device_memory(mhd):
    """After a first call (which may load the library's device code on this
    device, and with it the scratch array), further calls leave the device's
    free memory unchanged."""
    import torch
    cfg, st = CASES["turbulent3d-12x10x8-wenoz-hlld-rk3"]()
    dev = {k: torch.from_numpy(np.ascontiguousarray(st[k])).cuda() for k in KEYS}
    mhd.step_noalloc(cfg, dev, 1e-4)
    b_cfg, b_st = CASES["orszag-tang2d-64-plm-hlld-rk2"]()
    b_dev = {k: torch.from_numpy(np.ascontiguousarray(b_st[k])).cuda() for k in KEYS}
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        mhd.step_noalloc(cfg, dev, 1e-4)
        mhd.step_noalloc(b_cfg, b_dev, 1e-4)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
