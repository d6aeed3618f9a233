"""Guard words around the device arrays (include/mhd.h "guard words").

Every field of a context's pool (and every run's block of a batch, every
brick and halo-buffer region of a domain) is followed by guard words holding
a canary.  These tests run each scheme, grid shape and entry point and check
that no launch wrote past the end (or before the start) of any array it was
given: the out-of-bounds check of the library's own kernels.  The detection
itself is shown by writes planted from the host into chosen guard words."""
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


def rand(ndim, n, seed, **kw):
    x1 = (1.0, 1.3) if ndim == 2 else (1.0, 1.3, 0.9)
    cfg = W.base_cfg(ndim, n, (0.0,) * ndim, x1, **kw)
    return cfg, W.random_state(cfg, seed)


MIXED_2D = ["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"]
MIXED_3D = ["periodic", "periodic", "outflow", "outflow", "outflow", "outflow"]

# (generator, seglens to run): 2D and 3D, every reconstruction, both solvers
# and edge-field forms, both RK orders, periodic / outflow / mixed axes, ragged
# sizes (so the used words of a field are not a multiple of 32), grids small
# enough for the side-by-side sweeps and large enough for the staged ones
SIM_CASES = {
    "ot2d-64-plm-hlld-rk2": (lambda: W.orszag_tang_2d(64), (None, 2, 256)),
    "ot2d-48-wenoz-ucthlld-rk3": (lambda: W.orszag_tang_2d(48, recon="wenoz", rk=3, emf="uct_hlld"), (None, 5)),
    "rand2d-37x23-ppm-hll-rk3-outflow": (lambda: rand(2, (37, 23), 1, recon="ppm", riemann="hll", rk=3,
                                                      bc="outflow"), (None, 3)),
    "rand2d-29x31-plm-hll-mixed": (lambda: rand(2, (29, 31), 2, bc=MIXED_2D), (None,)),
    "rand2d-300x17-wenoz-hlld-rk3": (lambda: rand(2, (300, 17), 3, recon="wenoz", rk=3), (None, 7)),
    "rand3d-13x11x9-wenoz-hlld-rk3-outflow": (lambda: rand(3, (13, 11, 9), 4, recon="wenoz", rk=3,
                                                           bc="outflow"), (None, 2)),
    "rand3d-17x12x10-ppm-hll-mixed": (lambda: rand(3, (17, 12, 10), 5, recon="ppm", riemann="hll",
                                                   bc=MIXED_3D), (None,)),
    "turb3d-24-plm-hlld-ucthlld": (lambda: W.turbulent_3d(24, seed=6, emf="uct_hlld"), (None, 4)),
    "blast3d-40x36x33-wenoz-rk3-floor": (lambda: W.blast_3d((40, 36, 33)), (None, 64)),
    "cpa3d-20-plm-hlld": (lambda: W.cpa_3d(20), (None,)),
    "glm2d-ot-40": (lambda: W.to_glm(*W.orszag_tang_2d(40, recon="wenoz", rk=3)), (None, 3)),
    "glm3d-rand-15x13x11-outflow": (lambda: W.to_glm(*rand(3, (15, 13, 11), 7, bc="outflow")), (None,)),
}


@pytest.mark.parametrize("case", list(SIM_CASES))
def test_no_launch_writes_outside_its_arrays(mhd, case):
    gen, seglens = SIM_CASES[case]
    cfg, st = gen()
    for seglen in seglens:
        g = mhd.Sim(cfg, st)
        assert g.check_guards() is None, "fresh context"
        if seglen:
            g.set_seglen(seglen)
        g.advance(4)
        g.step(0.25 * g.cfl_dt())
        g.get_conserved()
        assert g.status() == (0, -1)
        assert g.check_guards() is None, f"{case} seglen {seglen}"


def test_guards_across_the_other_entry_points(mhd):
    """Per-phase and fused launches, autotune (which saves and restores U^n),
    the div B monitor, set_prim, and the adjoint's forward, recompute and
    reverse passes on the context."""
    cfg, st = W.orszag_tang_2d(96)
    g = mhd.Sim(cfg, st)
    g.set_fused(False)
    g.advance(3)
    g.set_fused(True)
    g.advance(3)
    g.autotune()
    g.set_divb_check(1e-10)
    g.advance(2)
    assert g.check_guards() is None
    acfg, ast = W.adjoint_2d(40)
    a = mhd.Sim(acfg, ast)
    a.adjoint(9, None, ckpt_every=4)
    a.grad_prim()
    a.grad_conserved()
    assert a.check_guards() is None
    pcfg, pst = rand(3, (11, 14, 9), 8, recon="wenoz")
    p = mhd.Sim(pcfg, pst)
    out = p.get_conserved()
    rho = out["rho"]
    v = [out[k] / rho for k in ("mx", "my", "mz")]
    p.set_prim(rho, v, np.full_like(rho, 0.7), [out["b0"], out["b1"], out["b2"]])
    p.advance(3)
    assert p.check_guards() is None


def test_batch_guards(mhd):
    sizes = [12, 16, 33, 20, 48, 7, 31]
    members = W.ensemble_members(len(sizes), seed=4, sizes=(16,))
    cases = [W.ensemble_member_state(dict(m, n=n), recon="wenoz", rk=3) for n, m in zip(sizes, members)]
    bt = mhd.Batch([c for c, _ in cases], [s for _, s in cases])
    assert bt.check_guards() is None
    bt.step(5)
    bt.autotune()
    bt.step(2)
    for r in range(len(sizes)):
        bt.get_conserved(r)
    assert bt.check_guards() is None


@pytest.mark.parametrize("gen,parts", [
    (lambda: W.orszag_tang_2d(37), (2, 3, 1)),
    (lambda: rand(3, (19, 14, 11), 9, recon="wenoz", rk=3, bc="outflow"), (2, 2, 2)),
    (lambda: W.turbulent_3d(20, seed=3), (3, 1, 2)),
])
def test_domain_guards(mhd, gen, parts):
    cfg, st = gen()
    d = mhd.Domain(cfg, parts, st)
    assert d.check_guards() is None
    d.advance(4)
    d.get_conserved()
    assert d.check_guards() is None


def test_a_planted_write_is_found_where_it_was_made(mhd):
    cfg, st = rand(2, (21, 19), 10)
    g = mhd.Sim(cfg, st)
    nfields, used, after = g.guard_layout
    assert 22 * 20 <= used <= 40 * 40        # the 21 x 19 cells with ghost zones and a face row
    assert after >= 32 and (used + after) % 32 == 0
    for field, word in [(0, -1), (0, -32), (0, 0), (3, 5), (nfields - 1, after - 1), (nfields // 2, 31)]:
        h = mhd.Sim(cfg, st)
        h.advance(1)
        assert h.check_guards() is None
        h.inject_guard_write(field, word)
        assert h.check_guards() == (field, word)
        h.advance(2)                        # no launch reads the guard words
        assert h.status() == (0, -1)
        assert h.check_guards() == (field, word)
    h = mhd.Sim(cfg, st)
    h.inject_guard_write(4, 9)
    h.inject_guard_write(2, 30)
    assert h.check_guards() == (2, 30)      # the first damaged word in pool order
    for field, word in [(-1, 0), (nfields, 0), (0, -33), (1, -1), (0, after)]:
        with pytest.raises(mhd.MhdError) as err:
            h.inject_guard_write(field, word)
        assert err.value.code == -1
