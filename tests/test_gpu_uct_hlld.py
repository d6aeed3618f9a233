"""The UCT-HLLD edge field (emf="uct_hlld") on the GPU against the oracle:
the sweeps' HLLD weights face by face over every region of the wave fan, one
step to 1e-12, twenty steps and 100 CFL steps to 1e-10 (normwise per array),
the CFL step bitwise; plus properties that hold at any size (the plane-parallel CT B_y =
finite-volume B_z identity, conservation, div B, segment-length invariance),
the batched and allocation-free entry points equal to the context API
bitwise, and the configurations that must be refused."""
import numpy as np
import pytest

import oracle
from paper_2511_20337_b300 import workloads as W
from conftest import relerr
from test_oracle_uct_hlld import plane_parallel_state, random_pair, region

pytestmark = pytest.mark.gpu

KEYS = oracle.KEYS
G = 5.0 / 3.0


@pytest.fixture(scope="module")
def mhd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20337_b300 import mhd as M
    M.lib()
    return M


def test_face_weights_match_oracle_in_every_region(mhd):
    """Flux to 1e-13 and weights to 1e-11 of their size (the GPU forms its
    reciprocals and square roots by refined seeds, so its wave speeds differ
    from the oracle's by an ulp; the weights are continuous across the region
    boundaries of the rotational fan)."""
    rng = np.random.default_rng(2511)
    pairs = [random_pair(rng, t) for t in range(4000)]
    x = np.array([np.concatenate([wl, wr, [bn]]) for wl, wr, bn in pairs])
    F, ing = mhd.probe_riemann("hlld", x, G, emf="uct_hlld")
    Fh, ingh = mhd.probe_riemann("hlld", x, G)
    np.testing.assert_array_equal(F, Fh)  # the weights do not change the flux
    seen = {}
    for f, (wl, wr, bn) in enumerate(pairs):
        Fo, io = oracle.riemann("hlld", wl, wr, bn, G, emf="uct_hlld")
        r = region(io)
        seen[r] = seen.get(r, 0) + 1
        fscale = np.max(np.abs(Fo)) + 1e-300
        assert np.max(np.abs(F[f] - Fo)) <= 1e-13 * fscale, (f, r)
        wscale = 1.0 + np.sum(np.abs(io))
        assert np.max(np.abs(ing[f] - io)) <= 1e-11 * wscale, (f, r, ing[f], io)
        # the GPU's own weights reproduce the GPU's transverse flux
        for iB, iv in ((4, 2), (5, 3)):
            FL = wl[1] * wl[iB] - bn * wl[iv]
            FR = wr[1] * wr[iB] - bn * wr[iv]
            aL, aR, dL, dR = ing[f][0], ing[f][1], ing[f][2], ing[f][5]
            dec = aL * FL + aR * FR + dL * wl[iB] - dR * wr[iB]
            size = abs(aL * FL) + abs(aR * FR) + abs(dL * wl[iB]) + abs(dR * wr[iB]) + abs(F[f][iB]) + 1e-300
            assert abs(dec - F[f][iB]) <= 1e-13 * size, (f, r, iB)
    for r in ("left", "right", "star-left", "star-right", "double-star"):
        assert seen.get(r, 0) >= 30, seen
    # UCT-HLL ingredients: d^R repeats d
    np.testing.assert_array_equal(ingh[:, 5], ingh[:, 2])


def uct(cfg, st):
    return dict(cfg, emf="uct_hlld"), st


CASES = {
    "ot2d-48-plm-rk2": lambda: W.orszag_tang_2d(48, emf="uct_hlld"),
    "rand2d-31x35-wenoz-rk3": lambda: uct(*(lambda c: (c, W.random_state(c, 3)))(
        W.base_cfg(2, (31, 35), (0, 0), (1, 1), recon="wenoz", rk=3))),
    "rand3d-13x11x9-plm-rk2": lambda: uct(*(lambda c: (c, W.random_state(c, 5)))(
        W.base_cfg(3, (13, 11, 9), (0, 0, 0), (1, 1, 1)))),
    "rand3d-9x10x11-ppm-rk3-outflow": lambda: uct(*(lambda c: (c, W.random_state(c, 7)))(
        W.base_cfg(3, (9, 10, 11), (0, 0, 0), (1, 1, 1), recon="ppm", rk=3, bc="outflow"))),
    "ot3d-24-wenoz-rk3": lambda: W.orszag_tang_3d(24, recon="wenoz", rk=3, emf="uct_hlld"),
    "cpa3d-16-wenoz-rk3": lambda: W.cpa_3d(16, recon="wenoz", rk=3, emf="uct_hlld"),
    "turb3d-24-plm-rk2": lambda: W.turbulent_3d(24, seed=11, emf="uct_hlld"),
}


def compare(out, ref, tol, what):
    """Normwise per array; a face field relative to the largest field
    component (the 3D Orszag-Tang B_z starts at zero, and its round-off
    scales with |B|)."""
    bmax = max(np.max(np.abs(ref[k])) for k in ("b0", "b1", "b2"))
    for k in KEYS:
        if k in ("b0", "b1", "b2"):
            err = np.max(np.abs(out[k] - ref[k])) / bmax
        else:
            err = relerr(out[k], ref[k])
        assert err <= tol, (what, k, err)


@pytest.mark.parametrize("case", list(CASES))
def test_one_step_matches_oracle(mhd, case):
    cfg, st = CASES[case]()
    o = oracle.OracleSim(cfg, st)
    dt = o.cfl_dt()
    o.step(dt)
    g = mhd.Sim(cfg, st)
    assert g.cfl_dt() == dt
    g.step(dt)
    compare(g.get_conserved(), o.get_state(), 1e-12, case)
    assert g.counters()[0] == o.fallbacks


@pytest.mark.parametrize("case", ["ot2d-48-plm-rk2", "rand3d-9x10x11-ppm-rk3-outflow", "ot3d-24-wenoz-rk3",
                                  "turb3d-24-plm-rk2"])
def test_twenty_steps_match_oracle(mhd, case):
    cfg, st = CASES[case]()
    o = oracle.OracleSim(cfg, st)
    dts = o.advance(20, record_dt=True)
    g = mhd.Sim(cfg, st)
    for dt in dts:
        g.step(dt)
    compare(g.get_conserved(), o.get_state(), 1e-10, case)
    # and the edge weights matter: the UCT-HLL run is a different solution
    h = mhd.Sim(dict(cfg, emf="uct_hll"), st)
    for dt in dts:
        h.step(dt)
    assert relerr(h.get_conserved()["b0"], g.get_conserved()["b0"]) > 1e-9


def test_orszag_tang_2d_128_100_steps(mhd):
    """The 2D Orszag-Tang workload (128^2, PLM + HLLD + RK2, CFL 0.4) with the
    HLLD edge weights: 100 CFL steps each side with its own dt, state within
    1e-10, time to round-off."""
    cfg, st = W.orszag_tang_2d(128, emf="uct_hlld")
    o = oracle.OracleSim(cfg, st)
    o.advance(100)
    g = mhd.Sim(cfg, st)
    g.advance(100)
    compare(g.get_conserved(), o.get_state(), 1e-10, "OT 100 steps")
    assert abs(g.time - o.time) <= 1e-13 * o.time


@pytest.mark.parametrize("rk", [2, 3])
def test_plane_parallel_staggered_by_matches_cell_bz(mhd, rk):
    """B_n = 0 and a profile varying along x only: the CT-evolved face B_y
    equals the finite-volume cell B_z to round-off (exact in exact arithmetic
    with the HLLD weights, not with the HLL ones)."""
    cfg, st = plane_parallel_state(200, 3)
    cfg = dict(cfg, rk=rk)
    gaps = {}
    for emf in ("uct_hlld", "uct_hll"):
        g = mhd.Sim(dict(cfg, emf=emf), st)
        g.advance(100)
        out = g.get_conserved()
        by, bz = out["b1"][0, 0, :], out["b2"][0, 0, :]
        assert np.all(out["b1"][0] == by)
        gaps[emf] = np.max(np.abs(by - bz)) / np.max(np.abs(bz))
    assert gaps["uct_hlld"] <= 1e-13, gaps
    assert gaps["uct_hll"] >= 1e-5, gaps


def test_conservation_div_b_and_segment_length(mhd):
    from test_oracle_scheme import div_b, totals
    cfg, st = W.orszag_tang_3d(40, recon="wenoz", rk=3, emf="uct_hlld")
    outs = []
    for seg in (3, 64):
        g = mhd.Sim(cfg, st)
        g.set_seglen(seg)
        g.advance(5)
        outs.append(g.get_conserved())
    for k in KEYS:
        np.testing.assert_array_equal(outs[0][k], outs[1][k], err_msg=k)
    t0, t1 = totals(cfg, st), totals(cfg, outs[0])
    for k in t0:
        assert abs(t1[k][0] - t0[k][0]) <= 1e-13 * max(t0[k][1], t1[k][1], 1e-300), k
    div, scale = div_b(cfg, outs[0])
    assert div <= 1e-12 * scale


def test_batch_equals_single_grid_runs_bitwise(mhd):
    members = W.ensemble_members(5, seed=4, sizes=(16,))
    cases = [W.ensemble_member_state(dict(m, n=n), emf="uct_hlld") for n, m in zip([12, 33, 20, 48, 7], members)]
    bt = mhd.Batch([c for c, _ in cases], [s for _, s in cases])
    bt.step(6)
    for r, (cfg, st) in enumerate(cases):
        g = mhd.Sim(cfg, st)
        g.advance(6)
        out = g.get_conserved()
        got = bt.get_conserved(r)
        for k in KEYS:
            np.testing.assert_array_equal(got[k], out[k], err_msg=f"run {r}: {k}")
    with pytest.raises(mhd.MhdError):  # one scheme per batch
        mhd.Batch([cases[0][0], dict(cases[1][0], emf="uct_hll")])


def test_noalloc_equals_context_step(mhd):
    import torch
    cfg, st = W.turbulent_3d((12, 10, 8), seed=3, recon="wenoz", rk=3, emf="uct_hlld")
    sim = mhd.Sim(cfg, st)
    dt = sim.cfl_dt()
    sim.step(dt)
    ref = sim.get_conserved()
    dev = {k: torch.from_numpy(np.ascontiguousarray(st[k])).cuda() for k in KEYS}
    mhd.step_noalloc(cfg, dev, dt)
    torch.cuda.synchronize()
    for k in KEYS:
        np.testing.assert_array_equal(dev[k].cpu().numpy(), ref[k], err_msg=k)


def test_refused_configurations(mhd):
    cfg, st = W.orszag_tang_2d(32)
    with pytest.raises(mhd.MhdError):  # the HLL solver has no HLLD weights
        mhd.Sim(dict(cfg, riemann="hll", emf="uct_hlld"))
    with pytest.raises(mhd.MhdError):  # no edge fields under GLM
        mhd.Sim(dict(cfg, divb="glm", glm_alpha=0.1, emf="uct_hlld"))
    g = mhd.Sim(dict(cfg, emf="uct_hlld"), st)
    J, dts = g.adjoint(2)  # the adjoint transposes the UCT-HLLD edge fields too
    assert np.isfinite(J) and len(dts) == 2
