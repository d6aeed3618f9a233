"""The div B monitor (mhd_set_divb_check / mhd_divb, MHD_ERR_DIVB).

Constrained transport keeps the discrete divergence of the face field at
round-off (paper §2.2), so on clean runs the monitor stays silent; a face
value corrupted on the host breaks div B = 0 at the two cells sharing that
face, CT carries the error along unchanged, and the monitor reports it with
one of those cells.  Its value is checked against numpy on the face arrays."""
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


def divb_rel_numpy(cfg, st):
    """max_c |div B| h / max_c |B_c| from the state's face arrays."""
    nd = cfg["ndim"]
    dx = [(cfg["x1"][d] - cfg["x0"][d]) / cfg["n"][d] for d in range(nd)]
    bx, by, bz = st["b0"], st["b1"], st["b2"]
    div = (bx[..., 1:] - bx[..., :-1]) / dx[0] + (by[..., 1:, :] - by[..., :-1, :]) / dx[1]
    cx, cy = 0.5 * (bx[..., 1:] + bx[..., :-1]), 0.5 * (by[..., 1:, :] + by[..., :-1, :])
    if nd == 3:
        div = div + (bz[1:] - bz[:-1]) / dx[2]
        cz = 0.5 * (bz[1:] + bz[:-1])
    else:
        cz = bz
    return np.max(np.abs(div)) * min(dx) / np.sqrt(np.max(cx * cx + cy * cy + cz * cz))


CLEAN = {
    "ot2d-64": lambda: W.orszag_tang_2d(64),
    "blast3d-20-outflow": lambda: W.blast_3d(20),
    "turb3d-16": lambda: W.turbulent_3d(16, seed=2),
    "ot3d-16-ucthlld": lambda: W.orszag_tang_3d(16, recon="wenoz", rk=3, emf="uct_hlld"),
}


@pytest.mark.parametrize("case", list(CLEAN))
def test_monitor_is_silent_on_clean_runs(mhd, case):
    cfg, st = CLEAN[case]()
    g = mhd.Sim(cfg, st)
    g.set_divb_check(1e-12)
    g.advance(20)
    assert g.status() == (0, -1)
    assert g.divb() <= 1e-12
    out = g.get_conserved()
    assert divb_rel_numpy(cfg, out) <= 1e-12


@pytest.mark.parametrize("ndim", [2, 3])
def test_monitor_reports_a_corrupted_face(mhd, ndim):
    if ndim == 2:
        cfg, st = W.orszag_tang_2d(32)
        j, i = 11, 17
        st = {k: v.copy() for k, v in st.items()}
        st["b0"][0, j, i] += 1e-6                       # face between cells i-1 and i of row j
        cells = {j * 32 + i - 1, j * 32 + i}
    else:
        cfg, st = W.turbulent_3d(12, seed=4)
        k, j, i = 5, 3, 7
        st = {q: v.copy() for q, v in st.items()}
        st["b1"][k, j, i] -= 1e-6                       # face between cells j-1 and j
        cells = {(k * 12 + j - 1) * 12 + i, (k * 12 + j) * 12 + i}
    g = mhd.Sim(cfg, st)
    rel0 = g.divb()
    assert rel0 == pytest.approx(divb_rel_numpy(cfg, st), rel=1e-6)
    assert rel0 > 1e-9
    g.step(1e-4)                                        # monitor off: no error
    assert g.status()[0] == 0
    g.set_divb_check(1e-12)
    g.advance(2)
    rc, bad = g.status()
    assert rc == -8 and bad in cells, (rc, bad, cells)
    assert g.status()[0] == 0                           # cleared
    # CT carries the divergence along unchanged; the ratio moves only with max |B_c|
    assert g.divb() == pytest.approx(rel0, rel=2e-2)


def test_monitor_refuses_glm_and_bad_tolerances(mhd):
    cfg, st = W.turbulent_3d(12, seed=1)
    g = mhd.Sim(cfg, st)
    for tol in (-1.0, float("nan"), float("inf")):
        with pytest.raises(mhd.MhdError):
            g.set_divb_check(tol)
    gcfg, gst = W.to_glm(cfg, st)
    h = mhd.Sim(gcfg, gst)
    with pytest.raises(mhd.MhdError):
        h.set_divb_check(1e-12)
    with pytest.raises(mhd.MhdError):
        h.divb()
