"""Sampled-window oracle for full-size parity checks.

One RK step changes a cell only through a bounded stencil (per stage: the
reconstruction and Riemann stencil plus the edge-field stencil, under 6 cells
for WENO-Z / PPM).  So the oracle's result for the cells of a small box equals
its full-grid result if it steps the box together with a halo wider than the
dependency radius of the step, taken from the full initial state (wrapped on
periodic axes).  On axes where the box reaches a physical (outflow) boundary the
real boundary is used; elsewhere the halo's outer edge gets an outflow
condition that cannot reach the box within one step.
"""
import numpy as np

import oracle

KEYS = oracle.KEYS


def halo_for(cfg):
    """Halo covering the dependency radius of one step: about 4 cells per stage
    (reconstruction stencil 3 plus the edge-field stencil), plus one."""
    return 4 * cfg["rk"] + 1


def _pow2(w):
    p = 1
    while p < w:
        p *= 2
    return p


def extract(cfg, state, lo, size, halo):
    """Window config and state: cells [lo - halo, lo + size + halo) per axis,
    widened to a power-of-two width (so that width * dx is exact and the
    window's dx equals the grid's to the bit), wrapped on periodic axes and
    clipped at outflow boundaries; an axis that cannot be windowed is taken
    whole with the grid's own bounds.  Returns (wcfg, wstate, offsets) with offsets
    the per-axis position of the box inside the window."""
    nd = cfg["ndim"]
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    if nd == 2:
        n[2] = 1
    x0 = list(cfg["x0"]) + [0.0]
    x1 = list(cfg["x1"]) + [1.0]
    dx = [(x1[d] - x0[d]) / n[d] for d in range(3)]
    idx, inner, bc, wn, wx0, wx1 = [], [], [], [], [], []
    for d in range(nd):
        periodic = cfg["bc"][2 * d] == "periodic"
        a, b = lo[d] - halo, lo[d] + size[d] + halo
        if not periodic:
            a, b = max(a, 0), min(b, n[d])
        p = _pow2(b - a)
        whole = p >= n[d]
        if not whole:
            if periodic or a + p <= n[d]:
                b = a + p            # widen on the high side (wrapping if periodic)
            elif b - p >= 0:
                a = b - p            # widen on the low side
            else:
                whole = True
        if whole:
            a, b = 0, n[d]
            bc += [cfg["bc"][2 * d], cfg["bc"][2 * d + 1]]
            wx0.append(x0[d])
            wx1.append(x1[d])
        else:
            bl = cfg["bc"][2 * d] if (not periodic and a == 0) else "outflow"
            br = cfg["bc"][2 * d + 1] if (not periodic and b == n[d]) else "outflow"
            bc += [bl, br]
            wx0.append(0.0)
            wx1.append(p * dx[d])
        idx.append(np.arange(a, b))
        inner.append(lo[d] - a)
        wn.append(b - a)
    wcfg = dict(cfg)
    wcfg["n"] = tuple(wn)
    wcfg["x0"] = tuple(wx0)
    wcfg["x1"] = tuple(wx1)
    wcfg["bc"] = bc + ["periodic"] * (6 - len(bc))

    def take(a, face_axis):
        sl, gathers = [slice(None)] * a.ndim, []
        for d in range(nd):
            ax = 2 - d  # arrays are [z][y][x]
            ids = idx[d]
            if d == face_axis:
                ids = np.concatenate([ids, ids[-1:] + 1])
            if cfg["bc"][2 * d] == "periodic":
                ids = ids % n[d]   # the duplicate last face of a periodic axis is face 0
            if ids[-1] - ids[0] == len(ids) - 1:
                sl[ax] = slice(int(ids[0]), int(ids[-1]) + 1)   # a plain range: a view
            else:
                gathers.append((ax, ids))
        out = a[tuple(sl)]
        for ax, ids in gathers:  # wrapped ranges, on the already reduced array
            out = np.take(out, ids, axis=ax)
        return out

    ws = {}
    glm = cfg.get("divb", "ct") == "glm"
    for q, k in enumerate(oracle.GLM_KEYS if glm else KEYS):
        fa = q - 5 if (not glm and q >= 5 and (q - 5) < nd) else -1  # GLM: every field is cell-centred
        ws[k] = np.ascontiguousarray(take(state[k], fa))
    return wcfg, ws, inner


def window_step(cfg, state, lo, size, halo, dt):
    """Oracle values of the cells (and their left faces) of the box after one
    step of dt (the GLM scheme's oracle when cfg has divb = glm)."""
    wcfg, ws, offs = extract(cfg, state, lo, size, halo)
    if cfg.get("divb", "ct") == "glm":
        s = oracle.OracleGlm(wcfg, ws, alpha=cfg["glm_alpha"])
        keys = oracle.GLM_KEYS
    else:
        s = oracle.OracleSim(wcfg, ws)
        keys = KEYS
    s.step(dt)
    out = s.get_state()
    return {k: box(out[k], offs, size, wcfg["n"]) for k in keys}


def box(a, lo, size, n):
    """Cells (or left faces) [lo, lo + size) per axis of an array, indices
    taken modulo the cell count n (the last face of a periodic axis is face 0)."""
    out = a
    for d in range(len(size)):
        ids = np.arange(lo[d], lo[d] + size[d]) % n[d]
        out = np.take(out, ids, axis=2 - d)
    return out


def blockwise_cfl_dt(cfg, state, block=64):
    """The oracle's CFL step of the whole grid, taken block by block: each
    block's oracle returns C / (its largest cell rate), a cell's rate depending
    on that cell alone; division rounded to nearest is monotone, so the least
    block step is C / (the grid's largest rate), to the bit.  Keeps the oracle's
    memory to one block for grids far larger than a test would hold whole."""
    nd = cfg["ndim"]
    glm = cfg.get("divb", "ct") == "glm"
    starts = [range(0, cfg["n"][d], block) for d in range(nd)]
    best = None
    for lo in np.array(np.meshgrid(*starts, indexing="ij")).reshape(nd, -1).T:
        size = [min(block, cfg["n"][d] - int(lo[d])) for d in range(nd)]
        wcfg, ws, _ = extract(cfg, state, [int(v) for v in lo], size, 0)
        if list(wcfg["n"][:nd]) != size:
            raise ValueError("block sizes must be powers of two dividing the grid")
        o = oracle.OracleGlm(wcfg, ws) if glm else oracle.OracleSim(wcfg, ws)
        dt = o.cfl_dt()
        best = dt if best is None else min(best, dt)
    return best
