"""Writes tests/golden/flops_per_unit.json: the oracle's algorithmic flop count
per unit of work, for each scheme variant the benchmark runs.

    python tests/golden/make_flops.py

Counting (oracle/scalar.hpp): +, -, *, / and sqrt count one flop, compare,
fabs, min, max count none, a*b+c counts two.  The oracle (counting scalar)
runs one CFL evaluation and one step of the workload at a small size; each
phase's count is divided by the number of units that phase processed, using
the oracle's own loop ranges:
  c2p       per padded cell, per primitive pass (stages + 1 CFL pass)
  recon     per reconstructed cell and direction (n_d + 2 cells x (n_t + 2) rows)
  riemann   per face (n_d + 1 faces x (n_t + 2) rows)
  fluxdiff  per interior cell and stage
  emf       per edge and stage
  ct        per evolved face and stage
  rk        per evolved element and stage
  cfl       per interior cell
WENO-Z recon counts the face-independent part of each face value (the
smoothness indicators, tau5, the ratios and 1 + ratio^2) once per cell and
variable, as the method needs it; the oracle's per-face count is kept beside
it (recon_per_face_count).
Each variant also gets the reverse-mode (adjoint) work per unit of the same
phases, from the oracle's tape on one step: the forward flops, plus the flops
that form the partial derivatives, plus the backward sweep over the tape
links (an add for a partial of +-1, a multiply-add otherwise).  The CFL phase
is not differentiated (dt frozen).
The GLM variants (divergence cleaning) are counted on the oracle's GLM scheme
with its own loop ranges: recon per cell and direction ((n_d + 2) cells x the
interior pencils), riemann per face (the (B_n, psi) solution and the MHD
solver), fluxdiff per cell and stage, rk per variable (9) and cell per stage.
Only this script writes the file, and it calls only oracle/.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_20337_b300 import workloads as W  # noqa: E402

VARIANTS = {
    "turbulent3d_plm_hlld_rk2": lambda: W.turbulent_3d(16, seed=1),
    "turbulent3d_plm_hll_rk2": lambda: W.turbulent_3d(16, seed=1, riemann="hll"),
    "blast3d_wenoz_hlld_rk3": lambda: W.blast_3d(16),
    "blast3d_ppm_hlld_rk3": lambda: W.blast_3d(16, recon="ppm"),
    "orszag_tang2d_plm_hlld_rk2": lambda: W.orszag_tang_2d(32),
    "orszag_tang2d_plm_hll_rk2": lambda: W.orszag_tang_2d(32, riemann="hll"),
    "orszag_tang2d_wenoz_hlld_rk3": lambda: W.orszag_tang_2d(32, recon="wenoz", rk=3),
    "orszag_tang3d_wenoz_hlld_rk3": lambda: W.orszag_tang_3d(16, recon="wenoz", rk=3),
    "cpa3d_wenoz_hlld_rk3": lambda: W.cpa_3d(16, recon="wenoz", rk=3),
    "orszag_tang3d_wenoz_hlld_rk3_ucthlld": lambda: W.orszag_tang_3d(16, recon="wenoz", rk=3, emf="uct_hlld"),
    "cpa3d_wenoz_hlld_rk3_ucthlld": lambda: W.cpa_3d(16, recon="wenoz", rk=3, emf="uct_hlld"),
    "adjoint2d_plm_hlld_rk2": lambda: W.adjoint_2d(32),
    "adjoint2d_plm_hll_rk2": lambda: W.adjoint_2d(32, riemann="hll"),
    "adjoint2d_wenoz_hlld_rk3_ucthlld": lambda: W.adjoint_2d(32, recon="wenoz", rk=3, emf="uct_hlld"),
}


def units(cfg):
    nd = cfg["ndim"]
    n = list(cfg["n"])
    G = 2 if cfg["recon"] == "plm" else 3
    rk = cfg["rk"]
    cells = int(np.prod(n))
    padded = int(np.prod([m + 2 * G for m in n]))
    recon = faces = 0
    for d in range(nd):
        rows = int(np.prod([n[t] + 2 for t in range(nd) if t != d]))
        recon += (n[d] + 2) * rows
        faces += (n[d] + 1) * rows
    # edges: 2D one E_z per vertex; 3D E_c over (n_a+1)(n_b+1) n_c
    if nd == 2:
        edges = (n[0] + 1) * (n[1] + 1)
    else:
        edges = sum(int(np.prod([n[e] + (1 if e != c else 0) for e in range(3)])) for c in range(3))
    periodic = [cfg["bc"][2 * d] == "periodic" for d in range(nd)]
    ct_faces = 0
    for d in range(nd):
        ct_faces += int(np.prod([n[e] + (1 if (e == d and not periodic[d]) else 0) for e in range(nd)]))
    elems = cells * (6 if nd == 2 else 5) + ct_faces
    return {"c2p": padded * (rk + 1), "recon": recon * rk, "riemann": faces * rk, "fluxdiff": cells * rk,
            "emf": edges * rk, "ct": ct_faces * rk, "rk": elems * rk, "cfl": cells}


# The scheme with GLM divergence cleaning (oracle/glm_oracle.hpp): its own
# loop ranges (interior pencils only, no edges or faces), 9 variables.
GLM_VARIANTS = {
    "turbulent3d_plm_hlld_rk2_glm": lambda: W.turbulent_3d(16, seed=1),
    "orszag_tang3d_wenoz_hlld_rk3_glm": lambda: W.orszag_tang_3d(16, recon="wenoz", rk=3),
}


def units_glm(cfg):
    nd = cfg["ndim"]
    n = list(cfg["n"])
    G = 2 if cfg["recon"] == "plm" else 3
    rk = cfg["rk"]
    cells = int(np.prod(n))
    padded = int(np.prod([m + 2 * G for m in n]))
    recon = faces = 0
    for d in range(nd):
        rows = int(np.prod([n[t] for t in range(nd) if t != d]))
        recon += (n[d] + 2) * rows
        faces += (n[d] + 1) * rows
    return {"c2p": padded * (rk + 1), "recon": recon * rk, "riemann": faces * rk, "fluxdiff": cells * rk,
            "rk": 9 * cells * rk, "cfl": cells}


def glm_counts(cfg, st):
    bx, by, bz = W.cell_field(cfg, st["b0"], st["b1"], st["b2"])
    g = {k: st[k] for k in ("rho", "mx", "my", "mz", "E")}
    g.update(bx=bx, by=by, bz=bz, psi=np.zeros_like(bx))
    o = oracle.OracleGlm(cfg, g)
    dt = o.cfl_dt()
    return o.count_flops(1, dt)


def wenoz_once_per_cell(cfg, per, nvar):
    """WENO-Z: the oracle forms each face value as the formula states it, so
    the indicators, tau5, the ratios and 1 + ratio^2 -- the same for the two
    faces of a cell -- are counted twice per cell and variable.  The method's
    work forms them once: per["recon"] becomes that count (the oracle's count
    less one Counted run of those sub-expressions per reconstructed variable),
    and the oracle's own count is kept as per["recon_per_face_count"].
    nvar reconstructed variables per cell: 7 (rho, v, the two transverse B, p)
    for CT, 9 (all of B and psi) for GLM."""
    if cfg["recon"] != "wenoz":
        return
    shared = oracle.count_wenoz_shared()
    per["recon_per_face_count"] = per["recon"]
    per["wenoz_shared_per_variable"] = shared
    per["recon"] = per["recon"] - nvar * shared


def main():
    out = {"convention": "flops per unit: +,-,*,/,sqrt = 1; a*b+c = 2; compare/abs/min/max = 0",
           "variants": {}}
    for name, make in VARIANTS.items():
        cfg, st = make()
        dt = oracle.OracleSim(cfg, st).cfl_dt()
        counts = oracle.count_flops(cfg, st, 1, dt)
        u = units(cfg)
        per = {}
        for ph in ("c2p", "recon", "riemann", "fluxdiff", "emf", "ct", "rk", "cfl"):
            tot = sum(counts[ph].values())
            per[ph] = tot / u[ph]
        per["div_sqrt_per_face"] = (counts["riemann"]["div"] + counts["riemann"]["sqrt"]) / u["riemann"]
        wenoz_once_per_cell(cfg, per, nvar=7)
        tape = oracle.count_tape(cfg, st, 1, dt)
        adj = {}
        for ph in ("c2p", "recon", "riemann", "fluxdiff", "emf", "ct", "rk"):
            links, pfl = tape[ph]
            fwd = sum(counts[ph].values())
            # the counting run's c2p units include the CFL pass, which the tape run does not make
            u_adj = u[ph] * cfg["rk"] / (cfg["rk"] + 1) if ph == "c2p" else u[ph]
            adj[ph] = (fwd * u_adj / u[ph] + pfl + links) / u_adj
        out["variants"][name] = {"config": {k: cfg[k] for k in ("ndim", "n", "recon", "riemann", "rk", "bc", "emf")},
                                 "per_unit": per, "adjoint_per_unit": adj}
    for name, make in GLM_VARIANTS.items():
        cfg, st = make()
        counts = glm_counts(cfg, st)
        u = units_glm(cfg)
        per = {ph: sum(counts[ph].values()) / u[ph] for ph in ("c2p", "recon", "riemann", "fluxdiff", "rk", "cfl")}
        wenoz_once_per_cell(cfg, per, nvar=9)
        out["variants"][name] = {"config": {k: cfg[k] for k in ("ndim", "n", "recon", "riemann", "rk", "bc")},
                                 "divb": "glm", "per_unit": per}
    path = os.path.join(HERE, "flops_per_unit.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(path)


if __name__ == "__main__":
    main()
