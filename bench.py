"""Benchmark: FP64 cell-updates per second of the ideal-MHD CT step on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one full time step of the workload (CFL dt computed on the device,
then every RK stage: ghost fill, primitive recovery, three fused
reconstruct -> Riemann -> flux-difference sweeps, UCT edge fields, CT + RK
combine).  `value` is cell-updates per second with the state resident in HBM;
`e2e` is the same metric through the C-ABI with the state copied from pinned
host memory before, and read back after, every step.  Under torchrun each rank
runs its own replica (the step is not sharded across GPUs): value = all ranks'
cell-updates / max rank time.

The default workload is the 512^3 magnetised blast (WENO-Z + HLLD + SSP-RK3 +
UCT CT, outflow).  After its plain step, the same run measures the batched
ensemble (256 2D runs in one graph per step) and the adjoint (a 400-step
gradient of a 256^2 run) on the same GPU and adds them to the one JSON line as
batched_vs_plain and adjoint_vs_plain, each with its own cell-updates/s, its
roofline fraction and its ratio to the plain step (--no-companions skips them).

--impl reference times the FP64 CPU oracle on the host cores, on a bounded
sample of the same workload (a smaller grid of the same kind), same metric.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2511_20337_b300 import workloads as W  # noqa: E402

METRIC = "FP64 cell-updates/s per B300"
UNIT = "cell-updates/s"

WORKLOADS = {
    # name: (generator, flops variant, description)
    "turbulent3d-256": (lambda: W.turbulent_3d(256), "turbulent3d_plm_hlld_rk2",
                        "3D ideal MHD 256^3 periodic, uniform rho=1 p=1 B=(1,1,1)/sqrt3 + seeded Gaussian "
                        "rho/v perturbations (1%, |k|<=8); PLM-minmod + HLLD + SSP-RK2 + UCT-HLL CT, CFL 0.4"),
    "turbulent3d-512": (lambda: W.turbulent_3d(512), "turbulent3d_plm_hlld_rk2",
                        "3D ideal MHD 512^3 periodic, the turbulent3d-256 recipe and scheme at 512^3 "
                        "(PLM-minmod + HLLD + SSP-RK2 + UCT-HLL CT, CFL 0.4)"),
    "turbulent3d-128": (lambda: W.turbulent_3d(128), "turbulent3d_plm_hlld_rk2",
                        "3D ideal MHD 128^3 periodic (profiling size), same recipe and scheme as turbulent3d-256"),
    "blast3d-512": (lambda: W.blast_3d(512), "blast3d_wenoz_hlld_rk3",
                    "3D magnetised blast 512^3 outflow, rho=1, p=0.1 / 10 (r<=0.1), B=10/sqrt2 (1,1,0); "
                    "WENO-Z + HLLD + SSP-RK3 + UCT-HLL CT, CFL 0.4"),
    "blast3d-128": (lambda: W.blast_3d(128), "blast3d_wenoz_hlld_rk3",
                    "3D magnetised blast 128^3 (profiling size), same setup and scheme as blast3d-512"),
    "blast3d-512-ppm": (lambda: W.blast_3d(512, recon="ppm"), "blast3d_ppm_hlld_rk3",
                        "3D magnetised blast 512^3 outflow; PPM + HLLD + SSP-RK3 + UCT-HLL CT, CFL 0.4"),
    "blast3d-128-ppm": (lambda: W.blast_3d(128, recon="ppm"), "blast3d_ppm_hlld_rk3",
                        "3D magnetised blast 128^3 (profiling size), same setup and scheme as blast3d-512-ppm"),
    "orszag-tang3d-704": (lambda: W.orszag_tang_3d((704, 704, 352), recon="wenoz", rk=3, emf="uct_hlld"),
                          "orszag_tang3d_wenoz_hlld_rk3_ucthlld",
                          "3D Orszag-Tang of paper §4.1 at its per-node resolution 704x704x352 on the unit periodic cube, "
                          "rho = 25/9, p = 5/3; WENO-Z + HLLD + SSP-RK3 + CT with UCT-HLLD edge fields (the paper's "
                          "scheme), CFL 0.4"),
    "orszag-tang3d-704-ucthll": (lambda: W.orszag_tang_3d((704, 704, 352), recon="wenoz", rk=3),
                                 "orszag_tang3d_wenoz_hlld_rk3",
                                 "orszag-tang3d-704 with UCT-HLL instead of UCT-HLLD edge fields"),
    "orszag-tang3d-128": (lambda: W.orszag_tang_3d(128, recon="wenoz", rk=3, emf="uct_hlld"),
                          "orszag_tang3d_wenoz_hlld_rk3_ucthlld",
                          "3D Orszag-Tang 128^3 (profiling size), same setup and scheme as orszag-tang3d-704"),
    "cpa3d-704": (lambda: W.cpa_3d((704, 704, 352), recon="wenoz", rk=3, emf="uct_hlld"), "cpa3d_wenoz_hlld_rk3_ucthlld",
                  "3D circularly polarised Alfven wave of paper §4.2 at 704x704x352 on the unit periodic cube, "
                  "eps = 0.1, rho0 = 1, p0 = 0.1, k = 2 pi (1,1,1); WENO-Z + HLLD + SSP-RK3 + CT with UCT-HLLD edge "
                  "fields (the paper's scheme), CFL 0.4"),
    "turbulent3d-128-glm": (lambda: W.to_glm(*W.turbulent_3d(128)), "turbulent3d_plm_hlld_rk2_glm",
                            "turbulent3d-128 with GLM divergence cleaning (profiling size), same scheme as "
                            "turbulent3d-256-glm"),
    "turbulent3d-256-glm": (lambda: W.to_glm(*W.turbulent_3d(256)), "turbulent3d_plm_hlld_rk2_glm",
                            "turbulent3d-256 with GLM divergence cleaning instead of CT (cell-centred B, psi, "
                            "alpha = 0.1); PLM-minmod + HLLD + SSP-RK2, CFL 0.4"),
    "orszag-tang3d-704-glm": (lambda: W.to_glm(*W.orszag_tang_3d((704, 704, 352), recon="wenoz", rk=3)),
                              "orszag_tang3d_wenoz_hlld_rk3_glm",
                              "3D Orszag-Tang of paper §4.1 at 704x704x352 with GLM divergence cleaning (the "
                              "paper's strong-scaling configuration); WENO-Z + HLLD + SSP-RK3, alpha = 0.1, CFL 0.4"),
    "orszag-tang3d-128-glm": (lambda: W.to_glm(*W.orszag_tang_3d(128, recon="wenoz", rk=3)),
                              "orszag_tang3d_wenoz_hlld_rk3_glm",
                              "3D Orszag-Tang 128^3 with GLM (profiling size), same setup and scheme as "
                              "orszag-tang3d-704-glm"),
    "orszag-tang2d-128": (lambda: W.orszag_tang_2d(128), "orszag_tang2d_plm_hlld_rk2",
                          "2D Orszag-Tang 128^2 periodic; PLM-minmod + HLLD + SSP-RK2 + UCT-HLL CT, CFL 0.4"),
    "ensemble2d-256": (None, "orszag_tang2d_plm_hlld_rk2",
                       "256 independent 2D Orszag-Tang runs (sizes from {64..512}^2, plasma beta in [0.1,10] and "
                       "Mach in [0.5,3] log-uniform, numpy default_rng(4)), PLM-minmod + HLLD + SSP-RK2 + UCT-HLL CT, "
                       "CFL 0.4, per-run CFL dt; batched launches in one CUDA graph, autotuned segment lengths"),
    "adjoint2d-256": (lambda: W.adjoint_2d(256), "adjoint2d_plm_hlld_rk2",
                      "adjoint: 2D 256^2 periodic unit square, rho = 1 + 0.05 g, v = 0.05 (g_x, g_y, 0), p = 1, "
                      "B = (1, 0.5, 0), Gaussian random fields 1 <= |k| <= 6 from numpy default_rng(5); "
                      "PLM-minmod + HLLD + SSP-RK2 + UCT-HLL CT, 400 CFL steps (dt recorded, then frozen); "
                      "gradient of the final magnetic energy w.r.t. the initial rho and v, checkpoints every 20 steps"),
    "adjoint2d-256-hll": (lambda: W.adjoint_2d(256, riemann="hll"), "adjoint2d_plm_hll_rk2",
                          "adjoint2d-256 with the HLL Riemann solver"),
    "adjoint2d-256-paper": (lambda: W.adjoint_2d(256, recon="wenoz", rk=3, emf="uct_hlld"),
                            "adjoint2d_wenoz_hlld_rk3_ucthlld",
                            "adjoint2d-256 with the paper's scheme: WENO-Z + HLLD + SSP-RK3 + UCT-HLLD"),
}
ADJOINT_STEPS, ADJOINT_CKPT = 400, 20
# The paper's single-node FP64 3D Orszag-Tang throughput per GPU (its per-node figures over 4 GPUs), quoted
# as context: same workload class on other hardware, with UCT-HLLD edge fields.
PAPER_PER_GPU = {"orszag-tang3d-704": {"H100 (MareNostrum 5 ACC)": 1.511e8 / 4, "A100 64 GB (Leonardo Booster)": 1.118e8 / 4}}
# CPU-oracle sample of each workload: the same kind of state on a smaller grid
SAMPLES = {
    "turbulent3d-256": (lambda: W.turbulent_3d(48), "turbulent 3D 48^3 (same scheme and field recipe)"),
    "turbulent3d-128": (lambda: W.turbulent_3d(48), "turbulent 3D 48^3 (same scheme and field recipe)"),
    "turbulent3d-512": (lambda: W.turbulent_3d(48), "turbulent 3D 48^3 (same scheme and field recipe)"),
    "blast3d-512": (lambda: W.blast_3d(32), "blast 3D 32^3 (same scheme and setup)"),
    "blast3d-128": (lambda: W.blast_3d(32), "blast 3D 32^3 (same scheme and setup)"),
    "blast3d-512-ppm": (lambda: W.blast_3d(32, recon="ppm"), "blast 3D 32^3 PPM (same scheme and setup)"),
    "blast3d-128-ppm": (lambda: W.blast_3d(32, recon="ppm"), "blast 3D 32^3 PPM (same scheme and setup)"),
    "orszag-tang3d-128-glm": (lambda: W.to_glm(*W.orszag_tang_3d(32, recon="wenoz", rk=3)),
                              "3D Orszag-Tang 32^3 with GLM (same scheme)"),
    "orszag-tang3d-704": (lambda: W.orszag_tang_3d(32, recon="wenoz", rk=3, emf="uct_hlld"),
                          "3D Orszag-Tang 32^3 (same scheme)"),
    "orszag-tang3d-704-ucthll": (lambda: W.orszag_tang_3d(32, recon="wenoz", rk=3), "3D Orszag-Tang 32^3 (same scheme)"),
    "orszag-tang3d-128": (lambda: W.orszag_tang_3d(32, recon="wenoz", rk=3, emf="uct_hlld"),
                          "3D Orszag-Tang 32^3 (same scheme)"),
    "cpa3d-704": (lambda: W.cpa_3d(32, recon="wenoz", rk=3, emf="uct_hlld"), "3D CPA 32^3 (same scheme)"),
    "turbulent3d-256-glm": (lambda: W.to_glm(*W.turbulent_3d(48)), "turbulent 3D 48^3 with GLM (same scheme)"),
    "turbulent3d-128-glm": (lambda: W.to_glm(*W.turbulent_3d(48)), "turbulent 3D 48^3 with GLM (same scheme)"),
    "orszag-tang3d-704-glm": (lambda: W.to_glm(*W.orszag_tang_3d(32, recon="wenoz", rk=3)),
                              "3D Orszag-Tang 32^3 with GLM (same scheme)"),
    "orszag-tang2d-128": (lambda: W.orszag_tang_2d(128), "Orszag-Tang 2D 128^2 (the workload itself)"),
    "ensemble2d-256": (lambda: ensemble_cases(16, max_n=128)[0],
                       "the first 16 ensemble members of at most 128^2 cells"),
    "adjoint2d-256": (lambda: W.adjoint_2d(32), "the same recipe on 32^2, 8 steps"),
    "adjoint2d-256-hll": (lambda: W.adjoint_2d(32, riemann="hll"), "the same recipe on 32^2, 8 steps (HLL)"),
    "adjoint2d-256-paper": (lambda: W.adjoint_2d(32, recon="wenoz", rk=3, emf="uct_hlld"),
                            "the same recipe on 32^2, 8 steps (WENO-Z + HLLD + RK3 + UCT-HLLD)"),
}
ADJOINT_SAMPLE_STEPS = 8


def ensemble_cases(count=256, max_n=None):
    members = W.ensemble_members(256, seed=4)
    if max_n is not None:
        members = [m for m in members if m["n"] <= max_n]
    return [W.ensemble_member_state(m) for m in members[:count]]


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_time_ms(ms, world, dev):
    """The job's time: the slowest rank's (all-reduce MAX over the ranks)."""
    if world == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, t_max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (t_max_ms * 1e-3)


def cells_of(cfg):
    return int(np.prod(cfg["n"][:cfg["ndim"]]))


# ---------------------------------------------------------------------------
# algorithmic flops (per-unit counts of the oracle, stored by tests/golden/make_flops.py)
# ---------------------------------------------------------------------------
def per_unit_counts(variant, per_face=False):
    """The oracle's per-unit flop counts of a variant.  per_face=True takes
    the WENO-Z reconstruction as the oracle counts it, face by face (the
    face-independent indicators and ratios twice per cell); the default counts
    them once per cell, as the method needs them."""
    path = os.path.join(ROOT, "tests", "golden", "flops_per_unit.json")
    per = dict(json.load(open(path))["variants"][variant]["per_unit"])
    if per_face and "recon_per_face_count" in per:
        per["recon"] = per["recon_per_face_count"]
    return per


def glm_flop_model(cfg, per):
    """Algorithmic flops of the GLM scheme (its own loop ranges: interior pencils, 9 variables)."""
    nd = cfg["ndim"]
    n = list(cfg["n"][:nd])
    G = 2 if cfg["recon"] == "plm" else 3
    cells = int(np.prod(n))
    sweep = {}
    for d in range(nd):
        rows = int(np.prod([n[t] for t in range(nd) if t != d]))
        sweep[d] = per["recon"] * (n[d] + 2) * rows + per["riemann"] * (n[d] + 1) * rows + per["fluxdiff"] / nd * cells
    padded = int(np.prod([m + 2 * G for m in n]))
    stage = per["c2p"] * padded + sum(sweep.values()) + per["rk"] * 9 * cells
    step = cfg["rk"] * stage + per["cfl"] * cells
    return {"sweep_per_launch": sweep, "step": step, "per_cell_update": step / cells}


def flop_model(cfg, variant, per_face=False):
    per = per_unit_counts(variant, per_face)
    if cfg.get("divb", "ct") == "glm":
        return glm_flop_model(cfg, per)
    nd = cfg["ndim"]
    n = list(cfg["n"][:nd])
    G = 2 if cfg["recon"] == "plm" else 3
    rk = cfg["rk"]
    cells = int(np.prod(n))
    sweep = {}
    for d in range(nd):
        rows = int(np.prod([n[t] + 2 for t in range(nd) if t != d]))
        sweep[d] = (per["recon"] * (n[d] + 2) * rows + per["riemann"] * (n[d] + 1) * rows
                    + per["fluxdiff"] / nd * cells)
    padded = int(np.prod([m + 2 * G for m in n]))
    if nd == 2:
        edges = (n[0] + 1) * (n[1] + 1)
    else:
        edges = sum(int(np.prod([n[e] + (1 if e != c else 0) for e in range(3)])) for c in range(3))
    periodic = [cfg["bc"][2 * d] == "periodic" for d in range(nd)]
    ct_faces = sum(int(np.prod([n[e] + (1 if (e == d and not periodic[d]) else 0) for e in range(nd)]))
                   for d in range(nd))
    elems = cells * (6 if nd == 2 else 5) + ct_faces
    stage = (per["c2p"] * padded + sum(sweep.values()) + per["emf"] * edges + per["ct"] * ct_faces
             + per["rk"] * elems)
    step = rk * stage + per["cfl"] * cells
    return {"sweep_per_launch": sweep, "step": step, "per_cell_update": step / cells}


def adjoint_flop_model(cfg, variant):
    """Algorithmic reverse-mode flops of one step (tape count of the oracle:
    forward flops + partial derivatives + backward sweep, per unit) and of
    one Riemann-transpose launch (one direction, one stage)."""
    path = os.path.join(ROOT, "tests", "golden", "flops_per_unit.json")
    per = json.load(open(path))["variants"][variant]["adjoint_per_unit"]
    nd = cfg["ndim"]
    n = list(cfg["n"][:nd])
    rk = cfg["rk"]
    cells = int(np.prod(n))
    padded = int(np.prod([m + 4 for m in n]))
    recon = faces = 0
    faces_dir = []
    for d in range(nd):
        rows = int(np.prod([n[t] + 2 for t in range(nd) if t != d]))
        recon += (n[d] + 2) * rows
        faces += (n[d] + 1) * rows
        faces_dir.append((n[d] + 1) * rows)
    edges = (n[0] + 1) * (n[1] + 1) if nd == 2 else sum(
        int(np.prod([n[e] + (1 if e != c else 0) for e in range(3)])) for c in range(3))
    ct_faces = cells * nd
    elems = cells * (6 if nd == 2 else 5) + ct_faces
    stage = (per["c2p"] * padded + per["recon"] * recon + per["riemann"] * faces + per["fluxdiff"] * cells
             + per["emf"] * edges + per["ct"] * ct_faces + per["rk"] * elems)
    return {"step": rk * stage, "riemann_per_launch": per["riemann"] * sum(faces_dir) / nd}


SWEEP_SOURCES = ("mhd_math.cuh", "mhd_kernels.cuh")  # everything the sweep kernels are compiled from
GLM_SWEEP_SOURCES = SWEEP_SOURCES + ("mhd_glm.cuh",)


def sweep_source_hash(files=SWEEP_SOURCES):
    """Hash of the sweep kernels' code: the sources with comments and
    whitespace removed, so that an edit of a comment keeps the captures."""
    import re
    text = ""
    for f in files:
        s = open(os.path.join(ROOT, "paper_2511_20337_b300", "csrc", f)).read()
        s = re.sub(r"/\*.*?\*/", " ", s, flags=re.S)
        s = re.sub(r"//[^\n]*", " ", s)
        text += " ".join(s.split()) + "\n"
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def fp64_peak(dev):
    """The FP64 ALU roofline: SMs x 2 FP64 FMAs per clock (the FP64 pipe rate;
    1.25 TFLOP/s nominal) x 2 flops x the maximum SM clock of MEASURED_PEAKS.json
    (2032 MHz on this B300).  Also returns the pipe's measured issue rates by
    instruction form (mhd_probe_fp64_forms, GFLOP/s equivalents): a DFMA chain
    with its operands in registers reaches the derived peak; DFMA with a
    constant operand, DMUL and DADD issue at a lower rate.
    Returns (peak GFLOP/s, its source, rates)."""
    import torch
    from paper_2511_20337_b300 import mhd
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2032.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mhz = float(json.load(open(path)).get("sm_max_mhz", mhz))
    peak = sms * 2 * 2 * mhz * 1e6 / 1e9
    src = (f"derived: {sms} SMs x 2 FP64 FMA per clock x 2 flops x {mhz:.0f} MHz (MEASURED_PEAKS.json sm_max_mhz); "
           "fp64_issue_rates gives the measured pipe rate by instruction form (probe_gflops: DFMA with register operands)")
    return peak, src, mhd.probe_fp64_forms()


def sweep_traffic(cfg, faces_per_launch):
    """DRAM bytes per sweep launch from the committed ncu captures
    (profiles/sweep_traffic.json) of the same sweep kernel (dimension,
    reconstruction, Riemann solver, divergence control), scaled by faces per
    launch; None when the sweep kernels' sources changed since the capture or
    no capture of that kernel exists."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    scheme = {"ndim": cfg["ndim"], "recon": cfg["recon"], "riemann": cfg["riemann"], "divb": cfg.get("divb", "ct")}
    if scheme["divb"] == "ct":
        scheme["emf"] = cfg.get("emf", "uct_hll")
    files = GLM_SWEEP_SOURCES if scheme["divb"] == "glm" else SWEEP_SOURCES
    for v in rec.values():
        if isinstance(v, dict) and v.get("scheme") == scheme:
            if v.get("source_hash", rec.get("source_hash")) != sweep_source_hash(files):
                return None
            per = sum(v["bytes_per_launch"]) / len(v["bytes_per_launch"])
            return per * faces_per_launch / v["faces_per_launch"]
    return None


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_oracle_rate(sample_fn, seconds_budget=15.0, max_steps=None):
    """The oracle as it stands, single-threaded, on the sample grid: cell-updates/s."""
    import oracle
    cfg, st = sample_fn()
    s = (oracle.OracleGlm(cfg, st, alpha=cfg["glm_alpha"]) if cfg.get("divb", "ct") == "glm"
         else oracle.OracleSim(cfg, st))
    s.advance(1)  # warm
    steps = 0
    t0 = time.perf_counter()
    while True:
        s.advance(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_budget or (max_steps and steps >= max_steps):
            break
    return cells_of(cfg) * steps / el, steps, el


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    gen, desc = SAMPLES[args.workload]
    if args.workload.startswith("adjoint2d"):
        cfg, st = gen()
        for _ in range(min(args.warmup, 1)):
            oracle_gradient_rate(cfg, st, ADJOINT_SAMPLE_STEPS)
        rates = [oracle_gradient_rate(cfg, st, ADJOINT_SAMPLE_STEPS) for _ in range(args.steps)]
        el = sum(r[1] for r in rates)
        value = 3 * cells_of(cfg) * ADJOINT_SAMPLE_STEPS * args.steps / el
        desc = f"{desc}, one tape gradient per step"
    elif args.workload == "ensemble2d-256":
        cases = ensemble_cases(16, max_n=128)
        sims = [oracle.OracleSim(c, st) for c, st in cases]
        for _ in range(args.warmup):
            for o in sims:
                o.advance(1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for o in sims:
                o.advance(1)
        el = time.perf_counter() - t0
        value = sum(cells_of(c) for c, _ in cases) * args.steps / el
    else:
        cfg, st = gen()
        s = (oracle.OracleGlm(cfg, st, alpha=cfg["glm_alpha"]) if cfg.get("divb", "ct") == "glm"
             else oracle.OracleSim(cfg, st))
        for _ in range(args.warmup):
            s.advance(1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.advance(1)
        el = time.perf_counter() - t0
        value = cells_of(cfg) * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][2], "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{desc}, {args.steps} steps after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2511_20337_b300 import mhd

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    gen, variant, desc = WORKLOADS[args.workload]
    cfg, st = gen()
    ncell = cells_of(cfg)
    stream = torch.cuda.Stream(device=dev)
    host = {k: torch.from_numpy(v).pin_memory() for k, v in st.items()}
    devs = {k: v.to(dev) for k, v in host.items()}
    del st
    sim = mhd.Sim(cfg, devs, stream=ctypes_stream(stream))
    h2d = sum(v.numel() * 8 for v in host.values())
    out_host = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    if args.seglen:
        sim.set_seglen(args.seglen)
        seg = args.seglen
    else:
        seg = sim.autotune() if ncell <= 256 ** 3 else None  # larger grids keep the library's default
    # warm-up (also captures the step graph)
    sim.advance(args.warmup)
    torch.cuda.synchronize(dev)
    barrier()

    # ---- timed region: K steps, state resident in HBM ----
    launches0 = sim.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        barrier()
        e0.record(stream)
        sim.advance(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = e0.elapsed_time(e1)
    launches = sim.launches - launches0
    rc, bad = sim.status()
    if rc != 0:
        raise RuntimeError(f"device reported {rc} at cell {bad}")
    t_max = job_time_ms(ms, world, dev)
    value = job_rate(ncell * args.steps, world, t_max)

    # ---- per-kernel device times (events after each launch) for the roofline ----
    big = ncell > 256 ** 3   # a 512^3 step takes seconds: shorter profile and e2e legs
    prof_steps = max(1, min(args.steps, 5 if big else 10))
    kms, kcnt = sim.profile_steps(prof_steps)
    peak, peak_src, rates = fp64_peak(dev)
    probe = rates["dfma"]
    fm = flop_model(cfg, variant)
    fm_face = flop_model(cfg, variant, per_face=True)
    nd = cfg["ndim"]
    sweep_ms = sum(kms[f"sweep_{a}"] for a in "xyz"[:nd])
    sweep_launches = sum(kcnt[f"sweep_{a}"] for a in "xyz"[:nd])
    sweep_flops = sum(fm["sweep_per_launch"].values()) * cfg["rk"] * prof_steps  # all sweep launches
    achieved = sweep_flops / (sweep_ms * 1e-3) / 1e9
    step_ms_prof = sum(kms.values()) / prof_steps
    step_achieved = fm["step"] / (step_ms_prof * 1e-3) / 1e9
    face_frac = sum(fm_face["sweep_per_launch"].values()) * cfg["rk"] * prof_steps / (sweep_ms * 1e-3) / 1e9 / peak
    face_step_frac = fm_face["step"] / (step_ms_prof * 1e-3) / 1e9 / peak
    n = list(cfg["n"][:nd])
    faces_per_launch = sum((n[d] + 1) * int(np.prod([n[t] + 2 for t in range(nd) if t != d])) for d in range(nd)) / nd
    sweep_name = ("glm_sweep_kernel (fused reconstruct + (B_n, psi) solve + HLLD + flux difference)"
                  if cfg.get("divb", "ct") == "glm" else "sweep_kernel (fused reconstruct + HLLD + flux difference)")
    roofline = {"bound": "alu", "kernel": sweep_name,
                "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
                "peak_source": peak_src, "probe_gflops": probe, "frac_of_probe": achieved / probe,
                "fp64_issue_rates": rates,
                "algorithmic_flops_per_launch": sweep_flops / sweep_launches,
                "avg_launch_ms": sweep_ms / sweep_launches,
                "traffic": sweep_traffic(cfg, faces_per_launch),
                "traffic_note": "DRAM bytes per sweep launch (mean of the directions) from the ncu capture in "
                                "profiles/, scaled to this grid by faces; null if the kernels changed since",
                "step_achieved": step_achieved, "step_frac": step_achieved / peak,
                "flops_per_cell_update": fm["per_cell_update"],
                "kernel_ms_per_step": {k: v / prof_steps for k, v in kms.items()}}
    if cfg["recon"] == "wenoz":
        roofline["frac_per_face_count"] = face_frac
        roofline["step_frac_per_face_count"] = face_step_frac
        roofline["count_note"] = ("frac and step_frac count the WENO-Z indicators, tau5 and ratios once per cell, as the "
                                  "method needs them; the *_per_face_count fractions take the oracle's face-by-face "
                                  "count (those terms twice per cell)")

    # ---- end to end through the C-ABI with host buffers ----
    # Two contexts on two streams take the steps in turn: a step's host-to-device
    # copy overlaps the other context's step, and its device-to-host copy the
    # next one's.  Each step waits for the previous one to end (two steps at once
    # would share the SMs and finish together, leaving the GPU idle while both
    # copy).  Every step still copies its whole input in from pinned host memory
    # and its whole result out.
    streams = (stream, torch.cuda.Stream(device=dev))
    sim2 = mhd.Sim(cfg, devs, stream=ctypes_stream(streams[1]))
    if seg is not None:
        sim2.set_seglen(seg)
    ctxs = (sim, sim2)
    for c in ctxs:
        c.set_conserved(host)
        c.advance(1)                   # captures the step graph
        c.get_conserved(out_host)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_steps = max(2, min(args.steps, 8 if big else 20))
    t0 = time.perf_counter()
    prev, done = None, None
    for s in range(e2e_steps):
        c, cs = ctxs[s % 2], streams[s % 2]
        c.set_conserved(host)          # H2D of this step's input
        if done is not None:
            cs.wait_event(done)        # after the previous step
        c.advance(1)
        done = torch.cuda.Event()
        done.record(cs)
        if prev is not None:
            prev.get_conserved(out_host)   # D2H of the previous step's result (synchronous)
        prev = c
    prev.get_conserved(out_host)
    el = job_time_ms(time.perf_counter() - t0, world, dev)
    e2e = {"value": ncell * e2e_steps * world / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d, "steps": e2e_steps,
           "pipeline": "two contexts alternate, steps in order; copies of one overlap the other's step"}
    sim2.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sgen, sdesc = SAMPLES[args.workload]
        rate, steps, el = cpu_oracle_rate(sgen, seconds_budget=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sdesc}: {steps} steps in {el:.1f} s, single thread"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": desc, "grid": list(cfg["n"]), "cells": ncell,
                           "seglen": sim.seglen,
                           "l2": (f"inputs larger than L2 (state {h2d / 1e9:.2f} GB)" if h2d > 126e6 else
                                  f"state {h2d / 1e6:.1f} MB fits in L2 and is not flushed between steps "
                                  "(a parity-size workload, not the headline)"),
                           "dt": "CFL dt computed on the device every step", "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary()}
        if args.bricks:
            parts = [int(x) for x in args.bricks.split("x")]
            dom = measure_domain(cfg, devs, parts, args.steps, args.warmup, stream, seg)
            dom["value_over_undivided"] = dom["value"] / value
            line["decomposed"] = dom
        if world == 1 and not args.no_companions:
            sim.close()
            sim = None
            line["batched_vs_plain"], line["adjoint_vs_plain"] = companions(
                dev, stream, value, roofline["frac"], roofline["step_frac"], args.steps)
        if args.workload in PAPER_PER_GPU:
            line["paper_context"] = {"per_gpu_cell_updates_per_s": PAPER_PER_GPU[args.workload],
                                     "this_gpu_over_paper_gpu": {k: value / world / v
                                                                 for k, v in PAPER_PER_GPU[args.workload].items()},
                                     "note": "the paper's single-node 3D Orszag-Tang runs (704x704x352 per node of 4 "
                                             "GPUs, UCT-HLLD edge fields); context, not the target"}
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_domain(cfg, devs, parts, steps, warmup, stream, seglen=None):
    """The same workload split into bricks (mhd_domain_*: a halo exchange per
    RK stage, all bricks on this GPU): cell-updates/s over `steps` CFL steps
    after `warmup`, and the bytes one exchange moves."""
    import torch
    from paper_2511_20337_b300 import mhd
    d = mhd.Domain(cfg, parts, devs, stream=stream.cuda_stream)
    if seglen:
        d.set_seglen(seglen)
    d.advance(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = d.launches
    e0.record(stream)
    d.advance(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rc, bad = d.status()
    if rc != 0:
        raise RuntimeError(f"device reported {rc} at cell {bad}")
    out = {"bricks": list(parts), "value": cells_of(cfg) * steps / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms / steps, "steps": steps, "gpu_launches": d.launches - l0,
           "halo_bytes_per_exchange": d.halo_bytes, "exchanges_per_step": cfg["rk"],
           "what": "the same grid as bricks with a pack / device-copy / unpack halo exchange per RK stage, "
                   "all bricks on this GPU; state, dt and time equal the undivided run's to the bit"}
    d.close()
    return out


def measure_ensemble(dev, stream, steps, warmup, loop=True, clocks=None, barrier=lambda: None):
    """The batched ensemble (256 2D Orszag-Tang runs of 64^2..512^2 in one
    graph per step, autotuned segment lengths): `steps` timed steps after
    `warmup`, the batched sweep on the FP64 roofline, and (loop=True) the same
    runs as a loop of single-grid steps on the same stream, the plain step of
    those grids.  Returns the measurements and the live batch."""
    import torch
    from paper_2511_20337_b300 import mhd
    _, variant, desc = WORKLOADS["ensemble2d-256"]
    cases = ensemble_cases(256)
    cfgs = [c for c, _ in cases]
    ncell = sum(cells_of(c) for c in cfgs)
    host = [{k: torch.from_numpy(v).pin_memory() for k, v in st.items()} for _, st in cases]
    h2d = sum(v.numel() * 8 for h in host for v in h.values())
    del cases
    bt = mhd.Batch(cfgs, stream=stream.cuda_stream)
    for r, h in enumerate(host):
        bt.set_conserved(r, h)
    seg = bt.autotune()
    bt.step(warmup)
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = bt.launches
    clk = clocks if clocks is not None else _NullClocks()
    with clk:
        torch.cuda.synchronize(dev)
        barrier()
        e0.record(stream)
        bt.step(steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = e0.elapsed_time(e1)
    launches = bt.launches - launches0
    rc, bad_run, bad = bt.status()
    if rc != 0:
        raise RuntimeError(f"device reported {rc} in run {bad_run} at cell {bad}")

    # roofline of the batched sweep (events after each launch)
    prof_steps = max(1, min(steps, 5))
    kms, kcnt = bt.profile_steps(prof_steps)
    peak, peak_src, rates = fp64_peak(dev)
    probe = rates["dfma"]
    fms = [flop_model(c, variant) for c in cfgs]
    sweep_ms = kms["sweep_x"] + kms["sweep_y"]
    sweep_launches = kcnt["sweep_x"] + kcnt["sweep_y"]
    sweep_flops = sum(sum(f["sweep_per_launch"].values()) for f in fms) * cfgs[0]["rk"] * prof_steps
    achieved = sweep_flops / (sweep_ms * 1e-3) / 1e9
    step_flops = sum(f["step"] for f in fms)
    step_ms_prof = sum(kms.values()) / prof_steps
    roofline = {"bound": "alu", "kernel": "batch_sweep_kernel (fused reconstruct + HLLD + flux difference, all runs)",
                "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
                "peak_source": peak_src, "probe_gflops": probe, "frac_of_probe": achieved / probe,
                "fp64_issue_rates": rates,
                "algorithmic_flops_per_launch": sweep_flops / sweep_launches,
                "avg_launch_ms": sweep_ms / sweep_launches, "traffic": None,
                "traffic_note": "no ncu capture of the batched sweep",
                "step_achieved": step_flops / (step_ms_prof * 1e-3) / 1e9,
                "step_frac": step_flops / (step_ms_prof * 1e-3) / 1e9 / peak,
                "kernel_ms_per_step": {k: v / prof_steps for k, v in kms.items()}}

    loop_ms = None
    if loop:   # the same runs as a loop of single-grid steps on the same stream
        sims = [mhd.Sim(c, h, stream=stream.cuda_stream) for c, h in zip(cfgs, host)]
        for sm in sims:
            sm.advance(warmup)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for sm in sims:
            sm.advance(steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        loop_ms = e0.elapsed_time(e1)
        for sm in sims:
            sm.close()
        del sims
    return {"bt": bt, "cfgs": cfgs, "host": host, "ncell": ncell, "h2d": h2d, "seg": seg, "ms": ms,
            "launches": launches, "roofline": roofline, "loop_ms": loop_ms, "desc": desc, "clk": clk}


class _NullClocks:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def summary(self):
        return None


def run_ensemble(args):
    import torch
    from paper_2511_20337_b300 import mhd

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    m = measure_ensemble(dev, stream, args.steps, args.warmup, clocks=ClockSampler(local), barrier=barrier)
    bt, cfgs, host, ncell, h2d, seg, ms = m["bt"], m["cfgs"], m["host"], m["ncell"], m["h2d"], m["seg"], m["ms"]
    t_max = job_time_ms(ms, world, dev)
    value = job_rate(ncell * args.steps, world, t_max)
    loop_ms = m["loop_ms"]

    # end to end: every run's state in from pinned host memory, one step, every
    # state out, all runs as one packed array (one copy and one scatter or
    # gather kernel each way).  Three batches on three streams take the steps in
    # turn, each step after the previous one: while one batch steps, the next
    # one's states are written and the previous one's read out.
    streams = (stream, torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))
    bts = (bt, mhd.Batch(cfgs, stream=streams[1].cuda_stream), mhd.Batch(cfgs, stream=streams[2].cuda_stream))
    for b in bts[1:]:
        b.set_seglen(*seg)
    in_packed = bt.pack(host, out=torch.empty(bt.packed_size(), dtype=torch.float64).pin_memory())
    out_packed = torch.empty(bt.packed_size(), dtype=torch.float64).pin_memory()
    assert in_packed.numel() * 8 == h2d
    for b in bts:
        b.set_conserved_packed(in_packed)
        b.step(1)                      # captures the step graph
        b.get_conserved_packed(out_packed)
    torch.cuda.synchronize(dev)
    e2e_steps = max(3, min(args.steps, 10))

    def write(b):
        b.set_conserved_packed(in_packed)

    def read(b):
        b.get_conserved_packed(out_packed)   # waits for its copy

    t0 = time.perf_counter()
    write(bts[0])
    done = None
    for s in range(e2e_steps):
        b, bs = bts[s % 3], streams[s % 3]
        if done is not None:
            bs.wait_event(done)        # after the previous step
        b.step(1)
        done = torch.cuda.Event()
        done.record(bs)
        if s + 1 < e2e_steps:
            write(bts[(s + 1) % 3])    # the next step's states, into the batch read out a step ago
        if s > 0:
            read(bts[(s - 1) % 3])     # the previous step's states
    read(bts[(e2e_steps - 1) % 3])
    el = job_time_ms(time.perf_counter() - t0, world, dev)
    e2e = {"value": ncell * e2e_steps * world / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d, "steps": e2e_steps,
           "pipeline": "packed I/O; three batches in turn, steps in order; one's copies in and another's out overlap the third's step"}
    for b in bts[1:]:
        b.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        sub = ensemble_cases(16, max_n=128)
        osims = [oracle.OracleSim(c, st) for c, st in sub]
        steps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < args.cpu_seconds:
            for o in osims:
                o.advance(1)
            steps += 1
        el = time.perf_counter() - t0
        cpu = {"value": sum(cells_of(c) for c, _ in sub) * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first 16 ensemble members of at most 128^2 cells, {steps} steps each in {el:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": m["desc"], "runs": len(cfgs), "cells": ncell,
                           "sizes": sorted(set(c["n"][0] for c in cfgs)),
                           "autotuned_seglen": {"small_runs": seg[0], "large_runs": seg[1]},
                           "l2": f"inputs larger than L2 (states {h2d / 1e9:.2f} GB)",
                           "dt": "per-run CFL dt computed on the device every step",
                           "parallelism": f"replicas x{world}"},
                "loop_of_single_grid_steps": {"value": ncell * args.steps / (loop_ms * 1e-3), "unit": UNIT,
                                              "ms_per_step": loop_ms / args.steps,
                                              "batched_speedup": loop_ms / ms},
                "roofline": m["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": m["launches"],
                "clocks": m["clk"].summary()}
        print(json.dumps(line), flush=True)
    bt.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def oracle_gradient_rate(cfg, st, nsteps, which="magnetic_energy", seconds_budget=0.0):
    """The oracle's reverse-mode (tape) gradient of an nsteps run, as it
    stands, single-threaded, repeated until seconds_budget has passed:
    (cell-updates/s counted as for the GPU adjoint, 3 per cell and step;
    seconds; gradients taken)."""
    import oracle
    rho = st["rho"]
    v = [st[k] / rho for k in ("mx", "my", "mz")]
    bx, by, bz = W.cell_field(cfg, st["b0"], st["b1"], st["b2"])
    g = cfg["gamma"]
    p = (g - 1) * (st["E"] - 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) - 0.5 * (bx ** 2 + by ** 2 + bz ** 2))
    prim = {"rho": rho, "vx": v[0], "vy": v[1], "vz": v[2], "p": p}
    dts = oracle.OracleSim(cfg, st).advance(nsteps, record_dt=True)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.grad_prim(cfg, prim, (st["b0"], st["b1"], st["b2"]), dts, which)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds_budget:
            break
    return 3 * cells_of(cfg) * nsteps * reps / el, el, reps


def measure_adjoint(dev, stream, workload, gradients, warmup, seglen=0, clocks=None, barrier=lambda: None):
    """One gradient evaluation per step: ADJOINT_STEPS forward steps from the
    initial state with checkpoints, the block recomputes and the reverse pass.
    Times `gradients` evaluations after `warmup`, profiles the phases and the
    reverse kernel classes, places the Riemann transpose and the gradient on
    the FP64 roofline, and times the plain forward run of the same grid and
    steps on the same GPU.  Returns the measurements and the live context."""
    import torch
    from paper_2511_20337_b300 import mhd
    gen, variant, desc = WORKLOADS[workload]
    cfg, st = gen()
    ncell = cells_of(cfg)
    N, K = ADJOINT_STEPS, ADJOINT_CKPT
    host = {k: torch.from_numpy(v).pin_memory() for k, v in st.items()}
    devs = {k: v.to(dev) for k, v in host.items()}
    sim = mhd.Sim(cfg, devs, stream=stream.cuda_stream)
    if seglen:
        sim.set_seglen(seglen)
        seg = seglen
    else:
        seg = sim.autotune()
    _, dts = sim.adjoint(N, None, K)  # records the CFL steps, then frozen
    for _ in range(warmup):
        sim.set_conserved(devs)
        sim.adjoint(N, dts, K)
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = sim.launches
    clk = clocks if clocks is not None else _NullClocks()
    with clk:
        torch.cuda.synchronize(dev)
        barrier()
        e0.record(stream)
        for _ in range(gradients):
            sim.set_conserved(devs)
            J, _ = sim.adjoint(N, dts, K)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = e0.elapsed_time(e1)
    launches = sim.launches - launches0

    # phases and kernel classes (events on the library stream; syncs every reverse step)
    sim.set_conserved(devs)
    phases, classes = sim.adjoint_profile(N, dts, K)
    peak, peak_src, rates = fp64_peak(dev)
    probe = rates["dfma"]
    am = adjoint_flop_model(cfg, variant)
    nd = cfg["ndim"]
    riemann_launches = N * cfg["rk"] * nd
    riemann_ms = classes["adj_riemann"]
    achieved = am["riemann_per_launch"] * riemann_launches / (riemann_ms * 1e-3) / 1e9
    eval_ms = ms / gradients
    roofline = {"bound": "alu", "kernel": "adj_riemann_kernel (Riemann solver + flux difference transpose, per face)",
                "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
                "peak_source": peak_src, "probe_gflops": probe, "frac_of_probe": achieved / probe,
                "fp64_issue_rates": rates,
                "algorithmic_flops_per_launch": am["riemann_per_launch"],
                "algorithmic_definition": "reverse-mode work of the oracle's Riemann solve from its tape: forward "
                                          "flops + partial-derivative flops + backward sweep (1 flop per +-1 link, "
                                          "2 otherwise), per face",
                "avg_launch_ms": riemann_ms / riemann_launches, "traffic": None,
                "traffic_note": "the 256^2 working set of these kernels stays in L2, so DRAM bytes do not measure re-reads; "
                                "ncu summary in profiles/adj_riemann_kernel_adjoint2d-256.md",
                "gradient_achieved": am["step"] * N / (eval_ms * 1e-3) / 1e9,
                "gradient_frac": am["step"] * N / (eval_ms * 1e-3) / 1e9 / peak,
                "reverse_ms_by_class": classes}
    phase_rates = {k: {"ms": v, "cell_updates_per_s": ncell * N / (v * 1e-3)} for k, v in phases.items()}

    # the plain forward step on the same GPU, same grid and steps (graph replay)
    ref = mhd.Sim(cfg, devs, stream=stream.cuda_stream)
    ref.set_seglen(seg)
    ref.advance(3)
    ref.set_conserved(devs)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    ref.advance(N)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1)
    ref.close()
    return {"sim": sim, "cfg": cfg, "host": host, "devs": devs, "dts": dts, "ncell": ncell, "seg": seg, "ms": ms,
            "eval_ms": eval_ms, "J": J, "launches": launches, "roofline": roofline, "phases": phase_rates,
            "plain_ms": plain_ms, "desc": desc, "clk": clk}


def run_adjoint(args):
    """A step is one gradient evaluation (measure_adjoint).  Cell-updates count
    3 per cell and time step (forward, recompute, reverse); the phases are also
    reported separately."""
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    m = measure_adjoint(dev, stream, args.workload, args.steps, args.warmup, args.seglen,
                        clocks=ClockSampler(local), barrier=barrier)
    sim, cfg, host, ncell, N, K = m["sim"], m["cfg"], m["host"], m["ncell"], ADJOINT_STEPS, ADJOINT_CKPT
    t_max = job_time_ms(m["ms"], world, dev)
    value = job_rate(3 * ncell * N * args.steps, world, t_max)
    eval_ms = t_max / args.steps
    h2d = sum(v.numel() * 8 for v in host.values())
    grad_host = {k: torch.empty_like(host["rho"]).pin_memory() for k in ("rho", "vx", "vy", "vz")}
    d2h = sum(v.numel() * 8 for v in grad_host.values())

    # end to end: state in from pinned host memory, gradient out to pinned host memory
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_conserved(host)
        sim.adjoint(N, m["dts"], K)
        sim.grad_prim(grad_host)
    el = time.perf_counter() - t0
    e2e = {"value": 3 * ncell * N * e2e_steps * world / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        scfg, sst = SAMPLES[args.workload][0]()
        rate, sec, reps = oracle_gradient_rate(scfg, sst, ADJOINT_SAMPLE_STEPS, seconds_budget=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{SAMPLES[args.workload][1]}: {reps} tape gradients in {sec:.1f} s, single thread"}
    if rank == 0:
        plain_ms = m["plain_ms"]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": eval_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": m["desc"], "grid": list(cfg["n"]), "cells": ncell, "time_steps": N,
                           "checkpoint_every": K, "J": m["J"], "autotuned_seglen": m["seg"],
                           "step": "one gradient evaluation; 3 cell-updates per cell and time step "
                                   "(forward, recompute, reverse)",
                           "l2": "each gradient evaluation streams its checkpoints and stage states "
                                 f"({(N // K + K * cfg['rk'] + 1) * h2d / 1e6:.0f} MB) through HBM, larger than L2",
                           "dt": "CFL steps of the first run, then frozen", "parallelism": f"replicas x{world}"},
                "phases": m["phases"],
                "plain_step": {"value": ncell * N / (plain_ms * 1e-3), "unit": UNIT, "ms_per_step": plain_ms / N,
                               "gradient_vs_plain_time": eval_ms / plain_ms},
                "roofline": m["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": m["launches"],
                "clocks": m["clk"].summary()}
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def companions(dev, stream, plain_value, plain_frac, plain_step_frac, steps):
    """The batched and adjoint forms measured on the same GPU after the plain
    step, compactly (no e2e, no CPU baseline), each with its own cell-updates/s
    and roofline fraction and its ratio to the plain step: to the headline's
    plain step, and to the plain step of its own grids (the loop of
    single-grid steps of the same runs; the plain forward run of the same grid
    and time steps)."""
    import torch
    e = measure_ensemble(dev, stream, max(3, min(steps, 20)), 3)
    ens_value = e["ncell"] * max(3, min(steps, 20)) / (e["ms"] * 1e-3)
    loop_value = e["ncell"] * max(3, min(steps, 20)) / (e["loop_ms"] * 1e-3)
    batched = {"workload": e["desc"], "value": ens_value, "unit": UNIT, "steps": max(3, min(steps, 20)),
               "ms_per_step": e["ms"] / max(3, min(steps, 20)), "cells": e["ncell"], "gpu_launches": e["launches"],
               "frac": e["roofline"]["frac"], "step_frac": e["roofline"]["step_frac"],
               "roofline_kernel": e["roofline"]["kernel"],
               "plain_step_same_runs": {"value": loop_value, "unit": UNIT,
                                        "what": "the same 256 runs as a loop of single-grid steps, same stream"},
               "batched_over_plain_same_runs": ens_value / loop_value,
               "value_over_headline": ens_value / plain_value, "frac_over_headline": e["roofline"]["frac"] / plain_frac,
               "step_frac_over_headline": e["roofline"]["step_frac"] / plain_step_frac}
    e["bt"].close()
    del e
    torch.cuda.synchronize(dev)
    a = measure_adjoint(dev, stream, "adjoint2d-256", 2, 1)
    N = ADJOINT_STEPS
    adj_value = 3 * a["ncell"] * N / (a["eval_ms"] * 1e-3)
    plain_grid = a["ncell"] * N / (a["plain_ms"] * 1e-3)
    adjoint = {"workload": a["desc"], "value": adj_value, "unit": UNIT, "gradients": 2,
               "ms_per_gradient": a["eval_ms"], "cell_updates_counted": "3 per cell and time step (forward, "
                                                                        "recompute, reverse)",
               "frac": a["roofline"]["frac"], "gradient_frac": a["roofline"]["gradient_frac"],
               "roofline_kernel": a["roofline"]["kernel"], "gpu_launches": a["launches"],
               "phases": a["phases"], "reverse_ms_by_class": a["roofline"]["reverse_ms_by_class"],
               "phases_note": "the phases are timed in sequence by the profiling run; the timed gradients overlap "
                              "the block recomputes with the reverse pass",
               "plain_step_same_grid": {"value": plain_grid, "unit": UNIT, "ms_per_step": a["plain_ms"] / N,
                                        "what": "the plain forward run of the same 256^2 grid and 400 steps"},
               "gradient_over_plain_time": a["eval_ms"] / a["plain_ms"],
               "value_over_headline": adj_value / plain_value,
               "gradient_frac_over_headline_step_frac": a["roofline"]["gradient_frac"] / plain_step_frac}
    a["sim"].close()
    return batched, adjoint


def ctypes_stream(stream):
    return stream.cuda_stream


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blast3d-512", choices=list(WORKLOADS))
    ap.add_argument("--no-companions", action="store_true",
                    help="single-grid workloads: skip the batched-ensemble and adjoint measurements that follow "
                         "the plain step (batched_vs_plain, adjoint_vs_plain)")
    ap.add_argument("--bricks", default="",
                    help="single-grid workloads: also time the grid split into bricks, e.g. 2x2x2 (the halo "
                         "exchange of the domain decomposition, all bricks on this GPU)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seglen", type=int, default=0,
                    help="sweep segment length of single-grid workloads (0: autotune)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # timing rule: at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble2d-256":
        return run_ensemble(args)
    if args.workload.startswith("adjoint2d"):
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
