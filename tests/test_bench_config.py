"""bench.py's host logic (no GPU): every workload has an algorithmic flop
variant in tests/golden/flops_per_unit.json, a CPU-oracle sample and a
description; the flop model of each scheme is positive and its sweep share
adds up; traffic lookups give a positive byte count or null; and the flop
variant of each workload was counted on the workload's own scheme."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def golden():
    return json.load(open(os.path.join(ROOT, "tests", "golden", "flops_per_unit.json")))["variants"]


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_every_workload_has_variant_sample_and_description(name):
    gen, variant, desc = bench.WORKLOADS[name]
    assert variant in golden(), variant
    assert name in bench.SAMPLES, name
    assert isinstance(desc, str) and len(desc) > 20


def scheme_of(cfg):
    return (cfg["ndim"], cfg["recon"], cfg["riemann"], cfg["rk"], cfg.get("divb", "ct"), cfg.get("emf", "uct_hll"))


@pytest.mark.parametrize("name", sorted(n for n, w in bench.WORKLOADS.items() if w[0] is not None))
def test_flop_model_and_scheme_match(name):
    gen, variant, _ = bench.WORKLOADS[name]
    sgen, _ = bench.SAMPLES[name]
    cfg, _ = sgen()  # the small sample has the workload's scheme
    g = golden()[variant]
    rec = g["config"]
    assert (rec["ndim"], rec["recon"], rec["riemann"], rec["rk"]) == scheme_of(cfg)[:4], (name, variant)
    assert g.get("divb", "ct") == cfg.get("divb", "ct"), (name, variant)
    assert rec.get("emf", "uct_hll") == cfg.get("emf", "uct_hll"), (name, variant)
    fm = bench.flop_model(cfg, variant)
    assert fm["step"] > 0 and fm["per_cell_update"] > 0
    nd = cfg["ndim"]
    assert set(fm["sweep_per_launch"]) == set(range(nd))
    assert all(v > 0 for v in fm["sweep_per_launch"].values())
    # the sweeps are the bulk of the step's algorithmic work
    assert sum(fm["sweep_per_launch"].values()) * cfg["rk"] < fm["step"]
    t = bench.sweep_traffic(cfg, 1e6)
    assert t is None or t > 0


def test_default_workload_is_the_512_blast():
    """With no flags bench.py times the 512^3 magnetised blast (outflow,
    WENO-Z + HLLD + SSP-RK3 + UCT CT), the configuration whose roofline
    fraction is the target, and adds the batched and adjoint companions."""
    import argparse
    import sys
    argv = sys.argv
    seen = {}

    def fake_parse(self, *a, **k):
        ns = argparse.ArgumentParser.parse_known_args(self, [])[0]
        seen.update(vars(ns))
        raise SystemExit(0)
    old = argparse.ArgumentParser.parse_args
    argparse.ArgumentParser.parse_args = fake_parse
    try:
        sys.argv = ["bench.py"]
        with pytest.raises(SystemExit):
            bench.main()
    finally:
        argparse.ArgumentParser.parse_args = old
        sys.argv = argv
    assert seen["workload"] == "blast3d-512"
    assert not seen["no_companions"]
    cfg, _ = bench.SAMPLES["blast3d-512"][0]()
    assert (cfg["ndim"], cfg["recon"], cfg["riemann"], cfg["rk"]) == (3, "wenoz", "hlld", 3)
    assert cfg["bc"] == ["outflow"] * 6 or list(cfg["bc"]) == ["outflow"] * 6


@pytest.mark.parametrize("variant", sorted(v for v, g in golden().items() if g["config"]["recon"] == "wenoz"))
def test_wenoz_count_once_per_cell(variant):
    """WENO-Z: the face-independent part of a face value (indicators, tau5,
    ratios, 1 + ratio^2) is counted once per cell and variable.  By hand from
    the formulas: beta_0 and beta_2 take 12 flops each (curvature 3, one-sided
    difference 4, the weighted squares 5), beta_1 9, tau5 1, the three ratios 2
    each and 1 + r^2 2 each: 46.  The oracle's Counted run must agree, and the
    count bench.py uses is the per-face count less 46 per variable (7 for CT,
    9 for GLM)."""
    import oracle
    assert oracle.count_wenoz_shared() == 46
    g = golden()[variant]
    per = g["per_unit"]
    nvar = 9 if g.get("divb") == "glm" else 7
    assert per["wenoz_shared_per_variable"] == 46
    assert per["recon"] == per["recon_per_face_count"] - nvar * 46
    # per face the oracle counts 73 flops per variable (two faces per cell)
    assert per["recon_per_face_count"] == nvar * 2 * 73
    assert bench.per_unit_counts(variant, per_face=True)["recon"] == per["recon_per_face_count"]
    assert bench.per_unit_counts(variant)["recon"] == per["recon"]
