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
