"""Host-side checks of bench.py's roofline bookkeeping: the algorithmic bytes
per launch of each kernel label, the per-launch DRAM traffic recorded from ncu
(profiles/traffic.json) against those bytes, and which sources a label's
traffic entry depends on."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

V = 32 * 32 * 32 * 64  # the benchmark lattice


def test_algorithmic_bytes_per_site():
    # FP32 spinors 96 B per site, 18-real FP32 links 72 B, 12-real 48 B; per
    # lattice site V a hop reads the input once (V/2 sites), all 4V links,
    # writes the output (V/2) and, with axpy, reads the addend (V/2)
    assert bench.algo_bytes_per_site("hop_f32_l18") == 96 / 2 * 2 + 4 * 72
    assert bench.algo_bytes_per_site("hop_f32_l18_axpy") == 96 / 2 * 3 + 4 * 72
    assert bench.algo_bytes_per_site("hop_f32_l12_axpy_dag") == 96 / 2 * 3 + 4 * 48
    # the staged kernel computes the same hop: same algorithmic bytes
    for lab in ("hop_f32_l18", "hop_f32_l18_axpy", "hop_f32_l18_dag", "hop_f32_l18_axpy_dag"):
        assert bench.algo_bytes_per_site(lab.replace("hop_", "hop_staged_")) == bench.algo_bytes_per_site(lab)
    assert bench.algo_bytes_per_site("hop_f64_l18_axpy") == 192 / 2 * 3 + 4 * 144
    # one fused M_eo: input and output once, every link once
    assert bench.algo_bytes_per_site("fused_f32_l18_axpy") == 48 + 4 * 72 + 48


def test_useful_bytes_match_the_minimal_traffic_model():
    # minimal traffic of one M_eo per site V: 384 B (FP32 18-real), 288 B (12-real)
    assert bench.useful_bytes_per_site("f32", 18) == 384
    assert bench.useful_bytes_per_site("f32", 12) == 288
    assert bench.useful_bytes_per_site("f64", 18) == 768


def test_recorded_hop_traffic_is_close_to_the_algorithmic_bytes():
    """ncu DRAM bytes per launch of every recorded hop kernel (reads + writes
    still dirty in L2 at kernel end are not counted): within a few per cent
    below, and never more than 2 % above, the algorithmic bytes."""
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    hops = [k for k in d if k.startswith("hop_")]
    assert hops
    for lab in hops:
        algo = bench.algo_bytes_per_site(lab) * V
        got = d[lab]["bytes_per_launch"]
        assert 0.9 * algo <= got <= 1.02 * algo, (lab, got, algo)
        assert d[lab]["read_bytes"] + d[lab]["write_bytes"] == pytest.approx(got, abs=2)


def test_traffic_entries_name_their_sources():
    assert "hop_staged.cu" in bench.sources_for("hop_staged_f32_l18_axpy")
    assert "fused.cu" in bench.sources_for("fused_f32_l18_axpy")
    assert "hop_staged.cu" not in bench.sources_for("hop_f32_l18")


def test_both_arms_report_the_same_workload_config():
    """The reference arm and our arm print the same `config` dict (the workload,
    not the implementation: that goes to `impl_config` / `sample_lattice`)."""
    import argparse

    ns = argparse.Namespace(prec="f32", linkfmt=18, ff=False)
    cfg = bench.workload_config(ns, 1)
    assert set(cfg) == {"workload", "lattice", "kappa", "links", "prec", "flop_per_site_per_meo", "l2",
                        "parallelism"}
    assert cfg["lattice"] == [32, 32, 32, 64] and cfg["flop_per_site_per_meo"] == 1344
    assert "32x32x32x64" in cfg["workload"] and "FP32" in cfg["workload"]
    assert bench.workload_config(ns, 4)["parallelism"] == "replicas"
