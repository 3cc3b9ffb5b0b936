"""Host logic of bench.py (no GPU): the roofline object of the dominant stage
and the rule that a DRAM-traffic figure is reported only while the sources of
its kernel are unchanged since the ncu capture."""
import json
import os
import types

import pytest

import bench

ARGS = types.SimpleNamespace(N=1024, P=32)
PEAKS = {"hbm_gbs": 7000.0, "sm_max_mhz": 2070.0}


@pytest.mark.parametrize("stage_ms,kernel", [
    ([0.011, 0.067, 0.017], "recursions"),
    ([0.090, 0.067, 0.017], "prep"),
    ([0.011, 0.067, 0.170], "prob_forces"),
])
def test_roofline_follows_the_dominant_stage(stage_ms, kernel, monkeypatch):
    monkeypatch.setattr(bench, "load_traffic", lambda k: None)
    r = bench.roofline(stage_ms, ARGS, 2070.0, PEAKS)
    assert r["kernel"] == kernel
    assert r["achieved"] > 0
    if kernel == "recursions":
        # N dependent steps in the stage time, against one 64-cycle step per clock/64
        assert r["unit"] == "chain steps/s" and r["bound"] == "alu"
        assert r["achieved"] == pytest.approx(1024 / 0.067e-3)
        assert r["peak"] == pytest.approx(2070e6 / bench.DFMA_LATENCY_CYCLES)
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    elif kernel == "prep":
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])


def test_roofline_prep_counts_the_pair_factor_bytes_of_its_precision(monkeypatch):
    monkeypatch.setattr(bench, "load_traffic", lambda k: None)
    mixed = bench.roofline([1.0, 0.1, 0.1], ARGS, None, PEAKS, "mixed")
    fp64 = bench.roofline([1.0, 0.1, 0.1], ARGS, None, PEAKS, "fp64")
    pairs = 1024 * 1025 // 2
    # both copies of g: 4 more mantissa bytes per entry in float64
    assert (fp64["achieved"] - mixed["achieved"]) * 1e9 * 1e-3 == pytest.approx(2 * pairs * 4, rel=1e-9)


def test_traffic_figure_only_while_sources_match(tmp_path, monkeypatch):
    import hashlib
    rel = "csrc/kernel.cu"
    os.makedirs(tmp_path / "csrc")
    os.makedirs(tmp_path / "profiles")
    (tmp_path / rel).write_text("// a kernel\n")
    digest = hashlib.sha256((tmp_path / rel).read_bytes()).hexdigest()
    table = {"_about": "test", "recursions": {"kernel": "k", "dram_bytes_per_launch": 12345,
                                               "sources": [rel], "sources_sha256": digest}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("recursions") == 12345
    (tmp_path / rel).write_text("// a kernel, changed\n")
    assert bench.load_traffic("recursions") is None
    assert bench.load_traffic("no_such_stage") is None
