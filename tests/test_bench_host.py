"""Host logic of bench.py (no GPU): the roofline object of the dominant stage,
the rule that a DRAM-traffic figure is reported only while the sources of its
kernel are unchanged since the ncu capture, the clock summary taken from
nvidia-smi samples during the timed region, and the reference arm (the CPU
oracle timed on the same workload), which runs without a GPU."""
import json
import os
import subprocess
import sys
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
        # per-step latency: 67 us over 1024 steps at 2070 MHz
        assert r["ns_per_step"] == pytest.approx(0.067e-3 / 1024 * 1e9)
        assert r["cycles_per_step"] == pytest.approx(0.067e-3 / 1024 * 2070e6)
        assert r["floor_cycles_per_step"] == bench.DFMA_LATENCY_CYCLES
        assert r["frac"] == pytest.approx(r["floor_cycles_per_step"] / r["cycles_per_step"])
    elif kernel == "prep":
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])


def test_roofline_prep_counts_the_pair_factor_bytes_of_its_precision(monkeypatch):
    monkeypatch.setattr(bench, "load_traffic", lambda k: None)
    m32 = bench.roofline([1.0, 0.1, 0.1], ARGS, None, PEAKS, "mixed32")
    mixed = bench.roofline([1.0, 0.1, 0.1], ARGS, None, PEAKS, "mixed")
    fp64 = bench.roofline([1.0, 0.1, 0.1], ARGS, None, PEAKS, "fp64")
    pairs = 1024 * 1025 // 2
    # both copies of g: float64 mantissas in float64 and mixed, float32 in mixed32
    assert (fp64["achieved"] - m32["achieved"]) * 1e9 * 1e-3 == pytest.approx(2 * pairs * 4, rel=1e-9)
    assert mixed["achieved"] == fp64["achieved"]


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


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` prints exactly one JSON line with the keys
    of the bench contract; under a launcher, ranks other than 0 print nothing
    and exit 0."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
           "--steps", "3", "--warmup", "1", "--N", "64", "--P", "8"]
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 1
    assert d["config"]["N"] == 64 and d["config"]["P"] == 8
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-9 * d["ms_per_step"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root,
                         env=dict(env, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"))
    assert out.returncode == 0 and out.stdout.strip() == "", (out.stdout, out.stderr[-2000:])


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc, s.lines = _DoneProc(), list(lines)
    return s


def test_clock_summary_median_under_load_and_active_reasons():
    """nvidia-smi samples: the median SM clock over loaded samples (idle ones,
    below half the highest, are left out), the maximum clock, and every
    throttle reason seen active in any sample; malformed lines are skipped."""
    lines = [
        "345, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = _sampler(lines).stop()
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["samples"] == 4
    assert c["reasons"] == ["sw_power_cap"]
    hot = _sampler(["1500, 2070, 1000, 0x48, Not Active, Active, Active, Not Active"]).stop()
    assert hot["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_or_nvidia_smi():
    assert _sampler([]).stop()["reasons"] == ["no samples"]
    none = bench.ClockSampler(0)
    assert none.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}


def test_cpu_context_reports_every_workload():
    """The CPU-oracle context of the bench line: single-thread samples of the
    small trapped and helium workloads, the replica batch over spawned
    processes on all host cores, and Algorithm 2 against Algorithm 1 (small
    sizes here to keep the test short)."""
    args = types.SimpleNamespace(he_cells=2, he_P=8, batch_replicas=6)
    c = bench.cpu_context(args, seconds=0.05, alg2_sizes=(16, 32))
    for key in ("trapped_N16_P8_beta2", "trapped_N64_P32_beta1", "helium_exchange", "batched_256_replicas"):
        assert "error" not in c[key], c[key]
        assert c[key]["value"] > 0 and c[key]["cores"] >= 1
    assert c["batched_256_replicas"]["replica_evals_per_s"] == pytest.approx(6 * c["batched_256_replicas"]["value"])
    rows = c["algorithm2_vs_algorithm1"]
    assert set(rows) == {"N16_P32", "N32_P32"}
    assert all(r["algorithm2_ms"] > 0 and r["algorithm1_ms"] > 0 for r in rows.values())
    json.dumps(c)


@pytest.mark.parametrize("prec,bound", [("fp64", "fp64"), ("mixed", "int"), ("mixed32", "fp32")])
def test_every_stage_has_a_roofline_fraction(prec, bound, monkeypatch):
    monkeypatch.setattr(bench, "load_traffic", lambda k: None)
    units = {"fp64_fma_per_s": 1e12, "int_mad_per_s": 2e13}
    st = bench.roofline_stages([0.014, 0.096, 0.019], ARGS, 2070.0, PEAKS, units, prec)
    assert set(st) == {"prep", "recursions", "prob_forces"}
    for r in st.values():
        assert r["frac"] is not None and r["frac"] > 0
    assert st["prep"]["bound"] == "hbm"
    assert st["recursions"]["achieved"] == pytest.approx(1024 / 0.096e-3)
    assert st["recursions"]["cycles_per_step"] == pytest.approx(0.096e-3 / 1024 * 2070e6)
    assert st["prob_forces"]["bound"] == bound
    pairs = 1024 * 1025 / 2
    if prec == "fp64":
        assert st["prob_forces"]["achieved"] == pytest.approx(bench.PROB_F64_OPS * pairs / 0.019e-3)
        assert st["prep"]["fp64_pipe_frac"] == pytest.approx(bench.G_F64_OPS * pairs / 0.014e-3 / 1e12)
