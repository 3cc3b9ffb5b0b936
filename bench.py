#!/usr/bin/env python
"""Throughput of the bosonic exchange potential + forces on GB300.

Metric: exchange V_B + force evaluations per second for N = 1024 bosons with
P = 32 beads (beta = 1, m = hbar = 1, omega_P = sqrt(P)/beta), trapped-boson
positions (centres N(0,1), bead offsets N(0,0.1), seed 3), in the mixed form
(float32 bead differences and spring energies, everything after them at
float64 accuracy: the reported `value`), the plain float64 form (`fp64`) and
the fastest form with float32 pair factors and 32-bit recursion steps
(`mixed32`).  A step is one full evaluation: bead pass with pair factors, forward
and backward recursions with the prefix sums and V_B, probabilities with all
exterior-bead forces.  The line also carries MD steps/s (`md`) of the same
system with a trap and Gaussian repulsion (bpimd_step, CUDA-graph replays),
the throughput of a 256-replica batch of uneven N, P, beta (`batched`), and
MD steps/s of bulk liquid helium in a periodic box (`helium`).  `cpu_baseline`
is the CPU oracle on the headline workload; `cpu_context` times it on the other
workloads (small trapped systems, helium, the replica batch on all host cores)
and sets the paper's original O(P N^3) method against Algorithm 1.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas of the same workload (the
single-system evaluation does not shard); `value` is the sum over ranks.
`--impl reference` times the CPU oracle (Algorithm 1 in float64, one core) on
the same workload on rank 0.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exchange V_B+force evals/s at N=1024,P=32 (mixed vs FP64 GPU); MD steps/s"
N_DEF, P_DEF, BETA_DEF, SEED_DEF = 1024, 32, 1.0, 3
LAUNCHES_PER_EVAL = 4          # bead pass + pair factors, tile inverses, recursions (2 clusters), probabilities + forces
BATCH_LAUNCHES_PER_EVAL = 3    # replica batch: bead pass + pair factors, recursions, probabilities + forces
BATCH_MD = dict(dt=0.01, gamma=1.0, omega0=1.0, gaussian=(1.0, 0.5), seed=77)  # 256-replica workload
DFMA_LATENCY_CYCLES = 64       # measured on GB300: dependent float64 FMA latency
FLUSH_BYTES = 256 << 20        # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--P", type=int, default=P_DEF)
    ap.add_argument("--beta", type=float, default=BETA_DEF)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bounded CPU-oracle sample for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--md-steps", type=int, default=200, help="timed MD steps (mixed; float64 runs a quarter)")
    ap.add_argument("--batch-replicas", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=50, help="timed evaluations of the replica batch")
    ap.add_argument("--he-cells", type=int, default=10, help="FCC cells per side of the helium box (4 atoms each)")
    ap.add_argument("--he-P", type=int, default=64)
    ap.add_argument("--he-steps", type=int, default=20, help="timed helium MD steps (mixed; float64 a fifth)")
    ap.add_argument("--only", choices=["all", "headline", "md", "batched", "helium"], default="all",
                    help="run the headline exchange and only this one of the other workloads (for profiling)")
    return ap.parse_args()


def workload(args):
    return {"workload": f"trapped bosons N={args.N} P={args.P} beta={args.beta:g}: exchange V_B + all bead forces",
            "N": args.N, "P": args.P, "beta": args.beta, "m": 1.0, "hbar": 1.0,
            "positions": f"centres N(0,1), bead offsets N(0,0.1), seed {SEED_DEF}",
            "parallelism": "independent replicas, one per GPU"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for name, val in zip(names, p[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ roofline
def load_traffic(kernel):
    """dram bytes per launch from the committed ncu summary, if the kernel's
    sources are unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    ent = tab.get(kernel)
    if not ent:
        return None
    h = hashlib.sha256()
    for rel in ent.get("sources", []):
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        except OSError:
            return None
    if h.hexdigest() != ent.get("sources_sha256"):
        return None
    return ent.get("dram_bytes_per_launch")


def step_latency(t, N, clock):
    """Per-step latency of the recursions: the stage time t (s) spread over
    its N dependent steps, in ns and in SM cycles at the sampled clock (Hz),
    beside the reference floor of one dependent float64 FMA."""
    return {"ns_per_step": t / N * 1e9, "cycles_per_step": t / N * clock,
            "floor_cycles_per_step": DFMA_LATENCY_CYCLES}


def roofline(stage_ms_per_eval, args, sm_mhz, peaks, precision="mixed"):
    """Roofline object for the dominant stage."""
    import numpy as np
    from paper_2305_18025_gb300.bpimd import STAGE_NAMES
    i = int(np.argmax(stage_ms_per_eval))
    name = STAGE_NAMES[i]
    t = stage_ms_per_eval[i] * 1e-3
    N, P = args.N, args.P
    clock = (sm_mhz or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    if name == "recursions":
        # N dependent steps per chain (forward and backward run concurrently).
        # Reference floor: one dependent float64 FMA (64 cycles) per step; the
        # chain itself runs on the integer pipe (a 64-bit mantissa
        # multiply-add plus a shuffle, ~100 cycles per step measured alone).
        achieved = N / t
        peak = clock / DFMA_LATENCY_CYCLES
        obj = {"bound": "alu",
               "kind": "dependent-latency (integer-pipe chain; floor: one 64-cycle float64 FMA per step)",
               "achieved": achieved, "peak": peak, "unit": "chain steps/s",
               "frac": achieved / peak,
               "peak_source": f"measured DFMA latency {DFMA_LATENCY_CYCLES} cycles at the sampled SM clock"}
        obj.update(step_latency(t, N, clock))
    elif name == "prep":
        # positions read once, interior forces written, the per-particle
        # state, and both copies of g (mantissa + int exponent per pair)
        mant = 4 if precision == "mixed32" else 8
        bytes_ = (N * P * 24 + N * max(P - 2, 0) * 24 + N * 8 * 10
                  + 2 * (N * (N + 1) // 2) * (mant + 4))
        achieved = bytes_ / t / 1e9
        obj = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": achieved / peaks["hbm_gbs"], "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        pairs = N * (N + 1) / 2
        achieved = pairs / t
        obj = {"bound": "alu", "kind": "pair throughput", "achieved": achieved, "peak": None,
               "unit": "pairs/s", "frac": None}
    obj["kernel"] = name
    obj["traffic"] = load_traffic(name)
    return obj


# Counted per-pair work of the O(N^2) stages (thread-level operations of the
# kernels as written; the counts are listed with the kernels' rooflines):
#   probability pass, float64: 13 float64 ops per pair (bead differences,
#     Pr = alpha mu g, row and column terms) + 20 float64 adds of the column
#     butterfly (4 sums x 5 levels, every lane) = 33 float64 ops;
#   probability pass, mixed: 2 64 x 64-bit high products (alpha mu, then g)
#     = 8 integer 32 x 32 -> 64 multiply-adds per pair;
#   probability pass, mixed32: float32 only (12 ops per pair + 20 butterfly adds);
#   pair factors, float64: 6 float64 ops per pair (difference and square);
#   pair factors, mixed: the 128-bit product and 6 64-bit high products of
#     the integer power (pow2_fixed.cuh) = 28 integer multiply-adds.
PROB_F64_OPS, PROB_MIXED_IMADS, PROB_M32_F32OPS = 33, 8, 32
G_F64_OPS, G_MIXED_IMADS = 6, 28


def measure_unit_peaks(dev, stream, iters=2000):
    """Throughput of the float64 pipe and of 32-bit integer multiply-adds over
    the whole GPU, by the library's probe kernels (CUDA events, best of 3)."""
    import torch
    from paper_2305_18025_gb300 import bpimd
    sink = torch.empty(8 * 8 * 256, dtype=torch.float64, device=dev)
    out = {}
    for kind, name in ((0, "fp64_fma_per_s"), (1, "int_mad_per_s")):
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = bpimd.bpimd_peak_probe(kind, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            rate = ops / (e0.elapsed_time(e1) * 1e-3)
            best = rate if best is None else max(best, rate)
        out[name] = best
    return out


def roofline_stages(stage_ms_per_eval, args, sm_mhz, peaks, unit_peaks, precision):
    """A roofline fraction for each stage of one evaluation: the bead pass
    with pair factors against HBM (and, in float64, the float64 pipe), the
    recursions against their dependent-step floor, the probability pass
    against the unit its per-pair work loads (counts above)."""
    N = args.N
    pairs = N * (N + 1) / 2
    t_prep, t_rec, t_prob = (x * 1e-3 for x in stage_ms_per_eval)
    prep = roofline([1.0, 0.0, 0.0], args, sm_mhz, peaks, precision)  # HBM bytes of the stage
    prep["achieved"] = prep["achieved"] * 1e-3 / t_prep  # roofline() was given 1 ms
    prep["frac"] = prep["achieved"] / prep["peak"]
    if precision == "fp64":
        prep["fp64_pipe_frac"] = G_F64_OPS * pairs / t_prep / unit_peaks["fp64_fma_per_s"]
    elif precision == "mixed":
        prep["int_pipe_frac"] = G_MIXED_IMADS * pairs / t_prep / unit_peaks["int_mad_per_s"]
    rec = roofline([0.0, 1.0, 0.0], args, sm_mhz, peaks, precision)
    rec["achieved"] = N / t_rec
    rec["frac"] = rec["achieved"] / rec["peak"]
    rec.update(step_latency(t_rec, N, (sm_mhz or peaks.get("sm_max_mhz", 2070.0)) * 1e6))
    if precision == "fp64":
        prob = {"bound": "fp64", "unit": "float64 ops/s", "achieved": PROB_F64_OPS * pairs / t_prob,
                "peak": unit_peaks["fp64_fma_per_s"], "peak_source": "library float64 FMA probe (measured)"}
    elif precision == "mixed":
        prob = {"bound": "int", "unit": "32-bit integer multiply-adds/s", "achieved": PROB_MIXED_IMADS * pairs / t_prob,
                "peak": unit_peaks["int_mad_per_s"], "peak_source": "library integer multiply-add probe (measured)"}
    else:
        fp32_peak = (sm_mhz or peaks.get("sm_max_mhz", 2070.0)) * 1e6 * 152 * 128
        prob = {"bound": "fp32", "unit": "float32 ops/s", "achieved": PROB_M32_F32OPS * pairs / t_prob,
                "peak": fp32_peak, "peak_source": "nominal 128 float32 lanes per SM x 152 SMs x sampled clock"}
    prob["frac"] = prob["achieved"] / prob["peak"]
    prob["kernel"] = "prob_forces"
    for r in (prep, rec):
        r.pop("traffic", None)
    return {"prep": prep, "recursions": rec, "prob_forces": prob}


# ----------------------------------------------------- replicas across ranks
def reduce_max(x, dist, device):
    """The largest of every rank's x (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, units_per_rank, slowest_seconds):
    """Whole-job throughput of independent replicas: every rank processes
    units_per_rank units; the job takes as long as its slowest rank."""
    return world * units_per_rank / slowest_seconds


# ------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2305_18025_gb300 import bpimd, inputs
    from paper_2305_18025_gb300.exchange import ExchangeEnergy

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, dist, dev)

    N, P, beta = args.N, args.P, args.beta
    wP = inputs.omega_P(P, beta)
    pos_np = inputs.trapped_positions(N, P, SEED_DEF)
    pos = torch.from_numpy(pos_np).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        peaks = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}

    sampler = ClockSampler(local_rank)
    sampler.start()
    results = {}
    unit_peaks = measure_unit_peaks(dev, torch.cuda.current_stream(dev))
    # the context's own stream (as an application would bind one); the L2
    # flush and the timing events go on the same stream
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for prec in ("mixed", "fp64", "mixed32"):
            eng = ExchangeEnergy(N, P, 1.0, wP, beta, precision=prec, device=dev, stream=stream)
            F = torch.empty_like(pos)
            V = torch.empty((), dtype=torch.float64, device=dev)
            for _ in range(args.warmup):
                flush.fill_(1)
                eng.forces(pos, out=F, V_out=V)
            eng.sync()
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            bpimd.bpimd_profile_begin(eng.ctx, args.steps)
            barrier()
            torch.cuda.synchronize(dev)
            t_wall0 = time.perf_counter()
            for k in range(args.steps):
                flush.fill_(k & 255)          # untimed: evict L2 between steps
                starts[k].record(stream)
                eng.forces(pos, out=F, V_out=V)
                ends[k].record(stream)
            torch.cuda.synchronize(dev)
            barrier()
            wall = time.perf_counter() - t_wall0
            stage_ms, n_prof = bpimd.bpimd_profile_end(eng.ctx)
            eng.sync()
            step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
            total_ms = max_over_ranks(sum(step_ms))
            results[prec] = {
                "value": aggregate_rate(world, args.steps, total_ms * 1e-3),
                "ms_per_step": total_ms / args.steps,
                "median_ms": statistics.median(step_ms),
                "stage_ms": (stage_ms / max(n_prof, 1)).tolist(),
                "wall_s": wall,
                "V_B": float(V.item()),
            }
            # end-to-end through the host entry point (pinned buffers), same metric
            if prec == "mixed":
                pos_h = torch.from_numpy(pos_np.copy()).pin_memory()
                F_h = torch.empty_like(pos_h).pin_memory()
                for _ in range(args.warmup):
                    eng.forces_host(pos_h, F_h)
                barrier()
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    eng.forces_host(pos_h, F_h)
                e2e_s = max_over_ranks(time.perf_counter() - t0)
                barrier()
                results["e2e"] = {"value": aggregate_rate(world, args.steps, e2e_s), "unit": "evals/s",
                                  "h2d_bytes_per_step": pos_h.numel() * 8,
                                  "d2h_bytes_per_step": F_h.numel() * 8 + 8,
                                  "api": "bpimd_exchange_energy_forces_host (pinned host buffers; the call "
                                         "replays one captured CUDA graph of copies and kernels)"}
            eng.close()
    def want(name):
        return args.only in ("all", name)

    results["md"] = md_throughput(args, pos_np, wP, dev, max_over_ranks, barrier, world) if want("md") else {}
    results["batched"] = batched_throughput(args, dev, flush, max_over_ranks, barrier, world) if want("batched") else {}
    results["helium"] = helium_throughput(args, dev, flush, max_over_ranks, barrier, world) if want("helium") else {}
    clocks = sampler.stop()

    if rank != 0:
        return None
    mixed, fp64, m32 = results["mixed"], results["fp64"], results["mixed32"]
    from paper_2305_18025_gb300.bpimd import STAGE_NAMES
    roof = roofline(mixed["stage_ms"], args, clocks.get("sm_mhz"), peaks, "mixed")
    line = {
        "metric": METRIC, "value": mixed["value"], "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES["mixed"], "data": "synthetic",
        "config": workload(args),
        "precision": "mixed",
        "timing": {"l2": "flushed between timed steps (256 MiB device write, untimed)",
                   "stream": "a dedicated CUDA stream bound to the context (flush and events on it)"},
        "gpu_launches": LAUNCHES_PER_EVAL * args.steps,
        "clocks": clocks,
        "e2e": results["e2e"],
        "roofline": roof,
        "unit_peaks": unit_peaks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, pos_np, wP)
        line["cpu_context"] = cpu_context(args)
    line.update({
        "stages_ms": {p: dict(zip(STAGE_NAMES, results[p]["stage_ms"])) for p in ("mixed", "fp64", "mixed32")},
        "roofline_stages": {p: roofline_stages(results[p]["stage_ms"], args, clocks.get("sm_mhz"), peaks, unit_peaks, p)
                            for p in ("mixed", "fp64", "mixed32")},
        "V_B": {p: results[p]["V_B"] for p in ("mixed", "fp64", "mixed32")},
        "batched": results["batched"],
        "helium": results["helium"],
        "md": results["md"],
        "fp64": {"value": fp64["value"], "unit": "evals/s", "ms_per_step": fp64["ms_per_step"],
                 "dtype": DTYPES["fp64"],
                 "roofline": roofline(fp64["stage_ms"], args, clocks.get("sm_mhz"), peaks, "fp64")},
        "mixed32": {"value": m32["value"], "unit": "evals/s", "ms_per_step": m32["ms_per_step"],
                    "dtype": DTYPES["mixed32"],
                    "roofline": roofline(m32["stage_ms"], args, clocks.get("sm_mhz"), peaks, "mixed32")},
    })
    # the headline figures once more, last, so that a truncated log keeps them
    line["summary"] = {
        "evals_per_s": {"mixed": mixed["value"], "fp64": fp64["value"], "mixed32": m32["value"],
                        "e2e_mixed": results["e2e"]["value"]},
        "md_steps_per_s": {p: results["md"][p]["value"] for p in ("mixed", "fp64", "mixed32") if p in results["md"]},
        "batched_evals_per_s": {p: results["batched"][p]["value"] for p in ("mixed", "fp64", "mixed32")
                                if p in results["batched"]},
        "batched_md_steps_per_s": {p: v["value"] for p, v in results["batched"].get("md", {}).items()
                                   if p in ("mixed", "fp64")},
        "helium_md_steps_per_s": {p: results["helium"][p]["value"] for p in ("mixed", "fp64", "mixed32")
                                  if p in results["helium"]},
        "helium_exchange_evals_per_s": {k: v["value"] for k, v in results["helium"].get("exchange", {}).items()
                                        if isinstance(v, dict) and "value" in v},
        "recursion_frac": roof["frac"] if roof["kernel"] == "recursions" else None,
        "recursion_cycles_per_step": roof.get("cycles_per_step"),
    }
    return line


# arithmetic of each precision form (what the path computes in)
DTYPES = {
    "mixed": "f32+f64+u64 (float32 bead differences and spring energies; float64-accurate pair factors, "
             "64-bit integer recursions, integer-mantissa probabilities, "
             "compensated float32-pair force sums)",
    "fp64": "f64+u64 (float64, with 64-bit integer recursions and integer-pipe pair factors)",
    "mixed32": "f32+u64+f64 (float32 pair factors, recursion bulk sums and probabilities; 64-bit integer "
               "tile products; float64 prefix sums and outputs)",
}


MD_CFG = dict(dt=0.01, gamma=1.0, omega0=1.0, gaussian=(3.0, 0.5), seed=7)


def md_throughput(args, pos_np, wP, dev, max_over_ranks, barrier, world):
    """MD steps/s of the same system with a harmonic trap (w0 = 1) and Gaussian
    repulsion (g = 3, s = 0.5): bpimd_step replaying one captured CUDA graph per
    step (BAOAB + exchange force + pair force), mixed and float64."""
    import torch
    from paper_2305_18025_gb300.exchange import RingPolymerMD
    out = {}
    for prec, steps in (("mixed", args.md_steps), ("fp64", max(1, args.md_steps // 4)),
                        ("mixed32", args.md_steps)):
        side = torch.cuda.Stream(dev)
        md = RingPolymerMD(args.N, args.P, 1.0, wP, args.beta, precision=prec, stream=side, **MD_CFG)
        x = torch.from_numpy(pos_np.copy()).to(dev)
        v = torch.zeros_like(x)
        md.step(x, v, 5, energies=False)            # warm-up, graph capture
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(side)
        md.step(x, v, steps, energies=False)
        e1.record(side)
        torch.cuda.synchronize(dev)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        en = md.step(x, v, 1).cpu().tolist()
        md.close()
        out[prec] = {"value": aggregate_rate(world, steps, ms * 1e-3), "unit": "MD steps/s", "steps": steps,
                     "gpu_launches": (LAUNCHES_PER_EVAL + 3) * steps + LAUNCHES_PER_EVAL + 1,
                     "ms_per_step": ms / steps, "energies_after": dict(zip(["V_B", "U_bar", "kinetic", "E_prim"], en))}
    out["config"] = {"workload": f"trapped bosons N={args.N} P={args.P} beta={args.beta:g}, harmonic trap w0=1, "
                                 "Gaussian repulsion g=3 s=0.5 between equal-index beads",
                     "integrator": "BAOAB Langevin, dt=0.01, gamma=1, kT=1/beta, Philox4x32-10 noise",
                     "timing": "CUDA events around one bpimd_step call (one initial force evaluation + "
                               "the steps as CUDA-graph replays); L2 not flushed between MD steps, "
                               "which run back to back as in a production trajectory"}
    return out


def batched_throughput(args, dev, flush, max_over_ranks, barrier, world):
    """256 independent trapped replicas, N ~ U[16,512], P in {16,32,64},
    beta ~ U[0.5,4] (seed 11), evaluated together (bpimd_create_batched),
    launch shape picked by the autotuner; L2 flushed between timed batches."""
    import torch
    from paper_2305_18025_gb300 import autotune, inputs
    from paper_2305_18025_gb300.exchange import BatchedExchangeEnergy
    reps = inputs.batched_replicas(args.batch_replicas, seed=11)
    Ns = [r.N for r in reps]
    Ps = [r.P for r in reps]
    betas = [r.beta for r in reps]
    wPs = [inputs.omega_P(P, b) for P, b in zip(Ps, betas)]
    out = {}
    for prec in ("mixed", "fp64", "mixed32"):
        eng = BatchedExchangeEnergy(Ns, Ps, 1.0, wPs, betas, precision=prec, device=dev)
        x = eng.pack([torch.from_numpy(r.positions) for r in reps])
        tuned = autotune.tune(eng, x, reps=3)
        F = torch.empty_like(x)
        V = torch.empty(eng.R, dtype=torch.float64, device=dev)
        stream = eng.stream
        for _ in range(args.warmup):
            flush.fill_(1)
            eng.forces(x, out=F, V_out=V)
        steps = args.batch_steps
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.fill_(k & 255)
            starts[k].record(stream)
            eng.forces(x, out=F, V_out=V)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        eng.sync()
        ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
        out[prec] = {"value": aggregate_rate(world, steps, ms * 1e-3), "unit": "batch evals/s",
                     "replica_evals_per_s": aggregate_rate(world, steps * eng.R, ms * 1e-3),
                     "ms_per_batch": ms / steps, "steps": steps, "gpu_launches": BATCH_LAUNCHES_PER_EVAL * steps,
                     "tuning": {"choice": list(tuned["choice"]), "cached": tuned["cached"]}}
        eng.close()
    out["md"] = batched_md_throughput(args, dev, reps, wPs, max_over_ranks, barrier, world)
    out["config"] = {"workload": f"{args.batch_replicas} independent trapped replicas, N~U[16,512], "
                                 "P in {16,32,64}, beta~U[0.5,4], seed 11 (exchange V_B + all bead forces of each)",
                     "sum_N": int(sum(Ns)), "sum_NP": int(sum(n * p for n, p in zip(Ns, Ps))),
                     "sum_pairs": int(sum(n * (n + 1) // 2 for n in Ns)),
                     "l2": "flushed between timed batches (256 MiB device write, untimed)"}
    return out


def batched_md_throughput(args, dev, reps, wPs, max_over_ranks, barrier, world):
    """BAOAB molecular dynamics of the whole replica batch: harmonic trap w0 = 1
    and Gaussian repulsion g = 1, s = 0.5 between equal-index beads, each
    replica thermostatted at its own beta; the steps are CUDA-graph replays on
    a dedicated stream (batch evaluation, pair forces, integrator: 6 launches
    per step), with the pair tile (lanes per particle) picked by the
    autotuner on scratch copies first.  Back to back as in a trajectory, so
    the L2 is not flushed."""
    import numpy as np
    import torch
    from paper_2305_18025_gb300 import autotune
    from paper_2305_18025_gb300.exchange import BatchedExchangeEnergy
    Ns, Ps, betas = [r.N for r in reps], [r.P for r in reps], [r.beta for r in reps]
    out = {}
    for prec, steps in (("mixed", max(4, args.batch_steps)), ("fp64", max(4, args.batch_steps // 4))):
        side = torch.cuda.Stream(dev)
        eng = BatchedExchangeEnergy(Ns, Ps, 1.0, wPs, betas, precision=prec, device=dev, stream=side, md=BATCH_MD)
        rng = np.random.default_rng(12)
        x = eng.pack([torch.from_numpy(r.positions) for r in reps])
        v = eng.pack([torch.from_numpy(rng.normal(0.0, 1.0 / np.sqrt(r.beta), r.positions.shape)) for r in reps])
        tuned = autotune.tune_pair_tile(eng, x, v, steps=2, reps=2)
        eng.step(x, v, max(2, args.warmup), energies=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(side)
        eng.step(x, v, steps, energies=False)
        e1.record(side)
        torch.cuda.synchronize(dev)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        en = eng.step(x, v, 1).cpu().numpy()
        eng.close()
        out[prec] = {"value": aggregate_rate(world, steps, ms * 1e-3), "unit": "batch MD steps/s", "steps": steps,
                     "replica_steps_per_s": aggregate_rate(world, steps * len(reps), ms * 1e-3),
                     "ms_per_step": ms / steps, "gpu_launches": (BATCH_LAUNCHES_PER_EVAL + 3) * steps,
                     "finite": bool(np.isfinite(en).all()),
                     "tuning": {"pair_tile_lanes": int(tuned["choice"]), "cached": tuned["cached"],
                                "timings_ms": tuned["timings_ms"]},
                     "mean_E_prim_per_bead": float(np.mean(en[:, 3] / np.array([n * p for n, p in zip(Ns, Ps)])))}
    out["config"] = {"workload": "the same 256 replicas, harmonic trap w0=1 and Gaussian repulsion g=1 s=0.5 "
                                 "between equal-index beads",
                     "integrator": "BAOAB Langevin, dt=0.01, gamma=1, kT=1/beta of each replica, Philox4x32-10 noise",
                     "timing": "CUDA events around one bpimd_step call on a dedicated stream (CUDA-graph replays)"}
    return out


HE = dict(m=4.0026, T=1.5, eps=10.22, sigma=2.556, rho=0.0218, hbar=6.9648)  # A, K, amu units


def helium_throughput(args, dev, flush, max_over_ranks, barrier, world):
    """Bulk liquid helium: FCC start (10^3 cells, 4000 atoms) at 0.0218 A^-3,
    P = 64, T = 1.5 K, Lennard-Jones eps = 10.22 K, sigma = 2.556 A cut and
    shifted at 2.5 sigma (cell lists), periodic box with minimum-image springs,
    BAOAB dt = 1 fs.  MD steps/s, mixed and float64."""
    import numpy as np
    import torch
    from paper_2305_18025_gb300 import inputs
    from paper_2305_18025_gb300.exchange import RingPolymerMD
    cells, P = args.he_cells, args.he_P
    N = 4 * cells ** 3
    L = (N / HE["rho"]) ** (1.0 / 3.0)
    beta = 1.0 / HE["T"]
    wP = np.sqrt(P) / (beta * HE["hbar"])
    dt = 1e-15 / 1.0967e-12  # 1 fs in units of A sqrt(amu/K)
    pos = inputs.fcc_positions(cells, P, L, seed=5, jitter=0.05)
    lj = (HE["eps"], HE["sigma"], 2.5 * HE["sigma"])
    out = {}
    for prec, steps in (("mixed", args.he_steps), ("fp64", max(1, args.he_steps // 5)),
                        ("mixed32", args.he_steps)):
        side = torch.cuda.Stream(dev)
        md = RingPolymerMD(N, P, HE["m"], wP, beta, dt=dt, gamma=1.0, lennard_jones=lj, box=L, seed=3,
                           precision=prec, stream=side)
        x = torch.from_numpy(pos.copy()).to(dev)
        v = torch.zeros_like(x)
        md.step(x, v, 3, energies=False)  # warm-up, graph capture
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(side)
        md.step(x, v, steps, energies=False)
        e1.record(side)
        torch.cuda.synchronize(dev)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        en = md.step(x, v, 1).cpu().tolist()
        md.close()
        out[prec] = {"value": aggregate_rate(world, steps, ms * 1e-3), "unit": "MD steps/s", "steps": steps,
                     "ms_per_step": ms / steps,
                     "energies_after_K": dict(zip(["V_B", "U_bar", "kinetic", "E_prim"], en))}
    out["exchange"] = helium_exchange(args, dev, flush, pos, HE["m"], wP, beta, L, max_over_ranks, barrier, world)
    out["config"] = {"workload": f"liquid helium N={N} (FCC {cells}^3 x 4) P={P} T=1.5 K rho=0.0218/A^3 "
                                 f"box {L:.2f} A, Lennard-Jones eps=10.22 K sigma=2.556 A cut+shift 2.5 sigma",
                     "integrator": "BAOAB Langevin dt=1 fs gamma=1 (A, K, amu units), Philox noise",
                     "timing": "CUDA events around one bpimd_step call (one initial force evaluation + graph "
                               "replays); L2 not flushed between MD steps"}
    return out


def helium_exchange(args, dev, flush, pos, m, wP, beta, L, max_over_ranks, barrier, world, steps=10):
    """Exchange V_B + forces of the helium box alone (mixed form), with the
    pair factors tabulated (the default below N = 8192) and recomputed where
    they are used (no O(N^2) storage): evaluations/s, stage times, and the
    roofline of the recursions in recompute mode, whose DRAM traffic (from the
    committed ncu summary) is compared with the O(N P) algorithmic bytes
    (positions in, forces out)."""
    import torch
    from paper_2305_18025_gb300 import bpimd
    from paper_2305_18025_gb300.exchange import ExchangeEnergy
    N, P = pos.shape[0], pos.shape[1]
    x = torch.from_numpy(pos).to(dev)
    out = {}
    for name, rc in (("mixed_stored", False), ("mixed_recompute", True)):
        s = torch.cuda.Stream(dev)
        eng = ExchangeEnergy(N, P, m, wP, beta, precision="mixed", device=dev, stream=s, box=L, recompute=rc)
        F = torch.empty_like(x)
        V = torch.empty((), dtype=torch.float64, device=dev)
        with torch.cuda.stream(s):
            for _ in range(3):
                flush.fill_(1)
                eng.forces(x, out=F, V_out=V)
            eng.sync()
            bpimd.bpimd_profile_begin(eng.ctx, steps)
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
            barrier()
            torch.cuda.synchronize(dev)
            for k in range(steps):
                flush.fill_(k & 255)
                starts[k].record(s)
                eng.forces(x, out=F, V_out=V)
                ends[k].record(s)
            torch.cuda.synchronize(dev)
            barrier()
            stage_ms, n = bpimd.bpimd_profile_end(eng.ctx)
            eng.sync()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, ends)))
        out[name] = {"value": aggregate_rate(world, steps, ms * 1e-3), "unit": "evals/s", "ms_per_step": ms / steps,
                     "stages_ms": [x_ / max(n, 1) for x_ in stage_ms], "V_B": float(V.item())}
        eng.close()
    # O(N) algorithmic bytes of the two recursions in recompute mode: per
    # particle and recursion both float32 endpoint copies of the periodic
    # box (2 x 16 bytes), the coefficient c (12) and Y written (12); the
    # forward one also reads Ap, n (12) and writes C' (8).  The evaluation
    # as a whole moves O(N P): positions in, forces out (48 N P).
    algo_rec = N * (2 * (2 * 16 + 12 + 12) + 20)
    rec_t = out["mixed_recompute"]["stages_ms"][1] * 1e-3
    traffic = load_traffic("recursions_recompute_helium")
    out["roofline_recompute"] = {"kernel": "recursions (recompute mode)", "bound": "alu",
                                 "achieved": N / rec_t, "unit": "chain steps/s",
                                 "traffic": traffic, "algorithmic_bytes_O_N": algo_rec,
                                 "traffic_over_algorithmic": (traffic / algo_rec) if traffic else None,
                                 "stored_tables_bytes": 2 * (N * (N + 1) // 2) * 12,
                                 "eval_algorithmic_bytes_O_NP": 48 * N * P}
    return out


def cpu_baseline(args, pos_np, wP, seconds=None, max_evals=None):
    """The float64 oracle (Algorithm 1, single thread) on the host cores."""
    import oracle
    seconds = args.cpu_seconds if seconds is None else seconds
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.fast_pimdb(pos_np, 1.0, wP, args.beta)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_evals and n >= max_evals):
            break
    return {"value": n / el, "unit": "evals/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} full evaluations of the same workload in {el:.1f} s "
                      f"(C oracle, float64, single thread; host has {os.cpu_count()} cores)"}


def _timed_evals(fn, seconds, min_evals=1):
    """Call fn until `seconds` have passed (at least min_evals calls); evals/s and count."""
    n, t0 = 0, time.perf_counter()
    while True:
        fn()
        n += 1
        el = time.perf_counter() - t0
        if n >= min_evals and el >= seconds:
            return n / el, n, el


def _oracle_replicas(chunk):
    """Worker of the replica-batch baseline: the oracle on each (N, P, beta,
    seed) of its share, positions regenerated from the seed."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2305_18025_gb300 import inputs
    for N, P, beta, seed in chunk:
        oracle.fast_pimdb(inputs.trapped_positions(N, P, seed), 1.0, inputs.omega_P(P, beta), beta)
    return len(chunk)


def cpu_context(args, seconds=1.5, alg2_sizes=(64, 128, 256)):
    """The float64 oracle on the host cores for the other workloads of the
    measurement plan, each a bounded sample; context for the GPU figures, not a
    target.  Single thread: trapped N=16, P=8, beta=2 and N=64, P=32, beta=1;
    liquid helium N=4000, P=64 in its periodic box.  All host cores: the
    256-replica batch, one spawned process per core, replicas dealt round robin.
    The paper's original O(P N^3) method (Algorithm 2) against Algorithm 1 at
    N = 64, 128, 256, P = 32, one evaluation each, for the shape of the speedup.
    A failing item reports its error instead of a figure."""
    import multiprocessing
    import numpy as np
    import oracle
    from paper_2305_18025_gb300 import inputs
    out = {"kind": "oracle", "note": "float64 C oracle on this host's cores; bounded samples"}

    def guard(name, fn):
        try:
            out[name] = fn()
        except Exception as e:  # a baseline never fails the bench line
            out[name] = {"error": f"{type(e).__name__}: {e}"}

    def single(N, P, beta):
        pos, wP = inputs.trapped_positions(N, P, SEED_DEF), inputs.omega_P(P, beta)
        v, n, el = _timed_evals(lambda: oracle.fast_pimdb(pos, 1.0, wP, beta), seconds)
        return {"value": v, "unit": "evals/s", "cores": 1, "sample": f"{n} evaluations in {el:.2f} s"}

    guard("trapped_N16_P8_beta2", lambda: single(16, 8, 2.0))
    guard("trapped_N64_P32_beta1", lambda: single(64, 32, 1.0))

    def helium():
        he_N = 4 * args.he_cells ** 3
        L = (he_N / HE["rho"]) ** (1.0 / 3.0)
        beta = 1.0 / HE["T"]
        wP = np.sqrt(args.he_P) / (beta * HE["hbar"])
        x = inputs.fcc_positions(args.he_cells, args.he_P, L, 3)
        v, n, el = _timed_evals(lambda: oracle.float64.fast_pimdb(x, HE["m"], wP, beta, box=L), seconds)
        return {"value": v, "unit": "evals/s", "cores": 1,
                "sample": f"N={he_N} P={args.he_P} in a periodic box of {L:.2f} A: {n} evaluations in {el:.2f} s"}

    guard("helium_exchange", helium)

    def replicas():
        reps = inputs.batched_replicas(args.batch_replicas, seed=11)
        items = [(r.N, r.P, r.beta, 11 * 100003 + i) for i, r in enumerate(reps)]
        try:
            cores = len(os.sched_getaffinity(0))  # the CPUs this process may run on
        except AttributeError:
            cores = os.cpu_count() or 1
        cores = max(1, min(cores, 32))
        chunks = [items[c::cores] for c in range(cores)]

        def batch():  # bounded: a stuck worker becomes an error entry, not a hung bench
            return pool.map_async(_oracle_replicas, chunks).get(timeout=120)

        with multiprocessing.get_context("spawn").Pool(cores) as pool:
            batch()  # start-up and library load, untimed
            v, n, el = _timed_evals(batch, seconds)
        return {"value": v, "unit": "batch evals/s", "replica_evals_per_s": v * len(items), "cores": cores,
                "sample": f"{n} batches of {len(items)} replicas in {el:.2f} s, {cores} spawned processes"}

    guard("batched_256_replicas", replicas)

    def algorithm2():
        rows = {}
        for N in alg2_sizes:
            pos, wP = inputs.trapped_positions(N, 32, SEED_DEF), inputs.omega_P(32, 1.0)
            t0 = time.perf_counter()
            oracle.original_pimdb(pos, 1.0, wP, 1.0)
            t2 = time.perf_counter() - t0
            v1, _, _ = _timed_evals(lambda: oracle.fast_pimdb(pos, 1.0, wP, 1.0), 0.2)
            rows[f"N{N}_P32"] = {"algorithm2_ms": 1e3 * t2, "algorithm1_ms": 1e3 / v1, "ratio": t2 * v1}
        return rows

    guard("algorithm2_vs_algorithm1", algorithm2)
    return out


# ------------------------------------------------------ reference arm
def run_reference(args, rank):
    if rank != 0:
        return None
    from paper_2305_18025_gb300 import inputs
    wP = inputs.omega_P(args.P, args.beta)
    pos_np = inputs.trapped_positions(args.N, args.P, SEED_DEF)
    import oracle
    for _ in range(min(args.warmup, 3)):
        oracle.fast_pimdb(pos_np, 1.0, wP, args.beta)
    # bounded: at most ~120 s of oracle work however large --steps is
    t0 = time.perf_counter()
    oracle.fast_pimdb(pos_np, 1.0, wP, args.beta)
    one = time.perf_counter() - t0
    k = max(1, min(args.steps, int(120.0 / max(one, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(k):
        oracle.fast_pimdb(pos_np, 1.0, wP, args.beta)
    el = time.perf_counter() - t0
    value = k / el
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / k, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload(args),
        "precision": "fp64 (CPU oracle)",
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"{k} of {args.steps} requested steps timed (bounded to ~120 s); "
                                   f"C oracle Algorithm 1, float64, single thread, host has {os.cpu_count()} cores"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        from paper_2305_18025_gb300 import build as _b
        if not _b.up_to_date():
            if rank == 0:
                _b.build()
            if world > 1:
                # other ranks wait for rank 0's build
                for _ in range(600):
                    if _b.up_to_date():
                        break
                    time.sleep(1)
        line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
