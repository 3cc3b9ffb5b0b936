"""Autotuner of the batched launch shapes.

``tune`` picks the grid caps of the batched exchange passes
(bpimd_batch_set_tuning); ``tune_pair_tile`` picks the tile of the batch's MD
pair forces, lanes per particle (bpimd_batch_set_pair_tile).

The batched pair-factor and probability passes run a grid-stride loop over
(replica, block) tables; how many CTAs per SM they launch trades occupancy
against tail imbalance, and the best value depends on the batch (how many
blocks, how uneven) and on the GPU.  ``tune`` times a few candidates with CUDA
events on the engine's own stream and keeps the fastest; results are cached in
a JSON file keyed by GPU name, precision and a signature of the batch, so a
later run with the same kind of batch skips the timing.  The choice never
changes the numbers (every block's partial sums and the order in which they
are combined are fixed), only the time.
"""
import json
import os
import statistics

import torch

CANDIDATES = ((2, 2), (4, 4), (8, 8), (16, 16), (4, 8), (8, 16), (16, 8), (32, 32))


def cache_path():
    return os.environ.get("BPIMD_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bpimd", "autotune.json"))


def batch_key(engine):
    """GPU, precision and a coarse signature of the batch: R, sum N, sum N^2/32^2 blocks, sum N P."""
    name = torch.cuda.get_device_name(engine.device)
    blocks = sum(((n + 31) // 32) * ((n + 31) // 32 + 1) // 2 for n in engine.N)
    beads = sum(n * p for n, p in zip(engine.N, engine.P))
    return f"{name}|{engine.precision}|R={engine.R}|blocks={blocks}|beads={beads}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, table):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(engine, positions, reps=5, candidates=CANDIDATES, use_cache=True):
    """Pick (pair_blocks_per_sm, prob_blocks_per_sm) for a BatchedExchangeEnergy.

    Returns a dict with the choice, the median milliseconds of every candidate
    (empty when taken from the cache) and whether the cache answered."""
    path = cache_path()
    key = batch_key(engine)
    table = _load(path) if use_cache else {}
    if key in table:
        choice = tuple(table[key]["choice"])
        engine.set_tuning(*choice)
        return {"choice": choice, "timings_ms": {}, "cached": True, "key": key}
    F = torch.empty_like(positions)
    V = torch.empty(engine.R, dtype=torch.float64, device=engine.device)
    stream = engine.stream
    timings = {}
    for cand in candidates:
        engine.set_tuning(*cand)
        engine.forces(positions, out=F, V_out=V)  # warm-up
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            engine.forces(positions, out=F, V_out=V)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        timings[f"{cand[0]},{cand[1]}"] = statistics.median(ms)
    best = min(candidates, key=lambda c: timings[f"{c[0]},{c[1]}"])
    engine.set_tuning(*best)
    engine.sync()
    if use_cache:
        table = _load(path)
        table[key] = {"choice": list(best), "timings_ms": timings}
        _save(path, table)
    return {"choice": best, "timings_ms": timings, "cached": False, "key": key}


PAIR_TILES = (2, 4, 8)  # lanes per particle of the batched MD pair forces


def tune_pair_tile(engine, positions, velocities, steps=3, reps=3, candidates=PAIR_TILES, use_cache=True):
    """Pick the pair tile (lanes per particle) of a BatchedExchangeEnergy's MD.

    Each candidate runs ``steps`` BAOAB steps of scratch copies of the given
    positions and velocities (the caller's tensors are not touched), timed
    with CUDA events on the engine's stream; the fastest median wins.  The
    thermostat counter advances during the trials.  Cached like ``tune``
    (GPU, precision, batch signature, plus an ``md-pair-tile`` tag)."""
    path = cache_path()
    key = batch_key(engine) + "|md-pair-tile"
    table = _load(path) if use_cache else {}
    if key in table:
        choice = int(table[key]["choice"])
        engine.set_pair_tile(choice)
        return {"choice": choice, "timings_ms": {}, "cached": True, "key": key}
    x = positions.clone()
    v = velocities.clone()
    stream = engine.stream
    timings = {}
    for cand in candidates:
        engine.set_pair_tile(cand)
        engine.step(x, v, steps, energies=False)  # warm-up (and the graph capture)
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            engine.step(x, v, steps, energies=False)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        timings[str(cand)] = statistics.median(ms)
    best = min(candidates, key=lambda c: timings[str(c)])
    engine.set_pair_tile(best)
    engine.sync()
    if use_cache:
        table = _load(path)
        table[key] = {"choice": best, "timings_ms": timings}
        _save(path, table)
    return {"choice": best, "timings_ms": timings, "cached": False, "key": key}
