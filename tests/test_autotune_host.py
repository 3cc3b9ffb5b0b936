"""Host logic of the batched-launch autotuner (no GPU): it picks the fastest
candidate by the median of its timed repetitions, applies it to the engine,
stores it under a key of GPU name, precision and batch shape, answers a later
call for the same kind of batch from that cache without timing anything, keeps
the entries of other keys, and treats an unreadable cache file as empty.  The
engine and the CUDA events are fakes; what is timed is the fake's clock."""
import json
import os

import pytest
import torch

from paper_2305_18025_gb300 import autotune


class FakeEngine:
    """Stands in for BatchedExchangeEnergy: a tuning, a forces call, a clock."""

    def __init__(self, N, P, precision="mixed", cost=None):
        self.N, self.P, self.R = list(N), list(P), len(N)
        self.precision, self.device, self.stream = precision, torch.device("cpu"), None
        self.tuning, self.calls, self.applied = None, 0, []
        self.clock = 0.0
        # milliseconds per evaluation for each (pair, prob) blocks-per-SM choice
        self.cost = cost or {}

    def set_tuning(self, a, b):
        self.tuning = (a, b)
        self.applied.append((a, b))

    def forces(self, positions, out=None, V_out=None):
        self.calls += 1
        self.clock += self.cost.get(self.tuning, 5.0)

    def sync(self):
        pass


@pytest.fixture
def fake_cuda(monkeypatch, tmp_path):
    engines = []

    class Event:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = engines[-1].clock

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "FakeGPU")
    monkeypatch.setenv("BPIMD_AUTOTUNE_CACHE", str(tmp_path / "cache" / "autotune.json"))
    return engines


def test_picks_the_fastest_candidate_and_answers_from_the_cache(fake_cuda):
    cost = {c: 3.0 + i for i, c in enumerate(autotune.CANDIDATES)}
    cost[(8, 16)] = 1.0
    eng = FakeEngine([100, 40, 513], [32, 16, 64], cost=cost)
    fake_cuda.append(eng)
    x = torch.zeros(3 * sum(n * p for n, p in zip(eng.N, eng.P)), dtype=torch.float64)
    res = autotune.tune(eng, x, reps=3)
    assert res["choice"] == (8, 16) and not res["cached"]
    assert eng.tuning == (8, 16)
    assert set(res["timings_ms"]) == {f"{a},{b}" for a, b in autotune.CANDIDATES}
    assert res["timings_ms"]["8,16"] == pytest.approx(1.0)
    assert eng.calls == len(autotune.CANDIDATES) * (1 + 3)  # one warm-up + reps per candidate

    stored = json.load(open(autotune.cache_path()))
    assert stored[res["key"]]["choice"] == [8, 16]
    assert res["key"].startswith("FakeGPU|mixed|R=3|")

    again = FakeEngine([100, 40, 513], [32, 16, 64])
    fake_cuda.append(again)
    res2 = autotune.tune(again, x, reps=3)
    assert res2["cached"] and res2["choice"] == (8, 16) and res2["timings_ms"] == {}
    assert again.calls == 0 and again.applied == [(8, 16)]


def test_keys_separate_precision_and_batch_shape(fake_cuda):
    a = FakeEngine([64, 64], [32, 32], "mixed")
    b = FakeEngine([64, 64], [32, 32], "fp64")
    c = FakeEngine([64, 65], [32, 32], "mixed")   # one more row tile
    d = FakeEngine([64, 64], [32, 16], "mixed")   # fewer beads
    keys = {autotune.batch_key(e) for e in (a, b, c, d)}
    assert len(keys) == 4
    # the signature is coarse on purpose: the same blocks and beads share an entry
    e = FakeEngine([64, 64], [16, 48], "mixed")
    assert autotune.batch_key(e) == autotune.batch_key(a)


def test_other_entries_survive_and_a_broken_cache_reads_as_empty(fake_cuda):
    path = autotune.cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write("{not json")
    eng = FakeEngine([32], [8], cost={(2, 2): 0.5})
    fake_cuda.append(eng)
    x = torch.zeros(3 * 32 * 8, dtype=torch.float64)
    res = autotune.tune(eng, x, reps=2)
    assert res["choice"] == (2, 2) and not res["cached"]
    table = json.load(open(path))
    assert list(table) == [res["key"]]

    other = FakeEngine([32], [8], "fp64", cost={(32, 32): 0.1})
    fake_cuda.append(other)
    res_o = autotune.tune(other, x, reps=2)
    assert res_o["choice"] == (32, 32)
    table = json.load(open(path))
    assert set(table) == {res["key"], res_o["key"]}
    assert table[res["key"]]["choice"] == [2, 2]


def test_use_cache_false_times_again_and_writes_nothing(fake_cuda):
    eng = FakeEngine([50], [4], cost={(4, 8): 0.2})
    fake_cuda.append(eng)
    x = torch.zeros(3 * 50 * 4, dtype=torch.float64)
    res = autotune.tune(eng, x, reps=1, use_cache=False)
    assert res["choice"] == (4, 8) and not res["cached"]
    assert not os.path.exists(autotune.cache_path())


class FakeMDEngine(FakeEngine):
    """Adds the MD pair tile: each step costs the fake clock by the current tile."""

    def __init__(self, N, P, precision="mixed", step_cost=None):
        super().__init__(N, P, precision)
        self.tile, self.steps, self.tiles_applied = 4, 0, []
        self.step_cost = step_cost or {}

    def set_pair_tile(self, lanes):
        self.tile = lanes
        self.tiles_applied.append(lanes)

    def step(self, pos, vel, nsteps=1, energies=True):
        pos += 1.0  # the tuner must hand in scratch copies
        self.steps += nsteps
        self.clock += nsteps * self.step_cost.get(self.tile, 2.0)


def test_pair_tile_picks_the_fastest_on_scratch_copies_and_caches_apart(fake_cuda):
    eng = FakeMDEngine([300, 20], [32, 16], step_cost={2: 3.0, 4: 2.0, 8: 1.5})
    fake_cuda.append(eng)
    n = 3 * sum(a * b for a, b in zip(eng.N, eng.P))
    x, v = torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64)
    res = autotune.tune_pair_tile(eng, x, v, steps=2, reps=3)
    assert res["choice"] == 8 and eng.tile == 8 and not res["cached"]
    assert set(res["timings_ms"]) == {"2", "4", "8"}
    assert res["timings_ms"]["8"] == pytest.approx(2 * 1.5)
    assert eng.steps == len(autotune.PAIR_TILES) * 2 * (1 + 3)
    assert float(x.abs().max()) == 0.0 and float(v.abs().max()) == 0.0  # the caller's tensors untouched
    assert res["key"].endswith("|md-pair-tile")
    # the exchange tuning of the same batch is a different entry
    res_x = autotune.tune(eng, x, reps=1)
    table = json.load(open(autotune.cache_path()))
    assert set(table) == {res["key"], res_x["key"]} and table[res["key"]]["choice"] == 8

    again = FakeMDEngine([300, 20], [32, 16])
    fake_cuda.append(again)
    res2 = autotune.tune_pair_tile(again, x, v)
    assert res2["cached"] and res2["choice"] == 8 and again.steps == 0 and again.tiles_applied == [8]
