"""The seeded synthetic inputs follow their stated recipes: shapes, dtype and
layout, determinism per seed, the distributions of centres and bead offsets,
the lattice and density of the liquid-helium start, and the ranges of the
replica batch."""
import math

import numpy as np

from paper_2305_18025_gb300 import inputs


def test_trapped_recipe_and_determinism():
    N, P = 4000, 16
    a = inputs.trapped_positions(N, P, 3)
    assert a.shape == (N, P, 3) and a.dtype == np.float64 and a.flags.c_contiguous
    assert np.array_equal(a, inputs.trapped_positions(N, P, 3))
    assert not np.array_equal(a, inputs.trapped_positions(N, P, 4))
    centres = a.mean(axis=1)                      # offsets average out over P beads
    offsets = a - centres[:, None, :]
    # centres N(0, 1) per axis (the bead mean adds 0.1/sqrt(P) of spread)
    assert abs(centres.std() - math.sqrt(1.0 + 0.01 / P)) < 0.03
    assert abs(centres.mean()) < 0.05
    # offsets N(0, 0.1) per axis, measured about the bead mean (P-1 degrees of freedom)
    assert abs(offsets.std() * math.sqrt(P / (P - 1)) - 0.1) < 0.002


def test_coincident_separated_and_clustered():
    c = inputs.coincident_positions(5, 3)
    assert np.all(c == np.array([0.25, -0.5, 1.0]))
    s = inputs.separated_positions(10, 4, 1)
    centres = s.mean(axis=1)
    assert np.allclose(np.diff(centres[:, 0]), 100.0, atol=0.5)
    assert np.abs(centres[:, 1:]).max() < 0.5
    k = inputs.clustered_chain_positions(2000, 8, 2)
    steps = np.diff(k.mean(axis=1), axis=0)       # walk steps N(0, 0.05) plus bead-mean noise
    assert abs(steps.std() - math.sqrt(0.05 ** 2 + 2 * 0.01 / 8)) < 0.005


def test_fcc_helium_start_fills_the_box_at_the_density():
    cells, P, rho = 4, 8, 0.0218
    N = 4 * cells ** 3
    L = (N / rho) ** (1.0 / 3.0)
    x = inputs.fcc_positions(cells, P, L, 5, jitter=0.0)
    assert x.shape == (N, P, 3)
    sites = x[:, 0, :]
    assert np.all(x == sites[:, None, :])                  # no jitter: every bead on its site
    assert sites.min() > 0.0 and sites.max() < L
    assert abs(N / L ** 3 - rho) < 1e-12
    diff = sites[:, None, :] - sites[None, :, :]
    diff -= L * np.round(diff / L)
    nn = np.sort(np.linalg.norm(diff, axis=-1), axis=1)
    a = L / cells
    assert np.allclose(nn[:, 1:13], a / math.sqrt(2.0))    # 12 nearest neighbours of FCC
    assert np.all(nn[:, 13] > a / math.sqrt(2.0) + 1e-9)
    j = inputs.fcc_positions(cells, P, L, 5)
    assert 0.04 < (j - x).std() < 0.06                     # the default jitter N(0, 0.05)


def test_replica_batch_ranges():
    reps = inputs.batched_replicas(256, seed=11)
    assert len(reps) == 256
    assert all(16 <= r.N <= 512 for r in reps)
    assert {r.P for r in reps} <= {16, 32, 64} and len({r.P for r in reps}) == 3
    assert all(0.5 <= r.beta <= 4.0 for r in reps)
    assert all(r.positions.shape == (r.N, r.P, 3) for r in reps)
    again = inputs.batched_replicas(256, seed=11)
    assert all(np.array_equal(a.positions, b.positions) and a.beta == b.beta for a, b in zip(reps, again))


def test_random_coordinates_are_distinct_and_in_range():
    idx = inputs.random_coordinates((64, 32, 3), 32, seed=4)
    assert len(set(idx.tolist())) == 32
    assert idx.min() >= 0 and idx.max() < 64 * 32 * 3


def test_omega_P():
    assert inputs.omega_P(32, 1.0) == math.sqrt(32.0)
    assert inputs.omega_P(64, 2.0, hbar=0.5) == math.sqrt(64.0)
