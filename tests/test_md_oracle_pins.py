"""Pins of the molecular-dynamics oracle (oracle/md_oracle.c) to facts that do
not come from the oracle itself: the generator's published known answers,
moments of the normal distribution, forces as derivatives of the potential,
the time reversibility and second-order energy error of velocity Verlet,
equipartition, and the closed-form canonical energy of trapped bosons at
finite P (the paper's "Numerical Validation" comparison)."""
import os

import numpy as np
import pytest

import oracle
from oracle import harmonic
from paper_2305_18025_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
o = oracle.float64


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        assert o.philox4x32_10(w[0:4], w[4:6]) == w[6:10]


def test_thermostat_normals_moments_and_independence():
    z = o.thermostat_normals(seed=7, step=3, n=1_000_003)
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1.0) < 5e-3
    assert abs((z ** 4).mean() - 3.0) < 3e-2          # Gaussian kurtosis
    assert abs((z[:-1] * z[1:]).mean()) < 5e-3       # neighbours uncorrelated
    z2 = o.thermostat_normals(seed=7, step=4, n=1_000_003)
    assert abs((z * z2).mean()) < 5e-3               # steps uncorrelated
    z3 = o.thermostat_normals(seed=8, step=3, n=1_000_003)
    assert abs((z * z3).mean()) < 5e-3               # seeds uncorrelated
    # a prefix of a longer draw is the shorter draw (element-wise counters)
    np.testing.assert_array_equal(o.thermostat_normals(7, 3, 10), z[:10])


@pytest.mark.parametrize("omega0,pair", [(1.0, 0), (0.0, 1), (0.7, 1)])
def test_external_forces_are_minus_gradient(omega0, pair):
    rng = np.random.default_rng(11)
    pos = rng.normal(0, 0.8, (5, 3, 3))
    U, F = o.external_forces(pos, 1.3, omega0, pair, 3.0, 0.5)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 1), (4, 1, 2), (2, 0, 2)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[idx] += h
        p2[idx] -= h
        fd = -(o.external_forces(p1, 1.3, omega0, pair, 3.0, 0.5)[0] -
               o.external_forces(p2, 1.3, omega0, pair, 3.0, 0.5)[0]) / (2 * h)
        assert abs(fd - F[idx]) < 1e-7 * max(1.0, abs(F[idx]))


def test_external_trap_closed_form_and_pair_symmetry():
    rng = np.random.default_rng(3)
    pos = rng.normal(0, 1.0, (4, 6, 3))
    U, F = o.external_forces(pos, 2.0, 0.5, 0)
    assert abs(U - 0.5 * 2.0 * 0.25 * (pos ** 2).sum() / 6) < 1e-12
    # pair forces are central: they sum to zero over particles for every bead
    _, Fp = o.external_forces(pos, 2.0, 0.0, 1, 3.0, 0.5)
    assert np.abs(Fp.sum(axis=0)).max() < 1e-12
    # two particles at distance d, one bead index: U = g exp(-d^2/(2 s^2)) / P
    two = np.zeros((2, 2, 3))
    two[1, :, 0] = 0.8
    U2, _ = o.external_forces(two, 1.0, 0.0, 1, 3.0, 0.5)
    assert abs(U2 - 3.0 * np.exp(-0.64 / 0.5)) < 1e-14


def _system(N, P, seed, spread=0.6):
    rng = np.random.default_rng(seed)
    pos = inputs.trapped_positions(N, P, seed)
    vel = rng.normal(0, 0.3, pos.shape)
    return pos, vel


def test_velocity_verlet_is_time_reversible():
    N, P, beta = 4, 5, 1.5
    wP = inputs.omega_P(P, beta)
    pos, vel = _system(N, P, 1)
    p1, v1, _ = o.md_run(pos, vel, 1.0, wP, beta, 0.02, 0.0, 50, omega0=1.0, pair_type=1,
                         pair_a=3.0, pair_b=0.5)
    p2, v2, _ = o.md_run(p1, -v1, 1.0, wP, beta, 0.02, 0.0, 50, omega0=1.0, pair_type=1,
                         pair_a=3.0, pair_b=0.5)
    np.testing.assert_allclose(p2, pos, atol=1e-10)
    np.testing.assert_allclose(-v2, vel, atol=1e-10)


def test_nve_energy_error_is_second_order():
    N, P, beta = 3, 4, 1.0
    wP = inputs.omega_P(P, beta)
    pos, vel = _system(N, P, 2)
    kw = dict(omega0=1.0, pair_type=1, pair_a=3.0, pair_b=0.5)

    def H(p, v):
        VB, _ = o.fast_pimdb(p, 1.0, wP, beta)
        U, _ = o.external_forces(p, 1.0, 1.0, 1, 3.0, 0.5)
        return 0.5 * (v ** 2).sum() + VB + U

    H0 = H(pos, vel)
    errs = []
    for dt, n in [(0.02, 100), (0.01, 200)]:
        p, v, _ = o.md_run(pos, vel, 1.0, wP, beta, dt, 0.0, n, **kw)
        errs.append(abs(H(p, v) - H0))
    assert errs[0] < 1e-3 * abs(H0)
    assert 2.5 < errs[0] / errs[1] < 6.0   # ~4 for a second-order integrator


def _sample(N, P, beta, dt, nsamp, every, seed, **kw):
    wP = inputs.omega_P(P, beta)
    rng = np.random.default_rng(seed)
    pos = rng.normal(0, 0.7, (N, P, 3))
    vel = np.zeros((N, P, 3))
    pos, vel, _ = o.md_run(pos, vel, 1.0, wP, beta, dt, 1.0, 2000, seed=seed, step0=0, **kw)
    step = 2000
    out = []
    for _ in range(nsamp):
        pos, vel, en = o.md_run(pos, vel, 1.0, wP, beta, dt, 1.0, every, seed=seed, step0=step, **kw)
        step += every
        out.append(en.copy())
    return np.array(out)


def test_equipartition_and_harmonic_closed_form():
    """<KE> = 3NP/(2 beta) and <E_prim> = -d ln Z/d beta of N bosons in a trap
    at finite P (closed form), both within four block standard errors."""
    N, P, beta = 2, 4, 2.0
    en = _sample(N, P, beta, 0.1, 40000, 10, seed=8, omega0=1.0)
    for col, exact in [(2, 1.5 * N * P / beta), (3, harmonic.mean_energy(N, P, beta, 1.0))]:
        b = en[:, col].reshape(100, -1).mean(axis=1)
        err = b.std(ddof=1) / np.sqrt(len(b))
        assert abs(b.mean() - exact) < 4 * err + 1e-3 * abs(exact), (col, b.mean(), exact, err)


def test_noise_offset_takes_the_counters_of_the_packed_position():
    """A replica at element offset e0 of a packed batch draws, for its element
    i, the normal of element e0 + i of one long system: the same Philox stream
    cut at e0 (offsets that are not a multiple of 4 included)."""
    o = oracle.float64
    N, P = 3, 5  # 45 elements
    pos = np.random.default_rng(4).normal(0, 1, (N, P, 3))
    c1 = np.exp(-50.0 * 1e-6)
    for e0 in (0, 6, 45):
        # dt -> 0, no forces to speak of: after one step v = c2 z, so v / c2 = z
        _, v, _ = o.md_run(pos, np.zeros((N, P, 3)), 1.0, 1e-9, 1.0, 1e-6, 50.0, 1, seed=9, kT=1.0, elem0=e0)
        z = v.reshape(-1) / np.sqrt(1 - c1 * c1)
        # the first e0 + 45 normals of one long system (elements of 3 particles of
        # P = 5 per 45; the long system has (e0 + 45) / 15 particles of P = 5)
        M = -(-(e0 + 45) // 15)
        _, vl, _ = o.md_run(np.zeros((M, 5, 3)), np.zeros((M, 5, 3)), 1.0, 1e-9, 1.0, 1e-6, 50.0, 1, seed=9, kT=1.0)
        zl = vl.reshape(-1) / np.sqrt(1 - c1 * c1)
        np.testing.assert_allclose(z, zl[e0:e0 + 45], rtol=0, atol=1e-6)
