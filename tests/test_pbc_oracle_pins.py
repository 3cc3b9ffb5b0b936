"""Pins of the oracle's periodic box (minimum-image springs) and Lennard-Jones
pair potential, used for bulk liquid helium, to facts that do not come from
the oracle itself: periodicity (moving any bead by a lattice vector changes
nothing), equality with open boundaries when no spring crosses the box, the
closed-form Lennard-Jones pair energy and its cutoff, forces as minus the
finite-difference gradient, Algorithm 1 = Algorithm 2 in a box, and the
time reversibility and second-order energy error of the MD step in a box."""
import numpy as np
import pytest

import oracle
from paper_2305_18025_gb300 import inputs

o = oracle.float64


def _wrapped_liquid(N, P, L, seed, spread=0.15):
    """Ring polymers scattered over the whole box, coordinates wrapped into
    [0, L), so that many springs cross the boundary."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, L, (N, 1, 3))
    pos = centres + rng.normal(0, spread, (N, P, 3))
    return np.mod(pos, L)


def test_open_boundaries_equal_a_large_box():
    pos = inputs.trapped_positions(12, 6, seed=3)
    for fn in (o.fast_pimdb, o.original_pimdb):
        V0, F0 = fn(pos, 1.0, 2.0, 1.1)
        V1, F1 = fn(pos, 1.0, 2.0, 1.1, box=1000.0)
        assert abs(V1 - V0) <= 1e-13 * abs(V0)
        np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-12 * np.abs(F0).max())


@pytest.mark.parametrize("N,P", [(7, 4), (20, 3)])
def test_lattice_translations_of_single_beads_change_nothing(N, P):
    L = 3.0
    pos = _wrapped_liquid(N, P, L, seed=N)
    V0, F0, V, W, M = o.fast_pimdb(pos, 1.0, 1.7, 0.8, full=True, box=L)
    rng = np.random.default_rng(1)
    shifted = pos + L * rng.integers(-2, 3, pos.shape)
    V1, F1, V_, W_, M_ = o.fast_pimdb(shifted, 1.0, 1.7, 0.8, full=True, box=L)
    assert abs(V1 - V0) <= 1e-12 * abs(V0)
    np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-11 * np.abs(F0).max())
    np.testing.assert_allclose(M_, M, rtol=0, atol=1e-12)
    # and the springs really do cross the box: the open-boundary value differs
    Vopen, _ = o.fast_pimdb(pos, 1.0, 1.7, 0.8)
    assert abs(Vopen - V0) > 1.0


def test_algorithm_1_equals_algorithm_2_in_a_box():
    L = 2.5
    pos = _wrapped_liquid(9, 5, L, seed=4)
    V1, F1 = o.fast_pimdb(pos, 1.0, 1.5, 1.2, box=L)
    V2, F2 = o.original_pimdb(pos, 1.0, 1.5, 1.2, box=L)
    assert abs(V1 - V2) <= 1e-11 * abs(V2)
    np.testing.assert_allclose(F1, F2, rtol=0, atol=1e-10 * np.abs(F2).max())


def test_box_forces_are_minus_gradient():
    L = 3.0
    pos = _wrapped_liquid(8, 4, L, seed=5)
    _, F = o.fast_pimdb(pos, 1.0, 1.6, 1.0, box=L)
    h = 1e-6
    for idx in inputs.random_coordinates(pos.shape, 16, seed=6):
        flat = pos.reshape(-1)
        a, b = flat.copy(), flat.copy()
        a[idx] += h
        b[idx] -= h
        Va, _ = o.fast_pimdb(a.reshape(pos.shape), 1.0, 1.6, 1.0, box=L)
        Vb, _ = o.fast_pimdb(b.reshape(pos.shape), 1.0, 1.6, 1.0, box=L)
        fd = -(Va - Vb) / (2 * h)
        assert abs(fd - F.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_lennard_jones_pair_closed_form_cutoff_and_minimum_image():
    eps, sig, rc, L = 10.22, 2.556, 2.5 * 2.556, 20.0
    shift = 4 * eps * ((sig / rc) ** 12 - (sig / rc) ** 6)
    for r in (2.3, 2.9, 4.0, 6.0):
        two = np.zeros((2, 3, 3))
        two[1, :, 0] = r
        U, F = o.external_forces(two, 4.0, 0.0, 2, eps, sig, rc, L)
        assert abs(U - (4 * eps * ((sig / r) ** 12 - (sig / r) ** 6) - shift)) <= 1e-12 * abs(U) + 1e-12
        fr = 24 * eps * (2 * (sig / r) ** 12 - (sig / r) ** 6) / r / 3  # 1/P, P = 3
        assert abs(F[0, 0, 0] + fr) <= 1e-12 * abs(fr) + 1e-12 and abs(F[1, 0, 0] - fr) <= 1e-12 * abs(fr) + 1e-12
        # the same pair seen across the boundary
        wrap = two.copy()
        wrap[1, :, 0] = L - r
        wrap[0, :, 0] = 0.0
        Uw, Fw = o.external_forces(wrap, 4.0, 0.0, 2, eps, sig, rc, L)
        assert abs(Uw - U) <= 1e-12 * abs(U) + 1e-12
        np.testing.assert_allclose(Fw[:, :, 0], -F[:, :, 0], rtol=1e-12, atol=1e-12)
    far = np.zeros((2, 2, 3))
    far[1, :, 1] = rc * 1.01
    U, F = o.external_forces(far, 4.0, 0.0, 2, eps, sig, rc, L)
    assert U == 0.0 and np.all(F == 0.0)


def test_lennard_jones_forces_are_minus_gradient_and_central():
    L = 12.0
    pos = inputs.fcc_positions(2, 3, L, seed=2, jitter=0.1)
    args = (4.0, 0.0, 2, 10.22, 2.556, 2.5 * 2.556, L)
    U, F = o.external_forces(pos, *args)
    assert np.abs(F.sum(axis=0)).max() <= 1e-10 * np.abs(F).max()
    h = 1e-6
    for idx in inputs.random_coordinates(pos.shape, 12, seed=3):
        flat = pos.reshape(-1)
        a, b = flat.copy(), flat.copy()
        a[idx] += h
        b[idx] -= h
        fd = -(o.external_forces(a.reshape(pos.shape), *args)[0] -
               o.external_forces(b.reshape(pos.shape), *args)[0]) / (2 * h)
        assert abs(fd - F.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_md_in_a_box_is_reversible_and_second_order():
    L = 12.0
    N, P, beta = 32, 4, 1.0 / 1.5
    hbar = 6.96
    wP = np.sqrt(P) / (beta * hbar)
    pos = inputs.fcc_positions(2, P, L, seed=7, jitter=0.1)
    vel = np.random.default_rng(8).normal(0, 0.2, pos.shape)
    kw = dict(pair_type=2, pair_a=10.22, pair_b=2.556, pair_rc=2.5 * 2.556, box=L)
    p1, v1, _ = o.md_run(pos, vel, 4.0, wP, beta, 0.002, 0.0, 40, **kw)
    p2, v2, _ = o.md_run(p1, -v1, 4.0, wP, beta, 0.002, 0.0, 40, **kw)
    np.testing.assert_allclose(p2, pos, atol=1e-9)

    # second-order energy error of the springs in the box (the truncated
    # Lennard-Jones force jumps at rc, which makes its error first order)
    spring_pos = _wrapped_liquid(12, 5, 3.0, seed=9, spread=0.3)
    spring_vel = np.random.default_rng(10).normal(0, 0.3, spring_pos.shape)

    def H(p, v):
        VB, _ = o.fast_pimdb(p, 1.0, 1.2, 1.0, box=3.0)
        return 0.5 * (v ** 2).sum() + VB

    H0 = H(spring_pos, spring_vel)
    errs = []
    for dt in (0.02, 0.01):
        p, v, m = spring_pos, spring_vel, 0.0
        for _ in range(10):
            p, v, _ = o.md_run(p, v, 1.0, 1.2, 1.0, dt, 0.0, int(round(0.1 / dt)), box=3.0)
            m = max(m, abs(H(p, v) - H0))
        errs.append(m)
    assert 3.0 < errs[0] / errs[1] < 5.5
