"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics -- never against the oracle itself.

Each test names the passage it checks.  Together they are chosen so that a
dropped term, a wrong sign or index, or a transposed operand anywhere in the
oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute, harmonic
from paper_2305_18025_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def params(P, beta, m=1.0):
    return m, inputs.omega_P(P, beta), beta


# ---------------------------------------------------------------- cycle energies

@pytest.mark.parametrize("N,P", [(1, 2), (2, 3), (5, 2), (7, 8), (12, 5)])
def test_cycle_energy_recurrence_matches_direct_sum(N, P):
    """Eq. e-recurrence-step/base (Algorithm 1) reproduces Eq. Ek's double sum."""
    pos = inputs.trapped_positions(N, P, seed=11 + N)
    m, w, _ = params(P, 1.3)
    Er = oracle.cycle_energies(pos, m, w)
    Ed = oracle.cycle_energies(pos, m, w, direct=True)
    iu = np.triu_indices(N)
    np.testing.assert_allclose(Er[iu], Ed[iu], rtol=1e-12, atol=1e-12)


def test_cycle_energy_equals_ring_of_consecutive_particles():
    """E^{[u,v]} is the Eq. eperm energy of the ring u -> ... -> v -> u, evaluated
    bead by bead with np.roll (independent of both oracle routines)."""
    N, P = 6, 4
    pos = inputs.trapped_positions(N, P, seed=5)
    m, w, _ = params(P, 0.7)
    E = oracle.cycle_energies(pos, m, w)
    for u in range(1, N + 1):
        for v in range(u, N + 1):
            ref = brute.consecutive_cycle_energy(pos, u, v, m, w)
            assert E[u - 1, v - 1] == pytest.approx(ref, rel=1e-12, abs=1e-12)


# ------------------------------------------------------------------ special cases

def textbook_ring(pos_one, m, w):
    """Ordinary ring polymer of one particle: energy and spring forces."""
    k = m * w * w
    d = pos_one - np.roll(pos_one, -1, axis=0)
    E = 0.5 * k * float(np.sum(d * d))
    F = -k * (2 * pos_one - np.roll(pos_one, -1, axis=0) - np.roll(pos_one, 1, axis=0))
    return E, F


@pytest.mark.parametrize("P", [2, 3, 16])
def test_single_particle_is_ordinary_ring_polymer(P):
    """N = 1: V^{[1,1]} = E^{[1,1]} and the forces are ordinary PIMD ring forces."""
    pos = inputs.trapped_positions(1, P, seed=3)
    m, w, beta = params(P, 2.0)
    VB, F = oracle.fast_pimdb(pos, m, w, beta)
    E, Fr = textbook_ring(pos[0], m, w)
    assert VB == pytest.approx(E, rel=1e-13)
    np.testing.assert_allclose(F[0], Fr, rtol=1e-12, atol=1e-12)


def test_two_particles_closed_form():
    """N = 2: exp(-beta V) = (1/2)(exp(-beta(E^{[1,1]} + E^{[2,2]})) + exp(-beta E^{[1,2]}))
    -- the two permutations of Eq. int-of-sum-all-permutations, both their own
    representatives.  Ring energies from np.roll over the wired beads."""
    P = 5
    pos = inputs.trapped_positions(2, P, seed=21)
    m, w, beta = params(P, 1.1)
    e1, _ = textbook_ring(pos[0], m, w)
    e2, _ = textbook_ring(pos[1], m, w)
    e12, _ = textbook_ring(np.concatenate([pos[0], pos[1]]), m, w)
    a, b = -beta * (e1 + e2), -beta * e12
    mx = max(a, b)
    ref = -(mx + math.log(0.5 * (math.exp(a - mx) + math.exp(b - mx)))) / beta
    VB, _ = oracle.fast_pimdb(pos, m, w, beta)
    assert VB == pytest.approx(ref, rel=1e-13)


def _parse_cycles(s):
    """'(12)(3)' -> permutation tuple sigma(1..N)."""
    cycles = [c for c in s.replace(")", ") ").split() if c]
    n = sum(len(c) - 2 for c in cycles)
    sigma = [0] * n
    for c in cycles:
        el = [int(ch) for ch in c.strip("()")]
        for i, e in enumerate(el):
            sigma[e - 1] = el[(i + 1) % len(el)]
    return tuple(sigma)


def _golden_n3():
    rows, maps, prs = [], [], []
    with open(os.path.join(GOLDEN, "n3_representative_weights.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "MAP":
                maps.append((parts[1], parts[2]))
            elif parts[0] == "PR":
                prs.append((int(parts[1]), int(parts[2]), parts[3:]))
            else:
                rows.append((parts[0], tuple(int(x) for x in parts[1:4]), Fraction(parts[4])))
    return rows, maps, prs


def test_n3_representative_map_matches_paper():
    """G of Definition representative-permutation reproduces the paper's N = 3 map."""
    _, maps, _ = _golden_n3()
    for s, g in maps:
        assert brute.representative(_parse_cycles(s)) == _parse_cycles(g)


def test_n3_worked_expansion():
    """Eq. vall-3-sum-permutations: weights 1/6, 1/3, 1/6, 1/3 over the four
    representatives give V^{[1,3]} (golden fixture)."""
    rows, _, _ = _golden_n3()
    assert sum(w for *_, w in rows) == 1
    P = 4
    pos = inputs.clustered_chain_positions(3, P, seed=8)
    m, w, beta = params(P, 1.5)
    terms = [(float(wt), brute.ring_energy(pos, sig, m, w)) for _, sig, wt in rows]
    emin = min(e for _, e in terms)
    ref = emin - math.log(sum(wt * math.exp(-beta * (e - emin)) for wt, e in terms)) / beta
    VB, _ = oracle.fast_pimdb(pos, m, w, beta)
    assert VB == pytest.approx(ref, rel=1e-13)


def test_n3_connection_probabilities_of_particle_one():
    """Section "Force on exterior beads", N = 3: Pr[1->1], Pr[1->2] as the
    weighted sums of the fixture, Pr[1->3] = 0."""
    rows, _, prs = _golden_n3()
    P = 3
    pos = inputs.clustered_chain_positions(3, P, seed=9)
    m, w, beta = params(P, 0.8)
    by_name = {name: brute.ring_energy(pos, sig, m, w) for name, sig, _ in rows}
    Z = sum(float(wt) * math.exp(-beta * by_name[name]) for name, _, wt in rows)
    _, _, _, _, M = oracle.fast_pimdb(pos, m, w, beta, full=True)
    for l, lp, terms in prs:
        val = 0.0
        for t in terms:
            name, wt = t.split(":")
            val += float(Fraction(wt)) * math.exp(-beta * by_name[name])
        assert M[l - 1, lp - 1] == pytest.approx(val / Z, rel=1e-12, abs=1e-15)
    assert M[0, 2] == 0.0


# ------------------------------------------------------------------- brute force

@pytest.mark.parametrize("N,P,beta,gen", [
    (1, 3, 1.0, "trapped"), (2, 4, 0.6, "trapped"), (3, 2, 2.0, "clustered"),
    (4, 3, 1.0, "clustered"), (5, 2, 0.9, "trapped"), (6, 3, 1.7, "clustered"),
])
def test_algorithm1_matches_sum_over_all_permutations(N, P, beta, gen):
    """Algorithm 1 (V, forces, connection probabilities) equals Definition
    forward-potential / Lemma expected-force evaluated over all N! permutations."""
    pos = (inputs.trapped_positions(N, P, seed=100 + N) if gen == "trapped"
           else inputs.clustered_chain_positions(N, P, seed=200 + N))
    m, w, _ = params(P, beta)
    Vb, Fb, Mb = brute.potential_by_permutations(pos, m, w, beta)
    VB, F, V, W, M = oracle.fast_pimdb(pos, m, w, beta, full=True)
    assert VB == pytest.approx(Vb, rel=1e-12)
    np.testing.assert_allclose(F, Fb, rtol=1e-10, atol=1e-10 * np.abs(Fb).max())
    np.testing.assert_allclose(M, Mb, rtol=1e-10, atol=1e-13)


def test_composition_weights_count_permutations():
    """Appendix "Some Combinatorics": 2^(N-1) representatives, and the cut
    v_1 < ... < v_m = N collects N!/prod(v_i) of the N! permutations."""
    for N in range(1, 7):
        counts = brute.representative_counts(N)
        assert len(counts) == 2 ** (N - 1)
        for ends, c in counts.items():
            assert c * math.prod(ends) == math.factorial(N)


@pytest.mark.parametrize("N", [7, 10, 12])
def test_algorithm1_matches_sum_over_representatives(N):
    """Eq. vall-sum-representatives grouped by representative (2^(N-1) terms)."""
    P = 3
    pos = inputs.clustered_chain_positions(N, P, seed=300 + N)
    m, w, beta = params(P, 1.2)
    ref = brute.potential_by_compositions(pos, m, w, beta)
    VB, _ = oracle.fast_pimdb(pos, m, w, beta)
    assert VB == pytest.approx(ref, rel=1e-12)


# -------------------------------------------------------------- Algorithm 2 / defs

@pytest.mark.parametrize("N,P,gen", [(8, 4, "clustered"), (16, 8, "trapped"), (24, 3, "clustered")])
def test_algorithm1_matches_original_algorithm2(N, P, gen):
    """Introduction: the new algorithm gives the same potential and forces as the
    original O(P N^3) one (Algorithm 2, per-bead differentiated recursion)."""
    pos = (inputs.trapped_positions(N, P, seed=400 + N) if gen == "trapped"
           else inputs.clustered_chain_positions(N, P, seed=500 + N))
    m, w, beta = params(P, 1.0)
    V1, F1 = oracle.fast_pimdb(pos, m, w, beta)
    V2, F2 = oracle.original_pimdb(pos, m, w, beta)
    assert V1 == pytest.approx(V2, rel=1e-12)
    np.testing.assert_allclose(F1, F2, rtol=1e-9, atol=1e-10 * np.abs(F2).max())


@pytest.mark.parametrize("N", [1, 2, 9, 40])
def test_backward_recursion_matches_definition(N):
    """Theorem backward-recurrence vs Definition backward-potential, and
    V^{[1,N]} from the backward side equals the forward one (remark after the
    definition)."""
    P = 4
    pos = inputs.clustered_chain_positions(N, P, seed=600 + N)
    m, w, beta = params(P, 0.9)
    E = oracle.cycle_energies(pos, m, w)
    W = oracle.backward_potentials(E, beta)
    Wd = oracle.backward_potentials_definition(E, beta)
    V = oracle.forward_potentials(E, beta)
    np.testing.assert_allclose(W, Wd, rtol=1e-12, atol=1e-12)
    assert W[0] == pytest.approx(V[N], rel=1e-12)
    assert W[N] == 0.0


@pytest.mark.parametrize("gen", ["trapped", "clustered"])
def test_shift_choice_does_not_change_potentials(gen):
    """Numerical Stability: every choice of the shift is valid -- Eq. full-elong
    and Eq. original-elong give the same V^{[1,v]} and V^{[u,N]}."""
    N, P = 30, 8
    pos = (inputs.trapped_positions(N, P, seed=7) if gen == "trapped"
           else inputs.clustered_chain_positions(N, P, seed=7))
    m, w, beta = params(P, 1.0)
    E = oracle.cycle_energies(pos, m, w)
    for fn in (oracle.forward_potentials, oracle.backward_potentials):
        a = fn(E, beta, oracle.SHIFT_MIN_ALL)
        b = fn(E, beta, oracle.SHIFT_TWO_TERM)
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-11)


# -------------------------------------------------------------------- invariants

@pytest.mark.parametrize("N,gen", [(5, "trapped"), (64, "trapped"), (64, "clustered"), (200, "clustered")])
def test_connection_matrix_invariants(N, gen):
    """Theorem backward-recurrence proof: each particle's bead 1 has exactly one
    predecessor (column sums 1); each bead P one successor (row sums 1);
    Lemma zero-connection-probability: Pr[l->l'] = 0 for l' > l + 1."""
    P = 8
    pos = (inputs.trapped_positions(N, P, seed=N) if gen == "trapped"
           else inputs.clustered_chain_positions(N, P, seed=N))
    m, w, beta = params(P, 1.0)
    _, _, _, _, M = oracle.fast_pimdb(pos, m, w, beta, full=True)
    np.testing.assert_allclose(M.sum(axis=0), 1.0, atol=1e-11)
    np.testing.assert_allclose(M.sum(axis=1), 1.0, atol=1e-11)
    assert np.all(np.triu(M, 2) == 0.0)
    assert M.min() > -1e-12


@pytest.mark.parametrize("N", [1, 4, 33])
def test_coincident_beads_closed_form(N):
    """All beads at one point: every E^{[u,v]} = 0, so V^{[1,v]} = 0,
    V^{[u,N]} = ln(u)/beta (exp(-beta V^{[u,N]}) = sum_{l=u}^{N-1} 1/(l(l+1)) + 1/N
    = 1/u), Pr[l->l+1] = l/(l+1), Pr[l->u<=l] = 1/(l(l+1)) for l < N and 1/N for
    l = N (Eq. direct-link and Eq. close-cycle), forces zero."""
    P = 6
    pos = inputs.coincident_positions(N, P)
    m, w, beta = params(P, 1.7)
    VB, F, V, W, M = oracle.fast_pimdb(pos, m, w, beta, full=True)
    assert np.all(V == 0.0)
    np.testing.assert_allclose(W[:N], np.log(np.arange(1, N + 1)) / beta, rtol=1e-14, atol=1e-15)
    ref = np.zeros((N, N))
    for l in range(1, N + 1):
        for u in range(1, l + 1):
            ref[l - 1, u - 1] = 1.0 / (l * (l + 1)) if l < N else 1.0 / N
        if l < N:
            ref[l - 1, l] = l / (l + 1)
    np.testing.assert_allclose(M, ref, rtol=1e-13, atol=1e-16)
    assert np.all(F == 0.0)


def test_well_separated_particles_do_not_exchange():
    """Particles far apart: only the identity permutation survives, so
    V^{[1,N]} = sum_l E^{[l,l]} + ln(N!)/beta, Pr = identity on the diagonal and
    the forces are N independent ring-polymer forces."""
    N, P = 7, 5
    pos = inputs.separated_positions(N, P, seed=1)
    m, w, beta = params(P, 1.0)
    VB, F, V, W, M = oracle.fast_pimdb(pos, m, w, beta, full=True)
    rings = [textbook_ring(pos[l], m, w) for l in range(N)]
    ref = sum(e for e, _ in rings) + math.log(math.factorial(N)) / beta
    assert VB == pytest.approx(ref, rel=1e-13)
    np.testing.assert_allclose(M, np.eye(N), atol=1e-14)
    np.testing.assert_allclose(F, np.stack([f for _, f in rings]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N,gen", [(12, "clustered"), (64, "trapped")])
def test_forces_have_no_net_force_or_torque(N, gen):
    """Springs are central pair forces: sum of forces and of torques vanish, and
    V is invariant under a rigid translation and rotation of all beads."""
    P = 8
    pos = (inputs.trapped_positions(N, P, seed=N) if gen == "trapped"
           else inputs.clustered_chain_positions(N, P, seed=N))
    m, w, beta = params(P, 1.0)
    VB, F = oracle.fast_pimdb(pos, m, w, beta)
    scale = np.abs(F).max()
    np.testing.assert_allclose(F.sum(axis=(0, 1)), 0.0, atol=1e-11 * scale * N * P)
    torque = np.cross(pos, F).sum(axis=(0, 1))
    np.testing.assert_allclose(torque, 0.0, atol=1e-11 * scale * N * P * np.abs(pos).max())
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    moved = pos @ R.T + np.array([3.0, -1.0, 0.5])
    V2, _ = oracle.fast_pimdb(moved, m, w, beta)
    assert V2 == pytest.approx(VB, rel=1e-11)


def test_forces_are_minus_gradient_by_central_differences():
    """F = -grad V^{[1,N]}: central differences (h = 1e-5) on 32 seeded coordinates
    of the N = 64, P = 32 trapped system."""
    N, P = 64, 32
    pos = inputs.trapped_positions(N, P, seed=2)
    m, w, beta = params(P, 1.0)
    _, F = oracle.fast_pimdb(pos, m, w, beta)
    h = 1e-5
    flat = pos.reshape(-1)
    for idx in inputs.random_coordinates(pos.shape, 32, seed=4):
        p1, p2 = flat.copy(), flat.copy()
        p1[idx] += h
        p2[idx] -= h
        v1, _ = oracle.fast_pimdb(p1.reshape(pos.shape), m, w, beta)
        v2, _ = oracle.fast_pimdb(p2.reshape(pos.shape), m, w, beta)
        fd = -(v1 - v2) / (2 * h)
        assert F.reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(F).max())


def test_expected_spring_energy_matches_permutation_average():
    """The expectation of E^{G[sigma]} under Eq. representative-distribution
    equals the interior springs plus the connection-probability-weighted
    exterior springs."""
    N, P = 5, 3
    pos = inputs.clustered_chain_positions(N, P, seed=12)
    m, w, beta = params(P, 1.0)
    import itertools
    reps = [brute.representative(s) for s in itertools.permutations(range(1, N + 1))]
    Es = np.array([brute.ring_energy(pos, g, m, w) for g in reps])
    wts = np.exp(-beta * (Es - Es.min()))
    ref = float(np.sum(wts * Es) / np.sum(wts))
    _, _, _, _, M = oracle.fast_pimdb(pos, m, w, beta, full=True)
    assert oracle.expected_spring_energy(pos, M, m, w) == pytest.approx(ref, rel=1e-12)


def test_oracle_rejects_invalid_arguments():
    pos = inputs.trapped_positions(3, 1, seed=0)
    with pytest.raises(ValueError):
        oracle.fast_pimdb(pos, 1.0, 1.0, 1.0)            # P = 1
    pos = inputs.trapped_positions(3, 4, seed=0)
    with pytest.raises(ValueError):
        oracle.fast_pimdb(pos, 1.0, 1.0, -1.0)           # beta <= 0


# ------------------------------------------------------------ harmonic closed form

def test_harmonic_single_particle_limits():
    """N = 1: at P -> infinity the textbook (3/2) w0 coth(beta w0 / 2); at P = 1 the
    classical 3/beta."""
    for beta in (0.5, 1.0, 4.0):
        assert harmonic.mean_energy(1, 200000, beta) == pytest.approx(
            1.5 / math.tanh(beta / 2), rel=1e-8)
        assert harmonic.mean_energy(1, 1, beta) == pytest.approx(3.0 / beta, rel=1e-12)


def test_harmonic_recursion_matches_cycle_index():
    """Z_2 = (z_1^2 + z_2)/2 and Z_3 = z_1^3/6 + z_1 z_2/2 + z_3/3 (sum over cycle
    types of S_3), and the energy is -d ln Z / d beta by central differences."""
    P, beta = 12, 1.3
    z = [None] + [harmonic.single_ring_partition(k, P, beta) for k in (1, 2, 3)]
    assert harmonic.partition_function(2, P, beta) == pytest.approx((z[1] ** 2 + z[2]) / 2, rel=1e-13)
    assert harmonic.partition_function(3, P, beta) == pytest.approx(
        z[1] ** 3 / 6 + z[1] * z[2] / 2 + z[3] / 3, rel=1e-13)
    h = 1e-5
    for N in (1, 3, 6):
        fd = -(math.log(harmonic.partition_function(N, P, beta + h))
               - math.log(harmonic.partition_function(N, P, beta - h))) / (2 * h)
        assert harmonic.mean_energy(N, P, beta) == pytest.approx(fd, rel=1e-7)


def test_harmonic_trap_energy_limits():
    """<U-bar> at P -> infinity is half the energy (virial theorem of the
    harmonic Hamiltonian, <T> = <U>, which holds for bosons as for any
    eigenstate mixture); at P = 1 (classical) it is dim N / (2 beta) for N = 1;
    and it is -(w0/(2 beta)) d ln Z/d w0 by central differences of the
    unscaled partition function."""
    for N in (1, 8):
        for beta in (0.5, 2.0):
            assert harmonic.mean_trap_energy(N, 200000, beta) == pytest.approx(
                0.5 * harmonic.mean_energy(N, 200000, beta), rel=1e-7)
    assert harmonic.mean_trap_energy(1, 1, 1.7) == pytest.approx(1.5 / 1.7, rel=1e-12)
    P, beta, w0, h = 10, 1.3, 0.8, 1e-6
    for N in (1, 4):
        fd = (math.log(harmonic.partition_function(N, P, beta, w0 + h))
              - math.log(harmonic.partition_function(N, P, beta, w0 - h))) / (2 * h)
        assert harmonic.mean_trap_energy(N, P, beta, w0) == pytest.approx(-(w0 / (2 * beta)) * fd, rel=1e-7)


def test_harmonic_ground_state_limit():
    """beta -> infinity at large P: all bosons in the ground state, 1.5 N w0."""
    assert harmonic.mean_energy(16, 100000, 60.0) == pytest.approx(1.5 * 16, rel=1e-6)
