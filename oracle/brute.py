"""Brute-force definitions of the exchange potential (test infrastructure only).

These evaluate the paper's *definitions* directly, with none of Algorithm 1's
recursions, so they pin the recursive oracle from outside:

* ``representative`` -- the map G of Definition representative-permutation
  (Methods, "Definition of G[sigma]"): write sigma in canonical cycle notation
  (appendix "Cycle Notation of Permutations"), order the cycles by their largest
  element, then relabel the elements 1..N consecutively keeping cycle lengths
  and order.
* ``ring_energy`` / ``ring_gradient`` -- Eq. eperm for an arbitrary permutation.
* ``potential_by_permutations`` -- Definition forward-potential,
  exp(-beta V^{[1,N]}) = (1/N!) sum_sigma exp(-beta E^{G[sigma]}), with the forces
  of Lemma expected-force and the connection probabilities summed over
  permutations as in Eq. force-on-1/P-sum-neighbors.
* ``potential_by_compositions`` -- the same sum grouped by the 2^(N-1)
  representative permutations (appendix "Some Combinatorics of Permutations"):
  a representative is a cut of [1, N] into consecutive cycles.

Pure Python/numpy; exponential cost, small N only.
"""
import itertools
import math

import numpy as np


def canonical_cycles(sigma):
    """Cycle notation of sigma (tuple, sigma[l-1] = sigma(l), 1-based values):
    start each cycle at the smallest element not yet used and follow sigma."""
    N = len(sigma)
    seen = [False] * (N + 1)
    cycles = []
    for start in range(1, N + 1):
        if seen[start]:
            continue
        c = [start]
        seen[start] = True
        x = sigma[start - 1]
        while x != start:
            c.append(x)
            seen[x] = True
            x = sigma[x - 1]
        cycles.append(c)
    return cycles


def representative(sigma):
    """G[sigma] as a tuple (G[l-1] = G[sigma](l))."""
    N = len(sigma)
    cycles = sorted(canonical_cycles(sigma), key=max)
    G = [0] * N
    first = 1
    for c in cycles:
        L = len(c)
        block = list(range(first, first + L))   # c' = (first, ..., first + L - 1)
        for i, e in enumerate(block):
            G[e - 1] = block[(i + 1) % L]
        first += L
    return tuple(G)


def ring_energy(pos, sigma, m, omega_P):
    """Eq. eperm: (1/2) m w_P^2 sum_l sum_{j=1}^{P} (r_l^j - r_l^{j+1})^2 with
    r_l^{P+1} = r_{sigma(l)}^1."""
    pos = np.asarray(pos, dtype=np.float64)
    N, P, _ = pos.shape
    total = 0.0
    for l in range(1, N + 1):
        for j in range(1, P + 1):
            nxt = pos[l - 1, j] if j < P else pos[sigma[l - 1] - 1, 0]
            d = pos[l - 1, j - 1] - nxt
            total += float(d @ d)
    return 0.5 * m * omega_P ** 2 * total


def ring_gradient(pos, sigma, m, omega_P):
    """Gradient of Eq. eperm with respect to every bead: each bead is pulled by
    its two neighbours in the ring that sigma wires up."""
    pos = np.asarray(pos, dtype=np.float64)
    N, P, _ = pos.shape
    k = m * omega_P ** 2
    inv = [0] * N
    for l in range(1, N + 1):
        inv[sigma[l - 1] - 1] = l
    g = np.zeros_like(pos)
    for l in range(1, N + 1):
        for j in range(1, P + 1):
            nxt = pos[l - 1, j] if j < P else pos[sigma[l - 1] - 1, 0]
            prv = pos[l - 1, j - 2] if j > 1 else pos[inv[l - 1] - 1, P - 1]
            g[l - 1, j - 1] = k * (2.0 * pos[l - 1, j - 1] - nxt - prv)
    return g


def potential_by_permutations(pos, m, omega_P, beta):
    """Definition forward-potential summed over all N! permutations.

    Returns (V, F, M): V^{[1,N]}, F = sum_sigma Pr(G[sigma]) (-grad E^{G[sigma]})
    (Lemma expected-force), and M[l-1, l'-1] = sum of Pr(G[sigma]) over the sigma
    whose representative sends l to l'.
    """
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    reps = [representative(s) for s in itertools.permutations(range(1, N + 1))]
    energies = {}
    for g in set(reps):
        energies[g] = ring_energy(pos, g, m, omega_P)
    Es = np.array([energies[g] for g in reps])
    Emin = Es.min()
    w = np.exp(-beta * (Es - Emin))
    Z = math.fsum(w)
    V = Emin - math.log(Z / math.factorial(N)) / beta
    pr = w / Z
    grads = {g: ring_gradient(pos, g, m, omega_P) for g in energies}
    F = np.zeros_like(pos)
    M = np.zeros((N, N))
    for p, g in zip(pr, reps):
        F -= p * grads[g]
        for l in range(1, N + 1):
            M[l - 1, g[l - 1] - 1] += p
    return V, F, M


def compositions(N):
    """All cuts of [1, N] into consecutive blocks, as lists of block ends
    v_1 < ... < v_m = N."""
    for mask in range(1 << (N - 1)):
        ends = [v for v in range(1, N) if mask >> (v - 1) & 1]
        ends.append(N)
        yield ends


def consecutive_cycle_energy(pos, u, v, m, omega_P):
    """Energy of the ring u -> u+1 -> ... -> v -> u (Eq. Ek with first index u),
    evaluated as the bead-by-bead sum of Eq. eperm restricted to that ring."""
    pos = np.asarray(pos, dtype=np.float64)
    P = pos.shape[1]
    beads = pos[u - 1:v].reshape(-1, 3)          # beads of u..v in ring order
    d = beads - np.roll(beads, -1, axis=0)       # last bead of v closes onto bead 1 of u
    return 0.5 * m * omega_P ** 2 * float(np.sum(d * d))


def potential_by_compositions(pos, m, omega_P, beta):
    """exp(-beta V^{[1,N]}) as the sum over the 2^(N-1) representative
    permutations: a cut v_1 < ... < v_m = N carries weight
    prod_i (1/v_i) exp(-beta E^{[v_{i-1}+1, v_i]}), the fraction of all N!
    permutations whose representative it is."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    cache = {}

    def Ecyc(u, v):
        if (u, v) not in cache:
            cache[(u, v)] = consecutive_cycle_energy(pos, u, v, m, omega_P)
        return cache[(u, v)]

    logs = []
    for ends in compositions(N):
        prev = 0
        e = 0.0
        logw = 0.0
        for v in ends:
            e += Ecyc(prev + 1, v)
            logw -= math.log(v)
            prev = v
        logs.append(logw - beta * e)
    logs = np.array(logs)
    mx = logs.max()
    return -(mx + math.log(math.fsum(np.exp(logs - mx)))) / beta


def representative_counts(N):
    """Number of permutations of [1, N] mapped by G to each representative,
    keyed by the representative's tuple of cycle ends."""
    counts = {}
    for s in itertools.permutations(range(1, N + 1)):
        cycles = sorted(canonical_cycles(s), key=max)
        ends, acc = [], 0
        for c in cycles:
            acc += len(c)
            ends.append(acc)
        counts[tuple(ends)] = counts.get(tuple(ends), 0) + 1
    return counts
