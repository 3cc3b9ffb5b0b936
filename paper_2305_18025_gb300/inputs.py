"""Seeded synthetic inputs for the exchange kernels and their tests.

This module holds input recipes only -- no arithmetic of the method -- so that
the CUDA path and the CPU oracle can be fed identical inputs without sharing
any code.  Every generator uses numpy's PCG64 (``numpy.random.default_rng``)
and is deterministic for a given seed.

Shapes follow the paper's workloads: trapped bosons with P = 32-36 beads and N
up to ~1600 (Benchmarks section, Methods "Simulation details"), and liquid
helium with P = 64-96 at number density 0.0218 per cubic angstrom.
"""
from dataclasses import dataclass
import math

import numpy as np


def omega_P(P, beta, hbar=1.0):
    """Ring-polymer spring frequency sqrt(P)/(beta hbar) (Eq. eperm)."""
    return math.sqrt(P) / (beta * hbar)


def trapped_positions(N, P, seed, centre_sigma=1.0, offset_sigma=0.1):
    """[N][P][3] float64: particle centres ~ N(0, centre_sigma) per axis, every
    bead displaced from its centre by N(0, offset_sigma) per axis."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, centre_sigma, size=(N, 1, 3))
    offsets = rng.normal(0.0, offset_sigma, size=(N, P, 3))
    return np.ascontiguousarray(centres + offsets)


def coincident_positions(N, P, point=(0.25, -0.5, 1.0)):
    """Every bead of every particle at one point: all springs vanish."""
    pos = np.empty((N, P, 3))
    pos[:] = np.asarray(point, dtype=np.float64)
    return pos


def separated_positions(N, P, seed, spacing=100.0, offset_sigma=0.1):
    """Particle centres on a line `spacing` apart (exchange negligible), beads
    jittered by N(0, offset_sigma)."""
    rng = np.random.default_rng(seed)
    centres = np.zeros((N, 1, 3))
    centres[:, 0, 0] = spacing * np.arange(N)
    return np.ascontiguousarray(centres + rng.normal(0.0, offset_sigma, size=(N, P, 3)))


def clustered_chain_positions(N, P, seed, step=0.05, offset_sigma=0.1):
    """Centres on a random walk with small steps: neighbouring particles overlap,
    so long exchange cycles carry weight and every connection probability of the
    lower Hessenberg band is far from 0 and 1."""
    rng = np.random.default_rng(seed)
    centres = np.cumsum(rng.normal(0.0, step, size=(N, 1, 3)), axis=0)
    return np.ascontiguousarray(centres + rng.normal(0.0, offset_sigma, size=(N, P, 3)))


def fcc_positions(cells, P, box_length, seed, jitter=0.05):
    """Liquid-helium-like start: an FCC lattice of 4*cells^3 atoms filling a cubic
    box of side `box_length`, every bead jittered by N(0, jitter)."""
    rng = np.random.default_rng(seed)
    a = box_length / cells
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    grid = np.array([[i, j, k] for i in range(cells) for j in range(cells) for k in range(cells)],
                    dtype=np.float64)
    centres = ((grid[:, None, :] + basis[None, :, :]).reshape(-1, 3) + 0.25) * a
    N = centres.shape[0]
    return np.ascontiguousarray(centres[:, None, :] + rng.normal(0.0, jitter, size=(N, P, 3)))


@dataclass
class Replica:
    N: int
    P: int
    beta: float
    positions: np.ndarray


def batched_replicas(count, seed, n_range=(16, 512), p_choices=(16, 32, 64),
                     beta_range=(0.5, 4.0)):
    """Independent trapped systems: N ~ U[n_range], P from p_choices, beta ~
    U[beta_range], positions from trapped_positions with per-replica seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        P = int(rng.choice(p_choices))
        beta = float(rng.uniform(*beta_range))
        out.append(Replica(N, P, beta, trapped_positions(N, P, seed * 100003 + r)))
    return out


def random_coordinates(pos_shape, count, seed):
    """`count` distinct flat indices into an array of shape pos_shape (for
    finite-difference spot checks)."""
    rng = np.random.default_rng(seed)
    return rng.choice(int(np.prod(pos_shape)), size=count, replace=False)
