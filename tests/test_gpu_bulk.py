"""GPU parity for bulk systems in a periodic box (liquid-helium workload).

* The exchange potential and forces with minimum-image springs against the
  oracle in the same box, for ring polymers scattered over the whole box (many
  springs cross it): FP64 to the single-system tolerances, MIXED (32-bit
  fixed-point endpoint differences) to 1e-6 / 1e-5.
* MD steps with Lennard-Jones pairs (eps = 10.22 K, sigma = 2.556 A, cutoff
  2.5 sigma; m = 4.0026 amu, T = 1.5 K, hbar = 6.9648 in A, K, amu units) from
  an FCC start at the liquid density, against the MD oracle: a box smaller than
  three cutoffs (all-pairs path) and one larger (cell-list path).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import inputs
from paper_2305_18025_gb300.exchange import ExchangeEnergy, RingPolymerMD

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
HBAR = 6.9648                    # hbar in A sqrt(amu K)
M_HE, BETA_HE = 4.0026, 1.0 / 1.5
LJ = (10.22, 2.556, 2.5 * 2.556)
RHO = 0.0218                     # A^-3


def wrapped_liquid(N, P, L, seed, spread):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, L, (N, 1, 3))
    return np.mod(centres + rng.normal(0, spread, (N, P, 3)), L)


def reference(pos, m, wP, beta, L):
    if pos.shape[0] < 128:
        VB, F = oracle.float64.fast_pimdb(pos, m, wP, beta, box=L)
    else:
        VB, F = oracle.long_double.fast_pimdb(pos, m, wP, beta, box=L)
    return float(VB), np.asarray(F, dtype=np.float64)


@pytest.mark.parametrize("prec,tv,tf", [("fp64", 1e-12, 1e-10), ("mixed", 1e-6, 1e-5), ("mixed32", 1e-6, 1e-5)])
@pytest.mark.parametrize("N,P,L,spread", [(20, 4, 3.0, 0.3), (100, 8, 5.0, 0.4), (300, 6, 8.0, 0.5)])
def test_exchange_in_a_box_matches_oracle(prec, tv, tf, N, P, L, spread):
    beta = 1.0
    wP = inputs.omega_P(P, beta)
    pos = wrapped_liquid(N, P, L, seed=N, spread=spread)
    VB, F = reference(pos, 1.0, wP, beta, L)
    eng = ExchangeEnergy(N, P, 1.0, wP, beta, precision=prec, device=DEV, box=L)
    V, G = eng.forces(torch.from_numpy(pos).to(DEV))
    eng.sync()
    V, G = float(V.cpu()), G.cpu().numpy()
    scale = max(abs(VB), 1.0 / beta)  # |V_B|, with kT as the floor where V_B is near 0
    assert abs(V - VB) <= tv * scale, (V, VB)
    assert np.linalg.norm(G - F) <= tf * np.linalg.norm(F)
    # periodicity: moving beads by lattice vectors changes nothing
    shifted = pos + L * np.random.default_rng(1).integers(-1, 2, pos.shape)
    V2, G2 = eng.forces(torch.from_numpy(shifted).to(DEV))
    eng.sync()
    assert abs(float(V2.cpu()) - V) <= 10 * tv * scale
    assert np.linalg.norm(G2.cpu().numpy() - G) <= 10 * tf * np.linalg.norm(F)
    eng.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-5), ("mixed32", 1e-5)])
@pytest.mark.parametrize("cells", [3, 4])
def test_helium_md_matches_oracle(prec, tol, cells):
    """cells = 3: 108 atoms, L = 17.0 A < 3 rc (all pairs); cells = 4: 256
    atoms, L = 22.7 A >= 3 rc (cell lists, 3^3 cells per bead index)."""
    P = 4
    N = 4 * cells ** 3
    L = (N / RHO) ** (1.0 / 3.0)
    wP = np.sqrt(P) / (BETA_HE * HBAR)
    pos = inputs.fcc_positions(cells, P, L, seed=cells, jitter=0.05)
    vel = np.random.default_rng(cells + 1).normal(0, np.sqrt(1.0 / (BETA_HE * M_HE)), pos.shape)
    dt, nsteps = 0.005, 3
    ox, ov, oen = oracle.float64.md_run(pos, vel, M_HE, wP, BETA_HE, dt, 1.0, nsteps, pair_type=2,
                                        pair_a=LJ[0], pair_b=LJ[1], pair_rc=LJ[2], box=L, seed=17)
    md = RingPolymerMD(N, P, M_HE, wP, BETA_HE, dt=dt, gamma=1.0, lennard_jones=LJ, box=L, seed=17,
                       precision=prec, device=DEV, stream=torch.cuda.Stream(DEV))
    x, v = torch.from_numpy(pos.copy()).to(DEV), torch.from_numpy(vel.copy()).to(DEV)
    en = md.step(x, v, nsteps).cpu().numpy()
    md.close()
    gx, gv = x.cpu().numpy(), v.cpu().numpy()
    assert np.abs(gx - ox).max() <= tol * L
    assert np.abs(gv - ov).max() <= tol * max(1.0, np.abs(ov).max())
    np.testing.assert_allclose(en, oen, rtol=0, atol=tol * np.abs(oen).max())
