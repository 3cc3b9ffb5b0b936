"""Trapped non-interacting bosons at the validation size: N = 64, P = 32,
beta in {0.5, 1, 2, 4}, m = hbar = w0 = 1, BAOAB Langevin with dt = 0.005,
gamma = 1 (the paper's harmonic-trap check, Methods "Numerical Validation",
whose bar is 0.5 % relative deviation from the analytical energy).

The sampled means are compared with the closed form of the same P-bead
discretisation (oracle.harmonic), so no Trotter error enters:
  * <U-bar>, the mean trap energy, a low-variance observable;
  * <E_prim>, the primitive estimator, whose variance grows with P.
Each mean must lie within four block standard errors plus 0.5 % of the exact
value.  BAOAB samples the configurations of a harmonic system without a
time-step bias, so the 0.5 % allowance is the paper's bar, not a dt correction.
Below beta = 2 the system is largely Bose-condensed (N = 64 in a trap: T_c is
about 3.8 hbar w0) and the sampled cycle structure decorrelates over hundreds
of time units: those two temperatures run 1e6 steps (mixed form), the others
1e5 steps in both forms.
Also: total energy under NVE (gamma = 0) over 1e4 steps at N = 64, P = 32.
"""
import numpy as np
import pytest
import torch

from oracle import harmonic
from paper_2305_18025_gb300 import inputs
from paper_2305_18025_gb300.exchange import RingPolymerMD

pytestmark = pytest.mark.gpu

N, P, DT = 64, 32, 0.005


def block_stats(x, nblocks=40):
    b = np.asarray(x[: len(x) // nblocks * nblocks]).reshape(nblocks, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nblocks)


@pytest.mark.parametrize("prec,beta,steps", [("mixed", 0.5, 1000000), ("mixed", 1.0, 1000000),
                                             ("fp64", 2.0, 100000), ("mixed", 2.0, 100000),
                                             ("fp64", 4.0, 100000), ("mixed", 4.0, 100000)])
def test_trapped_bosons_n64_p32_match_the_closed_form(prec, beta, steps):
    dev = torch.device("cuda", 0)
    wP = inputs.omega_P(P, beta)
    md = RingPolymerMD(N, P, 1.0, wP, beta, dt=DT, gamma=1.0, omega0=1.0, seed=2024 + int(8 * beta),
                       precision=prec, stream=torch.cuda.Stream(dev))
    x = torch.tensor(inputs.trapped_positions(N, P, seed=int(10 * beta)), device=dev)
    v = torch.zeros_like(x)
    md.step(x, v, steps // 10, energies=False)       # equilibration
    every = 100 if steps > 100000 else 25
    samples = [md.step(x, v, every).clone() for _ in range(steps // every)]
    en = torch.stack(samples).cpu().numpy()
    md.close()
    assert np.all(np.isfinite(en))
    for col, exact in [(1, harmonic.mean_trap_energy(N, P, beta, 1.0)), (3, harmonic.mean_energy(N, P, beta, 1.0))]:
        m, se = block_stats(en[:, col])
        assert abs(m - exact) <= 4 * se + 5e-3 * abs(exact), (col, m, exact, se)


def test_nve_energy_over_ten_thousand_steps_at_n64():
    """gamma = 0: velocity Verlet with the exchange, trap and Gaussian pair
    forces.  The total energy V_B + U-bar + KE stays within 1e-3 of its start
    and shows no drift beyond 1e-4 of it between the first and last tenth."""
    beta = 1.0
    dev = torch.device("cuda", 0)
    wP = inputs.omega_P(P, beta)
    pos = inputs.trapped_positions(N, P, seed=31)
    vel = np.random.default_rng(32).normal(0, 1.0, pos.shape)
    md = RingPolymerMD(N, P, 1.0, wP, beta, dt=DT, gamma=0.0, omega0=1.0, gaussian=(3.0, 0.5),
                       stream=torch.cuda.Stream(dev))
    x, v = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    H = []
    for _ in range(200):
        e = md.step(x, v, 50).cpu().numpy()
        H.append(e[0] + e[1] + e[2])
    md.close()
    H = np.array(H)
    assert np.abs(H - H[0]).max() <= 1e-3 * abs(H[0]), np.abs(H - H[0]).max() / abs(H[0])
    assert abs(H[-20:].mean() - H[:20].mean()) <= 1e-4 * abs(H[0])
