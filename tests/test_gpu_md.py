"""GPU parity of the molecular-dynamics step (bpimd_step) with the MD oracle.

Trajectories: the same seeded start, the same Philox4x32-10 thermostat noise
(both sides implement the published generator), k BAOAB steps; positions,
velocities and the four energies are compared element by element.
  FP64 : positions/velocities to 1e-10 of their scale; energies to 1e-10 relative.
  MIXED: float32 pair terms and float32 Box-Muller: 1e-5.
Statistics: <E_prim> of trapped bosons against the closed form at finite P and
equipartition, within four block standard errors; bounded NVE energy error.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import harmonic
from paper_2305_18025_gb300 import inputs
from paper_2305_18025_gb300.exchange import RingPolymerMD

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5, "mixed32": 1e-5}


def _start(N, P, seed):
    pos = inputs.trapped_positions(N, P, seed)
    vel = np.random.default_rng(seed + 1).normal(0, 0.5, pos.shape)
    return pos, vel


def _run_gpu(pos, vel, beta, prec, nsteps, calls=1, stream=None, **kw):
    N, P, _ = pos.shape
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream(dev) if stream == "side" else None
    md = RingPolymerMD(N, P, 1.0, inputs.omega_P(P, beta), beta, precision=prec, stream=s, **kw)
    x = torch.tensor(pos, device=dev)
    v = torch.tensor(vel, device=dev)
    en = None
    for _ in range(calls):
        en = md.step(x, v, nsteps)
    torch.cuda.synchronize()
    out = x.cpu().numpy(), v.cpu().numpy(), en.cpu().numpy()
    md.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
@pytest.mark.parametrize("stream", [None, "side"])
@pytest.mark.parametrize("N,P,beta,pair", [(16, 8, 2.0, True), (5, 4, 1.0, False), (40, 6, 1.5, True)])
def test_md_trajectory_matches_oracle(prec, stream, N, P, beta, pair):
    pos, vel = _start(N, P, 100 + N)
    kw = dict(dt=0.01, gamma=1.0, omega0=1.0, seed=12345)
    gkw = dict(kw)
    okw = dict(omega0=1.0, seed=12345)
    if pair:
        gkw["gaussian"] = (3.0, 0.5)
        okw.update(pair_type=1, pair_a=3.0, pair_b=0.5)
    nsteps, calls = 4, 2
    gx, gv, gen_ = _run_gpu(pos, vel, beta, prec, nsteps, calls, stream, **gkw)
    wP = inputs.omega_P(P, beta)
    ox, ov, oen = pos, vel, None
    for c in range(calls):
        ox, ov, oen = oracle.float64.md_run(ox, ov, 1.0, wP, beta, 0.01, 1.0, nsteps, step0=c * nsteps, **okw)
    t = TOL[prec]
    assert np.abs(gx - ox).max() <= t * max(1.0, np.abs(ox).max())
    assert np.abs(gv - ov).max() <= t * max(1.0, np.abs(ov).max())
    scale = np.abs(oen).max()
    np.testing.assert_allclose(gen_, oen, rtol=0, atol=t * scale)


def test_md_nve_energy_is_conserved():
    N, P, beta = 8, 8, 2.0
    pos, vel = _start(N, P, 7)
    wP = inputs.omega_P(P, beta)
    dev = torch.device("cuda", 0)
    md = RingPolymerMD(N, P, 1.0, wP, beta, dt=0.005, gamma=0.0, omega0=1.0, gaussian=(3.0, 0.5),
                       stream=torch.cuda.Stream(dev))
    x, v = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    H = []
    for _ in range(20):
        en = md.step(x, v, 50).cpu().numpy()
        H.append(en[0] + en[1] + en[2])
    H = np.array(H)
    assert np.abs(H - H[0]).max() < 2e-3 * abs(H[0])
    md.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_md_harmonic_closed_form_and_equipartition(prec):
    """N = 4 trapped bosons, P = 8, beta = 2 (beta hbar w0 = 2): <E_prim> equals
    -d ln Z/d beta of the P-bead discretisation (closed form), <KE> = 3NP/(2 beta)."""
    N, P, beta = 4, 8, 2.0
    wP = inputs.omega_P(P, beta)
    dev = torch.device("cuda", 0)
    md = RingPolymerMD(N, P, 1.0, wP, beta, dt=0.02, gamma=1.0, omega0=1.0, seed=99, precision=prec,
                       stream=torch.cuda.Stream(dev))
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.normal(0, 0.7, (N, P, 3)), device=dev)
    v = torch.zeros_like(x)
    md.step(x, v, 4000, energies=False)
    samples = []
    for _ in range(6000):
        samples.append(md.step(x, v, 25).clone())
    en = torch.stack(samples).cpu().numpy()
    md.close()
    for col, exact in [(2, 1.5 * N * P / beta), (3, harmonic.mean_energy(N, P, beta, 1.0))]:
        b = en[:, col].reshape(60, -1).mean(axis=1)
        err = b.std(ddof=1) / np.sqrt(len(b))
        assert abs(b.mean() - exact) < 4 * err + 2e-3 * abs(exact), (col, b.mean(), exact, err)


def test_md_rejects_invalid_parameters():
    dev = torch.device("cuda", 0)
    from paper_2305_18025_gb300 import bpimd
    x = torch.zeros((4, 3, 3), dtype=torch.float64, device=dev)
    v = torch.zeros_like(x)
    for bad in [dict(dt=0.0), dict(dt=0.01, gamma=-1.0), dict(dt=0.01, omega0=-1.0),
                dict(dt=0.01, gaussian=(1.0, 0.0))]:
        md = RingPolymerMD(4, 3, 1.0, 1.0, 1.0, **bad)
        with pytest.raises(bpimd.BpimdError) as e:
            md.step(x, v, 1)
        assert e.value.status == bpimd.BPIMD_ERR_ARG
        md.close()
