"""Molecular dynamics of replica batches (bpimd_step on a batch context).

Every replica of an uneven batch (N, P, beta differ; trap w0 = 1, Gaussian
repulsion g = 1, s = 0.5 as in the 256-replica workload) takes k BAOAB steps
in the batch; each is compared with the MD oracle run on that replica alone,
with the thermostat counters of its position in the packed arrays (elem0).
FP64 to 1e-10 of the scale of positions, velocities and energies; the mixed
forms to 1e-5 (float32 pair forces and Box-Muller).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import inputs
from paper_2305_18025_gb300.exchange import BatchedExchangeEnergy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5, "mixed32": 1e-5}
MD = dict(dt=0.01, gamma=1.0, omega0=1.0, gaussian=(1.0, 0.5), seed=4242)


@pytest.mark.parametrize("prec,tile", [("fp64", 4), ("mixed", 4), ("mixed32", 4), ("fp64", 2), ("fp64", 8),
                                       ("mixed", 2), ("mixed", 8)])
def test_batched_md_matches_the_oracle_per_replica(prec, tile):
    """Every pair tile (lanes per particle of the pair forces) of the batch."""
    spec = [(7, 4, 1.0), (33, 8, 0.6), (1, 3, 2.0), (64, 16, 3.1), (20, 6, 1.4), (150, 4, 0.9)]
    Ns, Ps, betas = zip(*spec)
    wPs = [inputs.omega_P(P, b) for P, b in zip(Ps, betas)]
    eng = BatchedExchangeEnergy(Ns, Ps, 1.0, wPs, betas, precision=prec, device="cuda:0",
                                stream=torch.cuda.Stream("cuda:0"), md=MD)
    eng.set_pair_tile(tile)
    pos = [inputs.trapped_positions(N, P, 900 + i) for i, (N, P, _) in enumerate(spec)]
    rng = np.random.default_rng(5)
    vel = [rng.normal(0, 0.5, p.shape) for p in pos]
    x = eng.pack([torch.from_numpy(p) for p in pos])
    v = eng.pack([torch.from_numpy(u) for u in vel])
    nsteps, calls = 3, 2
    for _ in range(calls):
        en = eng.step(x, v, nsteps)
    torch.cuda.synchronize()
    gx = [t.cpu().numpy() for t in eng.unpack(x)]
    gv = [t.cpu().numpy() for t in eng.unpack(v)]
    gen = en.cpu().numpy()
    eng.close()
    t = TOL[prec]
    for r, (N, P, beta) in enumerate(spec):
        ox, ov, oen = pos[r], vel[r], None
        for c in range(calls):
            ox, ov, oen = oracle.float64.md_run(ox, ov, 1.0, wPs[r], beta, MD["dt"], MD["gamma"], nsteps,
                                                omega0=1.0, pair_type=1, pair_a=1.0, pair_b=0.5, seed=MD["seed"],
                                                step0=c * nsteps, elem0=int(eng.offsets[r]))
        assert np.abs(gx[r] - ox).max() <= t * max(1.0, np.abs(ox).max()), r
        assert np.abs(gv[r] - ov).max() <= t * max(1.0, np.abs(ov).max()), r
        np.testing.assert_allclose(gen[r], oen, rtol=0, atol=t * np.abs(oen).max())


def test_batched_md_equals_single_system_runs_without_noise():
    """gamma = 0: no thermostat noise, so a replica in a batch follows exactly
    the trajectory of the same system run alone (same kernels per replica)."""
    from paper_2305_18025_gb300.exchange import RingPolymerMD
    spec = [(12, 4, 1.0), (40, 8, 2.0)]
    Ns, Ps, betas = zip(*spec)
    wPs = [inputs.omega_P(P, b) for P, b in zip(Ps, betas)]
    md = dict(MD, gamma=0.0)
    s = torch.cuda.Stream("cuda:0")
    eng = BatchedExchangeEnergy(Ns, Ps, 1.0, wPs, betas, device="cuda:0", stream=s, md=md)
    pos = [inputs.trapped_positions(N, P, 30 + i) for i, (N, P, _) in enumerate(spec)]
    x = eng.pack([torch.from_numpy(p) for p in pos])
    v = torch.zeros_like(x)
    eng.step(x, v, 10)
    torch.cuda.synchronize()
    gx = [t.cpu().numpy() for t in eng.unpack(x)]
    eng.close()
    for r, (N, P, beta) in enumerate(spec):
        one = RingPolymerMD(N, P, 1.0, wPs[r], beta, dt=md["dt"], gamma=0.0, omega0=1.0, gaussian=md["gaussian"],
                            stream=s)
        xs = torch.tensor(pos[r], device="cuda:0")
        vs = torch.zeros_like(xs)
        one.step(xs, vs, 10)
        torch.cuda.synchronize()
        one.close()
        np.testing.assert_allclose(gx[r], xs.cpu().numpy(), rtol=0, atol=1e-12 * max(1.0, np.abs(gx[r]).max()))


def test_a_pair_tile_changed_between_steps_continues_the_trajectory():
    """Steps 1-3 with 4 lanes per particle, steps 4-6 with 8: the same
    trajectory as the oracle's six steps (the thermostat counter goes on)."""
    spec = [(40, 8, 1.0), (90, 4, 2.0)]
    Ns, Ps, betas = zip(*spec)
    wPs = [inputs.omega_P(P, b) for P, b in zip(Ps, betas)]
    eng = BatchedExchangeEnergy(Ns, Ps, 1.0, wPs, betas, precision="fp64", device="cuda:0",
                                stream=torch.cuda.Stream("cuda:0"), md=MD)
    pos = [inputs.trapped_positions(N, P, 70 + i) for i, (N, P, _) in enumerate(spec)]
    rng = np.random.default_rng(9)
    vel = [rng.normal(0, 0.5, p.shape) for p in pos]
    x = eng.pack([torch.from_numpy(p) for p in pos])
    v = eng.pack([torch.from_numpy(u) for u in vel])
    eng.step(x, v, 3, energies=False)
    eng.set_pair_tile(8)
    eng.step(x, v, 3, energies=False)
    torch.cuda.synchronize()
    gx = [t.cpu().numpy() for t in eng.unpack(x)]
    for r, (N, P, beta) in enumerate(spec):
        ox, ov, _ = oracle.float64.md_run(pos[r], vel[r], 1.0, wPs[r], beta, MD["dt"], MD["gamma"], 6,
                                          omega0=1.0, pair_type=1, pair_a=1.0, pair_b=0.5, seed=MD["seed"],
                                          elem0=int(eng.offsets[r]))
        assert np.abs(gx[r] - ox).max() <= 1e-10 * max(1.0, np.abs(ox).max()), r
    eng.close()


def test_pair_tile_rejects_other_values_and_single_systems():
    from paper_2305_18025_gb300 import bpimd
    from paper_2305_18025_gb300.exchange import ExchangeEnergy
    eng = BatchedExchangeEnergy([8, 9], [4, 4], 1.0, [2.0, 2.0], [1.0, 1.0], precision="fp64", device="cuda:0")
    for bad in (0, 1, 3, 16):
        with pytest.raises(bpimd.BpimdError):
            eng.set_pair_tile(bad)
    eng.close()
    one = ExchangeEnergy(8, 4, 1.0, 2.0, 1.0, device="cuda:0")
    assert bpimd.load().bpimd_batch_set_pair_tile(one.ctx, 4) == bpimd.BPIMD_ERR_STATE
    one.close()
