"""GPU parity of replica batches (bpimd_create_batched) with the oracle.

Every replica of a batch of uneven N, P, beta is compared with the oracle's
Algorithm 1 on the same positions (float64 build below N = 128, long-double
referee from N = 128): FP64 to the single-system tolerances, MIXED to 1e-6 on
V_B and 1e-5 RMS-relative on forces.  The 256-replica workload (N ~ U[16,512],
P in {16,32,64}, beta ~ U[0.5,4]) is checked on a sample of replicas against
the oracle and on all of them for the zero net exchange force.  The launch
shape chosen by the autotuner must not change a single bit of the results.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import autotune, bpimd, inputs
from paper_2305_18025_gb300.exchange import BatchedExchangeEnergy, ExchangeEnergy

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TOL = {"fp64": dict(v=1e-12, f=1e-10), "mixed": dict(v=1e-6, f=1e-5), "mixed32": dict(v=1e-6, f=1e-5)}


def reference(pos, wP, beta):
    if pos.shape[0] < 128:
        VB, F = oracle.fast_pimdb(pos, 1.0, wP, beta)
    else:
        VB, F = oracle.long_double.fast_pimdb(pos, 1.0, wP, beta)
    return float(VB), np.asarray(F, dtype=np.float64)


def energy_floor(beta):
    """kT: V_B is compared relative to |V_B|, with tolerance x kT as an absolute
    floor that binds only where V_B is within kT of zero (coincident beads)."""
    return 1.0 / beta


def run_batch(systems, prec):
    Ns = [p.shape[0] for p, _ in systems]
    Ps = [p.shape[1] for p, _ in systems]
    betas = [b for _, b in systems]
    wPs = [inputs.omega_P(P, b) for P, b in zip(Ps, betas)]
    eng = BatchedExchangeEnergy(Ns, Ps, 1.0, wPs, betas, precision=prec, device=DEV)
    x = eng.pack([torch.from_numpy(p) for p, _ in systems])
    V, F = eng.forces(x)
    eng.sync()
    out = V.cpu().numpy(), [f.cpu().numpy() for f in eng.unpack(F)], eng, x
    return out


def check(systems, V, Fs, prec, idx=None):
    t = TOL[prec]
    for r in (range(len(systems)) if idx is None else idx):
        pos, beta = systems[r]
        wP = inputs.omega_P(pos.shape[1], beta)
        VB, F = reference(pos, wP, beta)
        assert abs(V[r] - VB) <= t["v"] * max(abs(VB), energy_floor(beta)), (r, V[r], VB)
        assert np.linalg.norm(Fs[r] - F) <= t["f"] * np.linalg.norm(F), (r, np.linalg.norm(Fs[r] - F) / np.linalg.norm(F))


MIX = [(1, 2, 1.0, "trapped"), (5, 3, 0.7, "clustered"), (31, 8, 2.0, "trapped"), (32, 4, 1.3, "clustered"),
       (33, 16, 0.5, "trapped"), (64, 2, 4.0, "trapped"), (100, 8, 1.0, "clustered"), (257, 6, 1.1, "trapped"),
       (20, 6, 1.0, "separated"), (40, 4, 1.0, "coincident"), (513, 5, 0.9, "clustered"), (2, 32, 3.0, "trapped")]


def make(kind, N, P, seed):
    if kind == "trapped":
        return inputs.trapped_positions(N, P, seed)
    if kind == "clustered":
        return inputs.clustered_chain_positions(N, P, seed)
    if kind == "separated":
        return inputs.separated_positions(N, P, seed)
    return inputs.coincident_positions(N, P)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_mixed_batch_matches_oracle(prec):
    systems = [(make(k, N, P, 500 + i), b) for i, (N, P, b, k) in enumerate(MIX)]
    V, Fs, eng, _ = run_batch(systems, prec)
    check(systems, V, Fs, prec)
    eng.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_256_replica_workload(prec):
    reps = inputs.batched_replicas(256, seed=11)
    systems = [(rep.positions, rep.beta) for rep in reps]
    V, Fs, eng, _ = run_batch(systems, prec)
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(systems), size=8, replace=False).tolist())
    check(systems, V, Fs, prec, idx=sample)
    ztol = 1e-8 if prec == "fp64" else 1e-4
    for r, F in enumerate(Fs):   # exchange + spring forces are internal: zero net force
        assert np.abs(F.sum(axis=(0, 1))).max() <= ztol * max(1.0, np.abs(F).max()), r
    eng.close()


def test_batch_equals_single_system_contexts():
    systems = [(make(k, N, P, 700 + i), b) for i, (N, P, b, k) in enumerate(MIX[:6])]
    V, Fs, eng, _ = run_batch(systems, "fp64")
    for r, (pos, beta) in enumerate(systems):
        N, P, _ = pos.shape
        one = ExchangeEnergy(N, P, 1.0, inputs.omega_P(P, beta), beta, device=DEV)
        v1, f1 = one.forces(torch.from_numpy(pos).to(DEV))
        one.sync()
        scale = max(abs(float(v1.cpu())), energy_floor(beta))
        assert abs(float(v1.cpu()) - V[r]) <= 1e-13 * scale
        np.testing.assert_allclose(Fs[r], f1.cpu().numpy(), rtol=0, atol=1e-11 * np.abs(Fs[r]).max())
        one.close()
    eng.close()


def test_autotuner_choice_does_not_change_results(tmp_path, monkeypatch):
    monkeypatch.setenv("BPIMD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    reps = inputs.batched_replicas(64, seed=12)
    systems = [(rep.positions, rep.beta) for rep in reps]
    V0, F0, eng, x = run_batch(systems, "mixed")
    res = autotune.tune(eng, x, reps=2)
    assert not res["cached"] and len(res["timings_ms"]) == len(autotune.CANDIDATES)
    for cand in ((2, 2), (32, 32), res["choice"]):
        eng.set_tuning(*cand)
        V, F = eng.forces(x)
        eng.sync()
        assert np.array_equal(V.cpu().numpy(), V0)
        for a, b in zip(eng.unpack(F), F0):
            assert np.array_equal(a.cpu().numpy(), b)
    again = autotune.tune(eng, x)
    assert again["cached"] and tuple(again["choice"]) == tuple(res["choice"])
    eng.close()


def test_single_system_calls_rejected_on_batch_context():
    systems = [(make("trapped", 8, 4, 1), 1.0), (make("trapped", 12, 3, 2), 2.0)]
    _, _, eng, x = run_batch(systems, "fp64")
    with pytest.raises(bpimd.BpimdError) as e:
        bpimd.bpimd_exchange_energy_forces(eng.ctx, x, None, torch.empty_like(x))
    assert e.value.status == bpimd.BPIMD_ERR_STATE
    eng.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_with_a_replica_above_4096(prec):
    """A replica larger than the one-CTA recursion holds (N = 5000) runs the
    cluster recursion kernel inside the batch; every replica matches the oracle."""
    systems = [(make("trapped", 5000, 2, 811), 1.0), (make("clustered", 40, 8, 812), 0.8),
               (make("trapped", 300, 4, 813), 2.0)]
    V, Fs, eng, _ = run_batch(systems, prec)
    eng.close()
    check(systems, V, Fs, prec)
