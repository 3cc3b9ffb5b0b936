"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element, on the same seeded inputs.

Tolerances (written here, from the target accuracy of each precision form):
  FP64 : |dV_B| <= 1e-12 |V_B|;  ||dF||_2 <= 1e-10 ||F||_2 and
         max|dF| <= 1e-10 max|F|;  every potential V^{[1,v]}, V^{[u,N]} to
         1e-12 of its own magnitude; probabilities to 1e-10 absolute.
  MIXED: |dV_B| <= 1e-6 |V_B|;  RMS-relative ||dF||_2 / ||F||_2 <= 1e-5;
         potentials to 1e-6 of their own magnitude; probabilities to 1e-5
         absolute.
  Energies are relative to their own magnitude with one absolute floor, the
  same tolerance times kT = 1/beta (energy_floor): it binds only where an
  energy is within kT of zero, as for coincident beads, where V_B = 0 exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import bpimd, inputs
from paper_2305_18025_gb300.exchange import ExchangeEnergy

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(v=1e-12, f=1e-10, fmax=1e-10, pot=1e-12, M=1e-10),
       "mixed": dict(v=1e-6, f=1e-5, fmax=None, pot=1e-6, M=1e-5),
       "mixed32": dict(v=1e-6, f=1e-5, fmax=None, pot=1e-6, M=1e-5)}


def gen(kind, N, P, seed):
    if kind == "trapped":
        return inputs.trapped_positions(N, P, seed)
    if kind == "clustered":
        return inputs.clustered_chain_positions(N, P, seed)
    if kind == "coincident":
        return inputs.coincident_positions(N, P)
    if kind == "separated":
        return inputs.separated_positions(N, P, seed)
    raise ValueError(kind)


def run_gpu(pos, beta, prec, want_M=False, m=1.0):
    N, P, _ = pos.shape
    wP = inputs.omega_P(P, beta)
    eng = ExchangeEnergy(N, P, m, wP, beta, precision=prec, device="cuda:0")
    V, F = eng.forces(torch.from_numpy(pos).cuda())
    eng.sync()
    Vf, Vb, Ei = eng.potentials()
    M = eng.connection_probabilities().cpu().numpy() if want_M else None
    out = float(V.cpu()), F.cpu().numpy(), Vf, Vb, Ei, M
    eng.close()
    return out


def energy_floor(beta):
    """kT: the absolute floor of energy comparisons (tolerance x kT), binding
    only where an energy is within kT of zero."""
    return 1.0 / beta


def assert_energy(got, want, tol, beta, what="V_B"):
    err = abs(got - want)
    assert err <= tol * max(abs(want), energy_floor(beta)), (what, got, want, err / max(abs(want), 1e-300))


def reference(pos, m, wP, beta, full=True):
    """The oracle's Algorithm 1.  From N = 128 on, the long-double build is the
    reference: the float64 oracle's own rounding (the shifted log-sum-exp adds
    about eps*|V| per step) reaches ~1e-10 on forces at N ~ 1000 for trapped
    inputs, and at N = 300 for well-separated particles, where the long-double
    build reproduces the exact ring-polymer forces to 3e-14."""
    N = pos.shape[0]
    if N < 128:
        return oracle.fast_pimdb(pos, m, wP, beta, full=full)
    out = oracle.long_double.fast_pimdb(pos, m, wP, beta, full=full)
    return tuple(float(x) if np.ndim(x) == 0 else (None if x is None else np.asarray(x, np.float64))
                 for x in out)


def check(pos, beta, prec, want_M=True, m=1.0):
    N, P, _ = pos.shape
    wP = inputs.omega_P(P, beta)
    VB, F, Vf, Vb, M = reference(pos, m, wP, beta, full=True)
    gV, gF, gVf, gVb, gEi, gM = run_gpu(pos, beta, prec, want_M=want_M, m=m)
    t = TOL[prec]
    assert_energy(gV, VB, t["v"], beta)
    nF = np.linalg.norm(F)
    if nF > 0:
        assert np.linalg.norm(gF - F) <= t["f"] * nF, np.linalg.norm(gF - F) / nF
        if t["fmax"]:
            assert np.abs(gF - F).max() <= t["fmax"] * np.abs(F).max()
    else:
        assert np.abs(gF).max() <= 1e-12
    floor = t["pot"] * energy_floor(beta)
    np.testing.assert_allclose(gVf, Vf, rtol=t["pot"], atol=floor)
    np.testing.assert_allclose(gVb, Vb, rtol=t["pot"], atol=floor)
    np.testing.assert_allclose(gEi, oracle.interior_energies(pos, m, wP), rtol=max(t["pot"], 1e-13),
                               atol=1e-13)
    if want_M:
        np.testing.assert_allclose(gM, M, rtol=0, atol=t["M"])
    return gV, gF


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
@pytest.mark.parametrize("N,P,kind", [
    (1, 2, "trapped"), (1, 5, "trapped"), (2, 3, "trapped"), (3, 4, "clustered"),
    (5, 2, "clustered"), (16, 8, "trapped"), (31, 8, "clustered"), (32, 8, "trapped"),
    (33, 3, "clustered"), (64, 32, "trapped"), (100, 16, "clustered"), (257, 6, "trapped"),
    (40, 4, "coincident"), (20, 6, "separated"), (300, 8, "separated"), (1024, 4, "coincident"),
])
def test_parity_small(prec, N, P, kind):
    check(gen(kind, N, P, seed=1000 + N), beta=1.3, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
@pytest.mark.parametrize("N", [256, 257, 289, 1313])
def test_parity_cluster_size_switch(prec, N):
    """The recursion switches from 8- to 16-CTA clusters above N = 256 (8 row
    tiles): the last 8-CTA size, the first 16-CTA size (a one-row ragged
    tail), fewer row tiles than bulk CTAs, and a tile count that is not a
    multiple of the 15 bulk CTAs."""
    check(inputs.trapped_positions(N, 4, seed=N), beta=1.0, prec=prec, want_M=False)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0, 4.0])
def test_parity_beta_sweep(prec, beta):
    check(inputs.trapped_positions(64, 32, seed=7), beta=beta, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_parity_headline_size(prec):
    """N = 1024, P = 32, beta = 1: the throughput configuration, element by element."""
    check(inputs.trapped_positions(1024, 32, seed=3), beta=1.0, prec=prec, want_M=False)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_parity_large_n(prec):
    """N = 4096, P = 64 (liquid-helium-sized system, trapped inputs)."""
    check(inputs.clustered_chain_positions(4096, 64, seed=5), beta=1.0, prec=prec, want_M=False)


def load_referee(name):
    import os
    d = {"F": {}, "VF": {}, "VBW": {}}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[0] in d:
                d[p[0]][int(p[1])] = float(p[2])
            else:
                d[p[0]] = float(p[1])
    return d


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_parity_maximum_size(prec):
    """Largest N the recursion kernel accepts (6912), against sampled outputs of
    the long-double oracle stored by tests/golden/make_referee_samples.py."""
    ref = load_referee("referee_N6912_P4_trapped_seed9_beta1.txt")
    N, P, beta = int(ref["N"]), int(ref["P"]), ref["beta"]
    pos = inputs.trapped_positions(N, P, int(ref["seed"]))
    gV, gF, gVf, gVb, _, _ = run_gpu(pos, beta, prec)
    t = TOL[prec]
    assert_energy(gV, ref["VB"], t["v"], beta)
    idx = np.array(sorted(ref["F"]))
    want = np.array([ref["F"][i] for i in idx])
    got = gF.reshape(-1)[idx]
    # the sample's share of the full norm: compare on the sampled components
    assert np.linalg.norm(got - want) <= t["f"] * np.linalg.norm(want)
    if t["fmax"]:
        assert np.abs(got - want).max() <= t["fmax"] * ref["FMAX"]
    for v, val in ref["VF"].items():
        assert_energy(gVf[v], val, t["pot"], beta, f"V^[1,{v}]")
    for v, val in ref["VBW"].items():
        assert_energy(gVb[v], val, t["pot"], beta, f"V^[{v + 1},N]")


def test_gpu_probability_invariants():
    """Row and column sums of Pr are 1; zero above the superdiagonal."""
    pos = inputs.clustered_chain_positions(300, 8, seed=2)
    *_, M = run_gpu(pos, 1.0, "fp64", want_M=True)
    np.testing.assert_allclose(M.sum(axis=0), 1.0, atol=1e-11)
    np.testing.assert_allclose(M.sum(axis=1), 1.0, atol=1e-11)
    assert np.all(np.triu(M, 2) == 0.0)


def test_gpu_deterministic():
    pos = torch.from_numpy(inputs.trapped_positions(700, 16, seed=4)).cuda()
    eng = ExchangeEnergy(700, 16, 1.0, inputs.omega_P(16, 1.0), 1.0, device="cuda:0")
    V1, F1 = eng.forces(pos)
    V1, F1 = V1.clone(), F1.clone()
    V2, F2 = eng.forces(pos)
    eng.sync()
    assert torch.equal(V1, V2) and torch.equal(F1, F2)


def test_host_entry_point_matches_device():
    pos = inputs.trapped_positions(128, 8, seed=6)
    wP = inputs.omega_P(8, 1.0)
    eng = ExchangeEnergy(128, 8, 1.0, wP, 1.0, device="cuda:0")
    V, F = eng.forces(torch.from_numpy(pos).cuda())
    Vh, Fh = eng.forces_host(torch.from_numpy(pos.copy()).pin_memory())
    assert Vh == float(V.cpu())
    assert torch.equal(Fh, F.cpu())


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_point_pinned_and_pageable(prec, pinned):
    """Pinned and pageable host buffers give the device entry point's bits,
    also when a context's staging buffers are reused by a second call."""
    N, P = 300, 6
    pos = inputs.trapped_positions(N, P, seed=8)
    wP = inputs.omega_P(P, 1.0)
    eng = ExchangeEnergy(N, P, 1.0, wP, 1.0, precision=prec, device="cuda:0")
    V, F = eng.forces(torch.from_numpy(pos).cuda())
    eng.sync()
    x = torch.from_numpy(pos.copy())
    Fh = torch.full((N, P, 3), float("nan"), dtype=torch.float64)
    if pinned:
        x, Fh = x.pin_memory(), Fh.pin_memory()
    for _ in range(2):  # the second call reuses the first call's buffers
        Vh, Fh = eng.forces_host(x, Fh)
        assert Vh == float(V.cpu())
        assert torch.equal(Fh, F.cpu())
    eng.close()


def test_nonfinite_positions_are_reported():
    pos = inputs.trapped_positions(8, 4, seed=0)
    pos[3, 2, 1] = np.nan
    eng = ExchangeEnergy(8, 4, 1.0, 2.0, 1.0, device="cuda:0")
    eng.forces(torch.from_numpy(pos).cuda())
    with pytest.raises(bpimd.BpimdError) as ei:
        eng.sync()
    assert ei.value.status == bpimd.BPIMD_ERR_NONFINITE
    # the context stays usable after the error is reported
    good = inputs.trapped_positions(8, 4, seed=0)
    eng.forces(torch.from_numpy(good).cuda())
    eng.sync()


def test_host_call_graph_replay_reports_status_and_follows_the_data():
    """Pinned buffers on a non-default stream: the host call is captured once
    and replayed.  Replays read the buffer's current contents, a non-finite
    input is reported (and cleared), and the context stays usable."""
    N, P = 40, 6
    wP = inputs.omega_P(P, 1.0)
    side = torch.cuda.Stream("cuda:0")
    eng = ExchangeEnergy(N, P, 1.0, wP, 1.0, device="cuda:0", stream=side)
    x = torch.empty((N, P, 3), dtype=torch.float64).pin_memory()
    Fh = torch.empty((N, P, 3), dtype=torch.float64).pin_memory()
    for seed in (1, 2):  # same buffers, new contents: the replay follows them
        pos = inputs.trapped_positions(N, P, seed=seed)
        x.copy_(torch.from_numpy(pos))
        Vh, Fh = eng.forces_host(x, Fh)
        VB, F = oracle.fast_pimdb(pos, 1.0, wP, 1.0)
        assert_energy(Vh, float(VB), 1e-12, 1.0)
        assert np.linalg.norm(Fh.numpy() - F) <= 1e-10 * np.linalg.norm(F)
    bad = inputs.trapped_positions(N, P, seed=3)
    bad[5, 1, 2] = np.inf
    x.copy_(torch.from_numpy(bad))
    with pytest.raises(bpimd.BpimdError) as ei:
        eng.forces_host(x, Fh)
    assert ei.value.status == bpimd.BPIMD_ERR_NONFINITE
    pos = inputs.trapped_positions(N, P, seed=4)
    x.copy_(torch.from_numpy(pos))
    Vh, Fh = eng.forces_host(x, Fh)  # cleared: the next call succeeds
    VB, F = oracle.fast_pimdb(pos, 1.0, wP, 1.0)
    assert_energy(Vh, float(VB), 1e-12, 1.0)
    eng.close()


def test_invalid_size_rejected_on_host():
    with pytest.raises(bpimd.BpimdError) as ei:
        ExchangeEnergy(8, 1, 1.0, 2.0, 1.0, device="cuda:0")
    assert ei.value.status == bpimd.BPIMD_ERR_ARG


@pytest.fixture(scope="module")
def condensed_snapshot():
    """N = 64, P = 32, beta = 0.5 trapped bosons after 4e4 BAOAB steps from a
    compact start: a configuration from the equilibrium of the sampler, with
    long exchange cycles (the closed-form energy of this state point is that of
    a largely condensed system), unlike the seeded test inputs."""
    from paper_2305_18025_gb300.exchange import RingPolymerMD
    N, P, beta = 64, 32, 0.5
    dev = torch.device("cuda", 0)
    md = RingPolymerMD(N, P, 1.0, inputs.omega_P(P, beta), beta, dt=0.005, gamma=1.0, omega0=1.0, seed=5,
                       precision="mixed32", stream=torch.cuda.Stream(dev))
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.normal(0, 0.5, (N, 1, 3)) + rng.normal(0, 0.05, (N, P, 3)), device=dev)
    v = torch.zeros_like(x)
    md.step(x, v, 40000, energies=False)
    md.close()
    return x.cpu().numpy(), beta


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_parity_on_an_equilibrated_condensed_snapshot(prec, condensed_snapshot):
    pos, beta = condensed_snapshot
    wP = inputs.omega_P(pos.shape[1], beta)
    VB, F, Vf, Vb, M = oracle.long_double.fast_pimdb(pos, 1.0, wP, beta, full=True)
    # the exchange is strong here: most of each row's probability is off the diagonal
    assert np.mean(np.diag(np.asarray(M, np.float64))) < 0.6
    check(pos, beta, prec)
