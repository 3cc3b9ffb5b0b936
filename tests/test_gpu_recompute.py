"""GPU parity of the recompute mode: no O(N^2) storage; the pair factors g
are recomputed by the recursions and the probability pass wherever they are
used (automatic above BPIMD_STORE_MAX_N, or with BPIMD_FLAG_RECOMPUTE).

* Against the oracle (long-double referee from N = 128), all three precision
  forms, with the tolerances of the stored mode (test_gpu_parity.py).
* Against the stored mode on the same inputs: the recursions see the same bits
  of g, so V_B and every V^{[1,v]}, V^{[u,N]} are identical; the forces differ
  only by the order of their sums (1e-13 relative).
* N = 16384, P = 4 (the largest N; recompute mode automatically) against
  sampled outputs of the long-double oracle stored by
  tests/golden/make_referee_samples.py.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import bpimd, inputs
from paper_2305_18025_gb300.exchange import ExchangeEnergy

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(v=1e-12, f=1e-10, pot=1e-12), "mixed": dict(v=1e-6, f=1e-5, pot=1e-6),
       "mixed32": dict(v=1e-6, f=1e-5, pot=1e-6)}


def gen(kind, N, P, seed):
    return {"trapped": lambda: inputs.trapped_positions(N, P, seed),
            "clustered": lambda: inputs.clustered_chain_positions(N, P, seed),
            "coincident": lambda: inputs.coincident_positions(N, P),
            "separated": lambda: inputs.separated_positions(N, P, seed)}[kind]()


def run(pos, beta, prec, recompute, box=0.0, want_M=False):
    N, P, _ = pos.shape
    eng = ExchangeEnergy(N, P, 1.0, inputs.omega_P(P, beta), beta, precision=prec, device="cuda:0",
                         box=box, recompute=recompute)
    V, F = eng.forces(torch.from_numpy(pos).cuda())
    eng.sync()
    Vf, Vb, _ = eng.potentials()
    M = eng.connection_probabilities().cpu().numpy() if want_M else None
    out = float(V.cpu()), F.cpu().numpy(), Vf, Vb, M
    eng.close()
    return out


def reference(pos, beta, box=0.0):
    wP = inputs.omega_P(pos.shape[1], beta)
    lib = oracle.float64 if pos.shape[0] < 128 else oracle.long_double
    VB, F, Vf, Vb, M = lib.fast_pimdb(pos, 1.0, wP, beta, full=True, **({"box": box} if box else {}))
    return float(VB), np.asarray(F, np.float64), np.asarray(Vf, np.float64), np.asarray(Vb, np.float64), M


def near(got, want, tol, beta):
    return abs(got - want) <= tol * max(abs(want), 1.0 / beta)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
@pytest.mark.parametrize("N,P,kind", [(1, 3, "trapped"), (5, 2, "clustered"), (33, 8, "trapped"),
                                      (100, 16, "clustered"), (300, 8, "separated"), (40, 4, "coincident"),
                                      (1024, 32, "trapped")])
def test_recompute_matches_oracle_and_stored_mode(prec, N, P, kind):
    beta = 1.3
    pos = gen(kind, N, P, 2000 + N)
    VB, F, Vf, Vb, M = reference(pos, beta)
    gV, gF, gVf, gVb, gM = run(pos, beta, prec, recompute=True, want_M=N <= 300)
    t = TOL[prec]
    assert near(gV, VB, t["v"], beta), (gV, VB)
    nF = np.linalg.norm(F)
    if nF > 0:
        assert np.linalg.norm(gF - F) <= t["f"] * nF
    else:
        assert np.abs(gF).max() <= 1e-12
    np.testing.assert_allclose(gVf, Vf, rtol=t["pot"], atol=t["pot"] / beta)
    np.testing.assert_allclose(gVb, Vb, rtol=t["pot"], atol=t["pot"] / beta)
    if gM is not None:
        np.testing.assert_allclose(gM, np.asarray(M, np.float64), rtol=0, atol=1e-10 if prec == "fp64" else 1e-5)
    sV, sF, sVf, sVb, _ = run(pos, beta, prec, recompute=False)
    assert gV == sV
    assert np.array_equal(gVf, sVf) and np.array_equal(gVb, sVb)
    if nF > 0:
        assert np.linalg.norm(gF - sF) <= 1e-13 * nF if prec != "mixed32" else 1e-6 * nF


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_recompute_in_a_periodic_box(prec):
    N, P, L, beta = 100, 8, 5.0, 1.0
    rng = np.random.default_rng(N)
    pos = np.mod(rng.uniform(0, L, (N, 1, 3)) + rng.normal(0, 0.4, (N, P, 3)), L)
    VB, F, *_ = reference(pos, beta, box=L)
    gV, gF, *_ = run(pos, beta, prec, recompute=True, box=L)
    t = TOL[prec]
    assert near(gV, VB, t["v"], beta)
    assert np.linalg.norm(gF - F) <= t["f"] * np.linalg.norm(F)


def load_referee(name):
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
def test_largest_n_against_the_long_double_referee(prec):
    """N = 16384, P = 4: above BPIMD_STORE_MAX_N, so nothing O(N^2) is stored."""
    ref = load_referee("referee_N16384_P4_trapped_seed13_beta1.txt")
    N, P, beta = int(ref["N"]), int(ref["P"]), ref["beta"]
    assert N == bpimd.BPIMD_MAX_N and N > bpimd.BPIMD_STORE_MAX_N
    pos = inputs.trapped_positions(N, P, int(ref["seed"]))
    gV, gF, gVf, gVb, _ = run(pos, beta, prec, recompute=False)
    t = TOL[prec]
    assert near(gV, ref["VB"], t["v"], beta), (gV, ref["VB"])
    idx = np.array(sorted(ref["F"]))
    want = np.array([ref["F"][i] for i in idx])
    got = gF.reshape(-1)[idx]
    assert np.linalg.norm(got - want) <= t["f"] * np.linalg.norm(want)
    for v, val in ref["VF"].items():
        assert near(gVf[v], val, t["pot"], beta), (v, gVf[v], val)
    for v, val in ref["VBW"].items():
        assert near(gVb[v], val, t["pot"], beta), (v, gVb[v], val)
