"""GPU checks of the autograd form of V^{[1,N]} (exchange_potential).

Its backward is the connection-probability force kernel (Lemma expected-force:
F = -grad V^{[1,N]}), so these tests compare pos.grad with
  * the O(P N^3) gradient of Algorithm 2 (the paper's original method, with its
    differentiated force recursion, in the oracle),
  * Algorithm 1 of the oracle,
  * central finite differences of the GPU's own V_B (h = 1e-5) at 32 seeded
    coordinates (the N = 64, P = 32 workload, beta in {0.5, 1, 2, 4}),
and check that the upstream gradient scales the result and that the only
tensor saved for backward is the [N][P][3] force (no O(N^2) state).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import inputs
from paper_2305_18025_gb300.exchange import ExchangeEnergy, exchange_potential

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _grad(pos_np, beta, prec="fp64", upstream=1.0):
    N, P, _ = pos_np.shape
    eng = ExchangeEnergy(N, P, 1.0, inputs.omega_P(P, beta), beta, precision=prec, device=DEV)
    x = torch.tensor(pos_np, device=DEV, requires_grad=True)
    V = exchange_potential(x, eng)
    (upstream * V).backward()
    torch.cuda.synchronize()
    out = float(V.detach().cpu()), x.grad.detach().cpu().numpy()
    eng.close()
    return out


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0, 4.0])
def test_gradient_matches_algorithm_2(beta):
    N, P = 64, 32
    pos = inputs.trapped_positions(N, P, seed=200)
    V, g = _grad(pos, beta)
    V2, F2 = oracle.original_pimdb(pos, 1.0, inputs.omega_P(P, beta), beta)
    assert abs(V - V2) <= 1e-12 * abs(V2) + 1e-12
    assert np.linalg.norm(g + F2) <= 1e-10 * np.linalg.norm(F2)
    assert np.abs(g + F2).max() <= 1e-10 * np.abs(F2).max()


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0, 4.0])
def test_gradient_matches_central_differences(beta):
    N, P = 64, 32
    wP = inputs.omega_P(P, beta)
    pos = inputs.trapped_positions(N, P, seed=201)
    _, g = _grad(pos, beta)
    eng = ExchangeEnergy(N, P, 1.0, wP, beta, precision="fp64", device=DEV)
    h = 1e-5
    flat = pos.reshape(-1)
    for idx in inputs.random_coordinates(pos.shape, 32, seed=4):
        vals = []
        for sgn in (1.0, -1.0):
            q = flat.copy()
            q[idx] += sgn * h
            V, _ = eng.forces(torch.tensor(q.reshape(pos.shape), device=DEV))
            vals.append(float(V.cpu()))
        fd = (vals[0] - vals[1]) / (2 * h)
        gi = g.reshape(-1)[idx]
        assert abs(fd - gi) <= 1e-6 * max(1.0, abs(gi)), (idx, fd, gi)
    eng.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5), ("mixed32", 1e-5)])
def test_gradient_matches_algorithm_1_and_scales(prec, tol):
    N, P, beta = 300, 16, 1.3
    pos = inputs.clustered_chain_positions(N, P, seed=202)
    _, F = oracle.long_double.fast_pimdb(pos, 1.0, inputs.omega_P(P, beta), beta)
    F = np.asarray(F, dtype=np.float64)
    _, g = _grad(pos, beta, prec, upstream=2.5)
    assert np.linalg.norm(g + 2.5 * F) <= tol * 2.5 * np.linalg.norm(F)


def test_backward_saves_only_the_force():
    N, P, beta = 40, 8, 1.0
    pos = inputs.trapped_positions(N, P, seed=203)
    eng = ExchangeEnergy(N, P, 1.0, inputs.omega_P(P, beta), beta, device=DEV)
    x = torch.tensor(pos, device=DEV, requires_grad=True)
    V = exchange_potential(x, eng)
    saved = V.grad_fn.saved_tensors
    assert len(saved) == 1 and tuple(saved[0].shape) == (N, P, 3)
    V.backward()
    assert x.grad.shape == x.shape
    eng.close()
