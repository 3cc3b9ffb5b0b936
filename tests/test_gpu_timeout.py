"""The error path of the recursions' bounded hand-off waits (BPIMD_ERR_TIMEOUT).

The CTAs of a recursion cluster hand results to one another through
shared-memory mbarriers, and every such wait gives up after one second of the
GPU's global timer.  BPIMD_FLAG_TEST_TIMEOUT makes the forward recursion wait
first for a hand-off that nothing makes, so the wait runs out on purpose.  No
fault or trap is involved: the waiting CTA records the expiry in the device
status word and stops waiting and handing off, the other CTAs' waits then run
out the same way, and every kernel reaches its end.  These tests check that
the host sees BPIMD_ERR_TIMEOUT, that the status is cleared once reported, and
that the process's CUDA context and a normal context afterwards still give
results that match the oracle.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2305_18025_gb300 import bpimd, inputs

pytestmark = pytest.mark.gpu


def _ctx(N, P, beta, prec, flags, stream):
    cfg = bpimd.make_config(N, P, 1.0, inputs.omega_P(P, beta), beta, bpimd.PRECISIONS[prec], flags=flags)
    return bpimd.bpimd_create(cfg, stream)


@pytest.mark.parametrize("N", [100, 1024])
def test_expired_wait_reports_timeout_and_the_gpu_stays_usable(N):
    P, beta, prec = 8, 1.0, "mixed"
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    pos = torch.from_numpy(inputs.trapped_positions(N, P, seed=31)).to(dev)
    F = torch.empty_like(pos)
    V = torch.empty((), dtype=torch.float64, device=dev)
    ctx = _ctx(N, P, beta, prec, bpimd.BPIMD_FLAG_TEST_TIMEOUT, stream)
    try:
        t0 = time.time()
        bpimd.bpimd_exchange_energy_forces(ctx, pos, V, F)
        rc = bpimd.load().bpimd_sync(ctx)
        elapsed = time.time() - t0
        assert rc == bpimd.BPIMD_ERR_TIMEOUT, bpimd.bpimd_status_string(rc)
        assert 0.5 < elapsed < 30.0, elapsed  # the waits give up after about a second
        assert bpimd.load().bpimd_sync(ctx) == bpimd.BPIMD_OK  # reported once, then cleared
    finally:
        bpimd.bpimd_destroy(ctx)
    # the same process, a normal context: correct results
    ctx = _ctx(N, P, beta, prec, 0, stream)
    try:
        bpimd.bpimd_exchange_energy_forces(ctx, pos, V, F)
        assert bpimd.load().bpimd_sync(ctx) == bpimd.BPIMD_OK
        ref = oracle.long_double if N >= 128 else oracle.float64
        VB, Fo = ref.fast_pimdb(pos.cpu().numpy(), 1.0, inputs.omega_P(P, beta), beta)
        assert abs(float(V.cpu()) - VB) <= 1e-6 * abs(VB)
        Fg = F.cpu().numpy()
        assert np.sqrt(np.mean((Fg - Fo) ** 2)) <= 1e-5 * np.sqrt(np.mean(Fo ** 2))
    finally:
        bpimd.bpimd_destroy(ctx)
