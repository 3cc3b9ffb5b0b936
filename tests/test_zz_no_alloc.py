"""The allocation-free entry point against the context-based one.

bpimd_exchange_energy_forces_noalloc serves callers that cannot allocate device
memory when they evaluate (their memory manager owns every device allocation,
or they may not call cudaMalloc/cudaFree, which can synchronise the device).
It must give the same V_B and forces as bpimd_exchange_energy_forces, within
the tolerances of the parity tests, on consecutive calls that share its fixed
scratch array.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2305_18025_gb300 import bpimd, inputs
from paper_2305_18025_gb300.exchange import ExchangeEnergy

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-12, 1e-10), "mixed": (1e-6, 1e-5), "mixed32": (1e-6, 1e-5)}


def with_context(pos, beta, prec):
    N, P, _ = pos.shape
    eng = ExchangeEnergy(N, P, 1.0, inputs.omega_P(P, beta), beta, precision=prec, device="cuda:0")
    V, F = eng.forces(pos)
    eng.sync()
    out = float(V.item()), F.clone()
    eng.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_noalloc_matches_context_entry_point_on_consecutive_calls(prec):
    beta = 1.0
    cases = [(bpimd.BPIMD_NOALLOC_MAX_N, 8, 11), (100, 16, 12)]  # largest size, then a smaller one
    stream = torch.cuda.current_stream()
    for N, P, seed in cases:
        pos = torch.from_numpy(inputs.trapped_positions(N, P, seed)).cuda()
        V_ref, F_ref = with_context(pos, beta, prec)
        cfg = bpimd.make_config(N, P, 1.0, inputs.omega_P(P, beta), beta,
                                bpimd.PRECISIONS[prec])
        for _ in range(2):  # two calls in a row share the scratch array
            V = torch.full((), float("nan"), dtype=torch.float64, device="cuda:0")
            F = torch.full_like(pos, float("nan"))
            bpimd.bpimd_exchange_energy_forces_noalloc(cfg, pos, V, F, stream)
            torch.cuda.synchronize()
            vt, ft = TOL[prec]
            assert abs(V.item() - V_ref) <= vt * abs(V_ref)
            assert torch.linalg.norm(F - F_ref).item() <= ft * torch.linalg.norm(F_ref).item()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    N, P = bpimd.BPIMD_NOALLOC_MAX_N + 1, 4
    pos = torch.zeros((N, P, 3), dtype=torch.float64, device="cuda:0")
    F = torch.empty_like(pos)
    cfg = bpimd.make_config(N, P, 1.0, 2.0, 1.0)
    with pytest.raises(bpimd.BpimdError) as ei:
        bpimd.bpimd_exchange_energy_forces_noalloc(cfg, pos, None, F)
    assert ei.value.status == bpimd.BPIMD_ERR_SIZE


FIRST_CALL_SCRIPT = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2305_18025_gb300 import bpimd, inputs
from paper_2305_18025_gb300.exchange import ExchangeEnergy
N, P, beta = 96, 8, 1.0
pos = torch.from_numpy(inputs.trapped_positions(N, P, 21)).cuda()
cfg = bpimd.make_config(N, P, 1.0, inputs.omega_P(P, beta), beta, {prec})
V = torch.full((), float("nan"), dtype=torch.float64, device="cuda:0")
F = torch.full_like(pos, float("nan"))
# the first library call of this process: symbol lookup and recursion set-up
bpimd.bpimd_exchange_energy_forces_noalloc(cfg, pos, V, F, torch.cuda.current_stream())
torch.cuda.synchronize()
eng = ExchangeEnergy(N, P, 1.0, inputs.omega_P(P, beta), beta, precision={name!r}, device="cuda:0")
Vr, Fr = eng.forces(pos)
eng.sync()
dv = abs(V.item() - Vr.item()) / abs(Vr.item())
df = (torch.linalg.norm(F - Fr) / torch.linalg.norm(Fr)).item()
print(dv, df)
"""


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed32"])
def test_noalloc_as_the_first_call_of_a_fresh_process(prec):
    """A caller whose very first library call is the allocation-free entry
    point (no context exists yet, so the scratch address and the recursion
    kernels are set up inside that call) gets the context entry point's result."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = FIRST_CALL_SCRIPT.format(root=root, name=prec, prec=bpimd.PRECISIONS[prec])
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    dv, df = (float(x) for x in r.stdout.split()[-2:])
    vt, ft = TOL[prec]
    assert dv <= vt and df <= ft, (dv, df)


def test_noalloc_without_a_V_B_output():
    """V_B may be NULL: the forces are still written."""
    N, P, beta = 64, 8, 1.0
    pos = torch.from_numpy(inputs.trapped_positions(N, P, 22)).cuda()
    _, F_ref = with_context(pos, beta, "fp64")
    cfg = bpimd.make_config(N, P, 1.0, inputs.omega_P(P, beta), beta, bpimd.BPIMD_FP64)
    F = torch.full_like(pos, float("nan"))
    bpimd.bpimd_exchange_energy_forces_noalloc(cfg, pos, None, F, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.linalg.norm(F - F_ref).item() <= 1e-10 * torch.linalg.norm(F_ref).item()
