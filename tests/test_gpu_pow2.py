"""The device's powers of two against numpy's float64 exp2 (correctly rounded
to within an ulp on these arguments) and against the exact values of the
integer-argument cases:
  * the float64 table method of the MD pair force (exp2_table.cuh, Tang's
    method, truncation below 3.6e-17) over y in [-1000, 0], including values at
    and next to the k/64 table boundaries: within 4 ulp;
  * the integer-pipe fixed-point method of the pair factors (pow2_fixed.cuh)
    over x in [0, 1000]: within 2 ulp, exact on integers.
"""
import numpy as np
import pytest
import torch

from paper_2305_18025_gb300 import bpimd

pytestmark = pytest.mark.gpu


def ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def run(method, x):
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    bpimd.bpimd_pow2_selftest(method, xt, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def arguments(sign):
    rng = np.random.default_rng(0)
    k = np.arange(-64000, 1) / 64.0  # every table boundary k/64 in [-1000, 0]
    near = np.concatenate([k, np.nextafter(k, -np.inf), np.nextafter(k, np.inf)])
    x = np.concatenate([near, rng.uniform(-1000, 0, 200000), -10.0 ** rng.uniform(-12, 3, 20000)])
    x = x[(x <= 0) & (x >= -1000)]
    return x if sign < 0 else -x


def test_float64_table_method_within_a_few_ulp():
    y = arguments(-1)
    got = run(0, y)
    want = np.exp2(y)
    assert ulps(got, want).max() <= 4.0
    assert run(0, np.array([0.0]))[0] == 1.0  # exact at 0 (the Gaussian self term relies on it)


def test_integer_fixed_point_method_within_two_ulp():
    x = arguments(+1)
    got = run(1, x)
    want = np.exp2(-x)
    assert ulps(got, want).max() <= 2.0
    ints = np.arange(0, 1001, dtype=np.float64)
    np.testing.assert_array_equal(run(1, ints), np.exp2(-ints))
