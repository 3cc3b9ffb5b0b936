"""The device's powers of two against numpy's float64 exp2 (correctly rounded
to within an ulp on these arguments) and against the exact values of the
integer-argument cases, both by the integer-pipe fixed-point method
(pow2_fixed.cuh):
  * 2^(-x/2) with the exact double x double product of the float64 Gaussian
    pair force (pow2neg_dd with c = 1/2, an exact factor, so that numpy's
    argument is exact too) over x in [0, 2000], including the arguments at and
    next to multiples of 1/128: within 2 ulp, exactly 1 at x = 0 (the Gaussian
    self term relies on it);
  * 2^(-x) as for the float64 pair factors over x in [0, 1000]: within 2 ulp,
    exact on integers.
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


def test_exact_product_method_of_the_gaussian_within_two_ulp():
    x = 2.0 * arguments(+1)
    got = run(0, x)
    want = np.exp2(-0.5 * x)
    assert ulps(got, want).max() <= 2.0
    assert run(0, np.array([0.0]))[0] == 1.0  # exact at 0 (the Gaussian self term relies on it)


def test_integer_fixed_point_method_within_two_ulp():
    x = arguments(+1)
    got = run(1, x)
    want = np.exp2(-x)
    assert ulps(got, want).max() <= 2.0
    ints = np.arange(0, 1001, dtype=np.float64)
    np.testing.assert_array_equal(run(1, ints), np.exp2(-ints))
