"""Pins of the integer-pipe power of two (csrc/pow2_fixed.cuh) on the CPU.

The header compiles for the host too (its 64 x 64-bit high products through
__int128), so the exact code path of the device is checked here against
2^(-x) to 50 digits (mpmath): Tang's table method in 64-bit fixed point must
be within one float64 rounding (2^-53 relative, plus the 2^-60 of the
polynomial and table), for double arguments and for the exact product of a
float32 and a double.  Arguments cover the table boundaries j/256, tiny and
large x, and the cut at 2^28 (read as zero by the recursions).
"""
import os
import struct
import subprocess
import tempfile

import numpy as np
import pytest
from mpmath import mp, mpf, power

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_2305_18025_gb300", "csrc", "pow2_fixed.cuh")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "%s"
int main() {
  char kind[8];
  double x, c;
  float a;
  while (std::scanf("%%7s", kind) == 1) {
    bpimd::pow2fx::mexp r;
    if (kind[0] == 'p') {
      unsigned long long b1, b2;
      std::scanf("%%llx %%llx", &b1, &b2);
      std::memcpy(&x, &b1, 8);
      std::memcpy(&c, &b2, 8);
      r = bpimd::pow2fx::pow2neg_dd(x, c, bpimd::pow2fx::T63);
    } else if (kind[0] == 'd') {
      unsigned long long b;
      std::scanf("%%llx", &b);
      std::memcpy(&x, &b, 8);
      r = bpimd::pow2fx::pow2neg(x, bpimd::pow2fx::T63);
    } else {
      unsigned ab;
      unsigned long long cb;
      std::scanf("%%x %%llx", &ab, &cb);
      std::memcpy(&a, &ab, 4);
      std::memcpy(&c, &cb, 8);
      r = bpimd::pow2fx::pow2neg_fd(a, c, bpimd::pow2fx::T63);
    }
    unsigned long long mb;
    std::memcpy(&mb, &r.m, 8);
    std::printf("%%llx %%d\n", mb, r.e);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("pow2")
    src = d / "drv.cpp"
    src.write_text(DRIVER % HDR)
    out = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(out), str(src)], check=True)
    return str(out)


def run(exe, lines):
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    res = []
    for ln in r.stdout.split("\n"):
        if ln.strip():
            mb, e = ln.split()
            m = struct.unpack("<d", struct.pack("<Q", int(mb, 16)))[0]
            res.append((m, int(e)))
    return res


def dbits(x):
    return "%x" % struct.unpack("<Q", struct.pack("<d", x))[0]


def fbits(a):
    return "%x" % struct.unpack("<I", struct.pack("<f", a))[0]


def rel_err(m, e, exact):
    mp.dps = 50
    return abs(mpf(m) * power(2, e) - exact) / exact


def test_double_arguments_within_one_rounding(exe):
    mp.dps = 50
    rng = np.random.default_rng(0)
    xs = [0.0, 1e-300, 2.0 ** -70, 1e-12, 0.5, 1.0, 2.0, 3.999999999, 1023.75, 2.0 ** 27 - 0.25]
    xs += [j / 256 + d for j in range(256) for d in (0.0, 1e-17, -1e-17) if j / 256 + d >= 0]
    xs += list(rng.uniform(0, 1, 300)) + list(rng.uniform(0, 60, 300)) + list(10 ** rng.uniform(-8, 8, 300))
    got = run(exe, ["d " + dbits(float(x)) for x in xs])
    worst = 0.0
    for x, (m, e) in zip(xs, got):
        assert 1.0 <= m < 2.0
        exact = power(2, -mpf(float(x)))
        worst = max(worst, float(rel_err(m, e, exact)))
    assert worst <= 1.2 * 2.0 ** -53, worst


def test_float_times_double_is_exact_before_the_power(exe):
    """x = a * c is formed from the float32 a and double c without rounding
    to float64 first: the result matches 2^(-a c) of the exact product."""
    mp.dps = 50
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 30, 500).astype(np.float32)
    c = -np.log(rng.uniform(0.01, 1, 500)) * 7.3
    lines = ["f " + fbits(float(ai)) + " " + dbits(float(ci)) for ai, ci in zip(a, c)]
    worst = 0.0
    for ai, ci, (m, e) in zip(a, c, run(exe, lines)):
        exact = power(2, -(mpf(float(ai)) * mpf(float(ci))))
        worst = max(worst, float(rel_err(m, e, exact)))
    assert worst <= 1.2 * 2.0 ** -53, worst


def test_large_arguments_read_as_zero_and_zero_as_one(exe):
    got = run(exe, ["d " + dbits(2.0 ** 28), "d " + dbits(1e300), "d " + dbits(0.0), "f " + fbits(0.0) + " " + dbits(3.0)])
    assert got[0] == (1.0, -(1 << 28)) and got[1] == (1.0, -(1 << 28))
    assert got[2] == (1.0, 0) and got[3] == (1.0, 0)


def test_integer_arguments_are_exact_powers(exe):
    got = run(exe, ["d " + dbits(float(k)) for k in range(0, 2000, 7)])
    for k, (m, e) in zip(range(0, 2000, 7), got):
        assert (m, e) == (1.0, -k)


def test_double_times_double_is_exact_before_the_power(exe):
    """x = a * c for two doubles, the 106-bit product truncated to 64 bits on
    the integer pipe (the float64 path of the pair factors)."""
    mp.dps = 50
    rng = np.random.default_rng(2)
    a = rng.uniform(0, 30, 500) ** 2
    c = -np.log(rng.uniform(0.01, 1, 500)) * 3.1
    lines = ["p " + dbits(float(ai)) + " " + dbits(float(ci)) for ai, ci in zip(a, c)]
    worst = 0.0
    for ai, ci, (m, e) in zip(a, c, run(exe, lines)):
        exact = power(2, -(mpf(float(ai)) * mpf(float(ci))))
        worst = max(worst, float(rel_err(m, e, exact)))
    assert worst <= 1.2 * 2.0 ** -53, worst
