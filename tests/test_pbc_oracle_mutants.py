"""Planted mistakes in the exchange oracle's periodic box must be caught by the
box pins of test_pbc_oracle_pins.py.

Each mutant is oracle/bpimd_oracle.c with one slip in the minimum-image
springs, compiled with the unchanged MD oracle into a temporary library:
- a wrap by floor instead of round, still periodic but not the minimum image;
- the open-boundary form of the spring Laplacian inside a box;
- one axis of the squared spring length taken without its image.
The pin aimed at each slip must fail on the mutant and hold on the real
oracle.  The pins: open boundaries equal a very large box, lattice
translations of single beads change nothing, and the box forces equal minus
the finite-difference gradient.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import build as oracle_build
from paper_2305_18025_gb300 import inputs


def _wrapped_liquid(N, P, L, seed, spread=0.15):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, L, (N, 1, 3))
    return np.mod(centres + rng.normal(0, spread, (N, P, 3)), L)


def pin_open_equals_large_box(o):
    pos = inputs.trapped_positions(12, 6, seed=3)
    V0, F0 = o.fast_pimdb(pos, 1.0, 2.0, 1.1)
    V1, F1 = o.fast_pimdb(pos, 1.0, 2.0, 1.1, box=1000.0)
    return abs(V1 - V0) <= 1e-13 * abs(V0) and np.abs(F1 - F0).max() <= 1e-12 * np.abs(F0).max()


def pin_lattice_translation(o):
    L = 3.0
    pos = _wrapped_liquid(10, 5, L, seed=10)
    V0, F0 = o.fast_pimdb(pos, 1.0, 1.7, 0.8, box=L)
    shifted = pos + L * np.random.default_rng(1).integers(-2, 3, pos.shape)
    V1, F1 = o.fast_pimdb(shifted, 1.0, 1.7, 0.8, box=L)
    return abs(V1 - V0) <= 1e-12 * abs(V0) and np.abs(F1 - F0).max() <= 1e-11 * np.abs(F0).max()


def pin_box_minus_gradient(o):
    L = 3.0
    pos = _wrapped_liquid(8, 4, L, seed=5)
    _, F = o.fast_pimdb(pos, 1.0, 1.6, 1.0, box=L)
    h = 1e-6
    flat = pos.reshape(-1)
    for idx in inputs.random_coordinates(pos.shape, 16, seed=6):
        a, b = flat.copy(), flat.copy()
        a[idx] += h
        b[idx] -= h
        Va, _ = o.fast_pimdb(a.reshape(pos.shape), 1.0, 1.6, 1.0, box=L)
        Vb, _ = o.fast_pimdb(b.reshape(pos.shape), 1.0, 1.6, 1.0, box=L)
        if not abs(-(Va - Vb) / (2 * h) - F.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(F.reshape(-1)[idx])):
            return False
    return True


MUTANTS = {
    "minimum_image_by_floor": ("d - g_box * RINT(d / g_box)", "d - g_box * floor(d / g_box)",
                               pin_open_equals_large_box),
    "laplacian_open_form_in_box": ("return g_box > 0.0 ? mi1(r - a) + mi1(r - b) : 2.0 * r - a - b;",
                                   "return 2.0 * r - a - b;", pin_box_minus_gradient),
    "squared_length_drops_z_image": ("dz = mi1(a[2] - b[2]);", "dz = a[2] - b[2];", pin_lattice_translation),
}


def _library(d, exchange_source):
    (d / "bpimd_oracle.c").write_text(exchange_source)
    here = os.path.dirname(oracle_build.SRC)
    shutil.copy(os.path.join(here, "bpimd_oracle.h"), d / "bpimd_oracle.h")
    shutil.copy(oracle_build.MD_SRC, d / "md_oracle.c")
    lib = d / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                    "-o", str(lib), str(d / "bpimd_oracle.c"), str(d / "md_oracle.c"), "-lm"], check=True)
    return lib


def _oracle_from(lib_path, monkeypatch):
    monkeypatch.setattr(oracle_build, "MUTANT_LIB", str(lib_path), raising=False)
    monkeypatch.setattr(oracle_build, "build", lambda *a, **k: oracle_build.LIB)
    return oracle._Oracle("MUTANT_LIB", np.float64, ctypes.c_double)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_box_pins_hold_on_the_real_oracle(tmp_path, monkeypatch):
    o = _oracle_from(_library(tmp_path, open(oracle_build.SRC).read()), monkeypatch)
    for name, (_, _, pin) in MUTANTS.items():
        assert pin(o), f"the pin used for {name} fails on the unmodified oracle"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_box_pin_catches_mutant(tmp_path, monkeypatch, name):
    old, new, pin = MUTANTS[name]
    src = open(oracle_build.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    o = _oracle_from(_library(tmp_path, src.replace(old, new, 1)), monkeypatch)
    assert not pin(o), f"mutant {name} was not detected by its pin"
