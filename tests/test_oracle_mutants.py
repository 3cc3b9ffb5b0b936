"""Planted mistakes in the oracle must be caught by its pins.

Each mutant is the oracle's C source with one plausible slip (a flipped sign, a
dropped term, a shifted index, a wrong sum limit), compiled on the CPU into a
temporary library.  The mutant's Algorithm 1 result is compared with the
brute-force definitions (sum over all permutations / over representatives); the
test passes only if every mutant disagrees.  This shows the pins would fail on
such a mistake rather than silently agreeing with it.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import brute
from paper_2305_18025_gb300 import inputs

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTANTS = {
    "step_sign_of_removed_spring": (
        "E[EIDX(N, u + 1, v)]\n                         - half_k",
        "E[EIDX(N, u + 1, v)]\n                         + half_k"),
    "step_drops_interior_energy": (
        "+ Eint[u - 1]\n", "\n"),
    "forward_drops_one_over_v": (
        "V[v] = Et - (1.0 / beta) * LOG(s / (ora_real)v);",
        "V[v] = Et - (1.0 / beta) * LOG(s);"),
    "backward_weight_one_over_u": (
        "s += (1.0 / (ora_real)l) * EXP(-beta * (E[EIDX(N, u, l)] + W[l] - Et));",
        "s += (1.0 / (ora_real)u) * EXP(-beta * (E[EIDX(N, u, l)] + W[l] - Et));"),
    "close_cycle_shifted_backward_index": (
        "EXP(-beta * (V[lp - 1] + E[EIDX(N, lp, l)] + W[l] - VN));",
        "EXP(-beta * (V[lp - 1] + E[EIDX(N, lp, l)] + W[l - 1] - VN));"),
    "direct_link_sign": (
        "-EXPM1(-beta * (V[l] + W[l] - VN))", "EXPM1(-beta * (V[l] + W[l] - VN))"),
    "bead1_force_wrong_neighbour_bead": (
        "BEAD(pos, P, l, 2)[d], BEAD(pos, P, lp, P)[d]);", "BEAD(pos, P, l, 2)[d], BEAD(pos, P, lp, 1)[d]);"),
    "beadP_force_drops_superdiagonal": (
        "int hi = l + 1 > N ? N : l + 1;", "int hi = l;"),
    "transposed_probability_in_bead1": (
        "ora_real pr = M[EIDX(N, lp, l)];", "ora_real pr = M[EIDX(N, l, lp)];"),
    "interior_force_sign": (
        "BEAD(F, P, l, j)[d] = -k * lap1(", "BEAD(F, P, l, j)[d] = k * lap1("),
    "base_case_drops_closing_spring": (
        "E[EIDX(N, v, v)] = Eint[v - 1] + half_k * sqdist(BEAD(pos, P, v, P), BEAD(pos, P, v, 1));",
        "E[EIDX(N, v, v)] = Eint[v - 1];"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(os.path.join(ORACLE_DIR, "bpimd_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(ORACLE_DIR, "bpimd_oracle.h"), d / "bpimd_oracle.h")
    (d / "bpimd_oracle.c").write_text(src.replace(old, new, 1))
    lib = d / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                    "-o", str(lib), str(d / "bpimd_oracle.c"), "-lm"], check=True)
    return ctypes.CDLL(str(lib))


def _run(lib, pos, m, w, beta):
    N, P, _ = pos.shape
    dp = ctypes.POINTER(ctypes.c_double)
    fn = lib.ora_fast_pimdb
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   ctypes.c_double, dp, dp, dp, dp, dp, dp]
    fn.restype = ctypes.c_int
    F = np.empty_like(pos)
    M = np.empty((N, N))
    V = np.empty(N + 1)
    W = np.empty(N + 1)
    VB = ctypes.c_double()
    p = lambda a: a.ctypes.data_as(dp)
    assert fn(N, P, m, w, beta, p(pos), ctypes.byref(VB), p(F), p(V), p(W), p(M)) == 0
    return VB.value, F, M


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_brute_force_pin_catches_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    N, P, beta = 5, 3, 1.1
    pos = inputs.clustered_chain_positions(N, P, seed=77)
    m, w = 1.0, inputs.omega_P(P, beta)
    Vb, Fb, Mb = brute.potential_by_permutations(pos, m, w, beta)
    VB, F, M = _run(lib, pos, m, w, beta)
    same = (abs(VB - Vb) <= 1e-12 * abs(Vb)
            and np.allclose(F, Fb, rtol=1e-10, atol=1e-10 * np.abs(Fb).max())
            and np.allclose(M, Mb, rtol=1e-10, atol=1e-13))
    assert not same, f"mutant {name} was not detected by the brute-force pin"
