"""FP64 CPU oracle for the bosonic exchange potential and forces.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2305_18025_gb300``), and the library never
imports it.

Contents
--------
* C routines (``bpimd_oracle.c``) reached through ctypes: Algorithm 1 stage by
  stage, Eq. Ek's direct cycle energies, Definition backward-potential,
  Algorithm 2 (the original O(P N^3) method with its differentiated forces).
* ``brute``: the definitions themselves -- the sum over all N! permutations with
  the representative map G (Definition representative-permutation and
  Definition forward-potential), and the sum over the 2^(N-1) representative
  permutations (appendix "Some Combinatorics of Permutations").
* ``harmonic``: the closed-form canonical energy of N non-interacting bosons in a
  harmonic trap at finite P.

Arrays use the layout of ``bpimd_oracle.h``: positions ``[N][P][3]`` float64,
``E[u-1, v-1] = E^{[u,v]}``, ``V[v] = V^{[1,v]}``, ``W[u-1] = V^{[u,N]}``,
``M[l-1, l'-1] = Pr[l -> l']``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

SHIFT_MIN_ALL = 0   # Eq. full-elong
SHIFT_TWO_TERM = 1  # Eq. original-elong


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i, d = ctypes.c_int, ctypes.c_double
        sig = {
            "ora_interior_energies": [i, i, d, d, dp, dp],
            "ora_cycle_energies": [i, i, d, d, dp, dp],
            "ora_cycle_energies_direct": [i, i, d, d, dp, dp],
            "ora_forward_potentials": [i, d, dp, i, dp],
            "ora_backward_potentials": [i, d, dp, i, dp],
            "ora_backward_potentials_definition": [i, d, dp, dp],
            "ora_connection_probabilities": [i, d, dp, dp, dp, dp],
            "ora_forces": [i, i, d, d, dp, dp, dp],
            "ora_fast_pimdb": [i, i, d, d, d, dp, dp, dp, dp, dp, dp],
            "ora_original_pimdb": [i, i, d, d, d, dp, dp, dp],
            "ora_expected_spring_energy": [i, i, d, d, dp, dp, dp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pos(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    if pos.ndim != 3 or pos.shape[2] != 3:
        raise ValueError("positions must be [N][P][3]")
    return pos


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments")


def interior_energies(pos, m, omega_P):
    pos = _pos(pos)
    N, P, _ = pos.shape
    out = np.empty(N)
    _check(_load().ora_interior_energies(N, P, m, omega_P, _p(pos), _p(out)), "interior_energies")
    return out


def cycle_energies(pos, m, omega_P, direct=False):
    """E[u-1, v-1] = E^{[u,v]} (u <= v); Algorithm 1's recurrence, or Eq. Ek if direct."""
    pos = _pos(pos)
    N, P, _ = pos.shape
    E = np.zeros((N, N))
    fn = _load().ora_cycle_energies_direct if direct else _load().ora_cycle_energies
    _check(fn(N, P, m, omega_P, _p(pos), _p(E)), "cycle_energies")
    return E


def forward_potentials(E, beta, shift=SHIFT_MIN_ALL):
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    V = np.empty(N + 1)
    _check(_load().ora_forward_potentials(N, beta, _p(E), shift, _p(V)), "forward_potentials")
    return V


def backward_potentials(E, beta, shift=SHIFT_MIN_ALL):
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    W = np.empty(N + 1)
    _check(_load().ora_backward_potentials(N, beta, _p(E), shift, _p(W)), "backward_potentials")
    return W


def backward_potentials_definition(E, beta):
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    W = np.empty(N + 1)
    _check(_load().ora_backward_potentials_definition(N, beta, _p(E), _p(W)),
           "backward_potentials_definition")
    return W


def connection_probabilities(E, V, W, beta):
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    V = np.ascontiguousarray(V, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    M = np.empty((N, N))
    _check(_load().ora_connection_probabilities(N, beta, _p(E), _p(V), _p(W), _p(M)),
           "connection_probabilities")
    return M


def forces(pos, M, m, omega_P):
    pos = _pos(pos)
    N, P, _ = pos.shape
    M = np.ascontiguousarray(M, dtype=np.float64)
    F = np.empty_like(pos)
    _check(_load().ora_forces(N, P, m, omega_P, _p(pos), _p(M), _p(F)), "forces")
    return F


def fast_pimdb(pos, m, omega_P, beta, full=False):
    """Algorithm 1.  Returns (V_B, F) or, with full=True, (V_B, F, V, W, M)."""
    pos = _pos(pos)
    N, P, _ = pos.shape
    F = np.empty_like(pos)
    VB = ctypes.c_double()
    V = np.empty(N + 1)
    W = np.empty(N + 1)
    M = np.empty((N, N)) if full else None
    rc = _load().ora_fast_pimdb(N, P, m, omega_P, beta, _p(pos), ctypes.byref(VB), _p(F),
                                _p(V), _p(W), _p(M) if full else None)
    _check(rc, "fast_pimdb")
    if full:
        return VB.value, F, V, W, M
    return VB.value, F


def original_pimdb(pos, m, omega_P, beta):
    """Algorithm 2 (O(P N^3)).  Returns (V_B, F)."""
    pos = _pos(pos)
    N, P, _ = pos.shape
    F = np.empty_like(pos)
    VB = ctypes.c_double()
    _check(_load().ora_original_pimdb(N, P, m, omega_P, beta, _p(pos), ctypes.byref(VB), _p(F)),
           "original_pimdb")
    return VB.value, F


def expected_spring_energy(pos, M, m, omega_P):
    pos = _pos(pos)
    N, P, _ = pos.shape
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = ctypes.c_double()
    _check(_load().ora_expected_spring_energy(N, P, m, omega_P, _p(pos), _p(M), ctypes.byref(out)),
           "expected_spring_energy")
    return out.value


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle.so")
