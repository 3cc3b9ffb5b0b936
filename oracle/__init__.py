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
* ``long_double``: the same C routines compiled with long double arithmetic, a
  higher-precision referee for cases where float64 rounding of the oracle itself
  approaches the comparison tolerances.
* ``harmonic``: the closed-form canonical energy of N non-interacting bosons in a
  harmonic trap at finite P.
* molecular dynamics (``md_oracle.c``): Philox4x32-10, thermostat normals, the
  trap and Gaussian pair forces, and BAOAB Langevin steps with the primitive
  energy estimator.

Arrays use the layout of ``bpimd_oracle.h``: positions ``[N][P][3]`` float64,
``E[u-1, v-1] = E^{[u,v]}``, ``V[v] = V^{[1,v]}``, ``W[u-1] = V^{[u,N]}``,
``M[l-1, l'-1] = Pr[l -> l']``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SHIFT_MIN_ALL = 0   # Eq. full-elong
SHIFT_TWO_TERM = 1  # Eq. original-elong


class _Oracle:
    """The C routines for one floating-point type (float64 or long double)."""

    def __init__(self, path_attr, dtype, ctype):
        self._path_attr = path_attr
        self.dtype = dtype
        self._ctype = ctype
        self._lib = None

    def lib(self):
        if self._lib is None:
            _build.build()
            lib = ctypes.CDLL(getattr(_build, self._path_attr))
            rp = ctypes.POINTER(self._ctype)
            i, r = ctypes.c_int, self._ctype
            sig = {
                "ora_interior_energies": [i, i, r, r, rp, rp],
                "ora_cycle_energies": [i, i, r, r, rp, rp],
                "ora_cycle_energies_direct": [i, i, r, r, rp, rp],
                "ora_forward_potentials": [i, r, rp, i, rp],
                "ora_backward_potentials": [i, r, rp, i, rp],
                "ora_backward_potentials_definition": [i, r, rp, rp],
                "ora_connection_probabilities": [i, r, rp, rp, rp, rp],
                "ora_forces": [i, i, r, r, rp, rp, rp],
                "ora_fast_pimdb": [i, i, r, r, r, rp, rp, rp, rp, rp, rp],
                "ora_original_pimdb": [i, i, r, r, r, rp, rp, rp],
                "ora_expected_spring_energy": [i, i, r, r, rp, rp, rp],
                "ora_external_forces": [i, i, r, r, i, r, r, r, r, rp, rp, rp],
                "ora_md_run": [i, i, r, r, r, r, r, r, r, i, r, r, r, r, ctypes.c_uint64, ctypes.c_uint64,
                               i, rp, rp, rp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.ora_philox4x32_10.restype = None
            lib.ora_thermostat_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                                   ctypes.POINTER(ctypes.c_double)]
            lib.ora_thermostat_normals.restype = None
            lib.ora_set_box.argtypes = [self._ctype]
            lib.ora_set_box.restype = None
            lib.ora_set_noise_offset.argtypes = [ctypes.c_uint64]
            lib.ora_set_noise_offset.restype = None
            self._lib = lib
        return self._lib

    def _p(self, a):
        return None if a is None else a.ctypes.data_as(ctypes.POINTER(self._ctype))

    def _arr(self, a):
        return np.ascontiguousarray(a, dtype=self.dtype)

    def _pos(self, pos):
        pos = self._arr(pos)
        if pos.ndim != 3 or pos.shape[2] != 3:
            raise ValueError("positions must be [N][P][3]")
        return pos

    @staticmethod
    def _check(rc, name):
        if rc != 0:
            raise ValueError(f"{name}: invalid arguments")

    def interior_energies(self, pos, m, omega_P):
        pos = self._pos(pos)
        N, P, _ = pos.shape
        out = np.empty(N, dtype=self.dtype)
        self._check(self.lib().ora_interior_energies(N, P, m, omega_P, self._p(pos), self._p(out)),
                    "interior_energies")
        return out

    def cycle_energies(self, pos, m, omega_P, direct=False):
        """E[u-1, v-1] = E^{[u,v]} (u <= v); Algorithm 1's recurrence, or Eq. Ek if direct."""
        pos = self._pos(pos)
        N, P, _ = pos.shape
        E = np.zeros((N, N), dtype=self.dtype)
        fn = self.lib().ora_cycle_energies_direct if direct else self.lib().ora_cycle_energies
        self._check(fn(N, P, m, omega_P, self._p(pos), self._p(E)), "cycle_energies")
        return E

    def forward_potentials(self, E, beta, shift=SHIFT_MIN_ALL):
        E = self._arr(E)
        N = E.shape[0]
        V = np.empty(N + 1, dtype=self.dtype)
        self._check(self.lib().ora_forward_potentials(N, beta, self._p(E), shift, self._p(V)),
                    "forward_potentials")
        return V

    def backward_potentials(self, E, beta, shift=SHIFT_MIN_ALL):
        E = self._arr(E)
        N = E.shape[0]
        W = np.empty(N + 1, dtype=self.dtype)
        self._check(self.lib().ora_backward_potentials(N, beta, self._p(E), shift, self._p(W)),
                    "backward_potentials")
        return W

    def backward_potentials_definition(self, E, beta):
        E = self._arr(E)
        N = E.shape[0]
        W = np.empty(N + 1, dtype=self.dtype)
        self._check(self.lib().ora_backward_potentials_definition(N, beta, self._p(E), self._p(W)),
                    "backward_potentials_definition")
        return W

    def connection_probabilities(self, E, V, W, beta):
        E, V, W = self._arr(E), self._arr(V), self._arr(W)
        N = E.shape[0]
        M = np.empty((N, N), dtype=self.dtype)
        self._check(self.lib().ora_connection_probabilities(N, beta, self._p(E), self._p(V),
                                                            self._p(W), self._p(M)),
                    "connection_probabilities")
        return M

    def forces(self, pos, M, m, omega_P):
        pos = self._pos(pos)
        N, P, _ = pos.shape
        M = self._arr(M)
        F = np.empty_like(pos)
        self._check(self.lib().ora_forces(N, P, m, omega_P, self._p(pos), self._p(M), self._p(F)),
                    "forces")
        return F

    def set_box(self, L):
        """Periodic cubic box of side L for the following calls (0: open boundaries)."""
        self.lib().ora_set_box(float(L))

    def fast_pimdb(self, pos, m, omega_P, beta, full=False, box=0.0):
        """Algorithm 1.  Returns (V_B, F) or, with full=True, (V_B, F, V, W, M).
        box > 0: periodic cubic box, every spring by minimum image."""
        if box:
            self.set_box(box)
            try:
                return self.fast_pimdb(pos, m, omega_P, beta, full)
            finally:
                self.set_box(0.0)
        pos = self._pos(pos)
        N, P, _ = pos.shape
        F = np.empty_like(pos)
        VB = np.zeros(1, dtype=self.dtype)
        V = np.empty(N + 1, dtype=self.dtype)
        W = np.empty(N + 1, dtype=self.dtype)
        M = np.empty((N, N), dtype=self.dtype) if full else None
        rc = self.lib().ora_fast_pimdb(N, P, m, omega_P, beta, self._p(pos), self._p(VB),
                                       self._p(F), self._p(V), self._p(W), self._p(M))
        self._check(rc, "fast_pimdb")
        if full:
            return VB[0], F, V, W, M
        return VB[0], F

    def original_pimdb(self, pos, m, omega_P, beta, box=0.0):
        """Algorithm 2 (O(P N^3)).  Returns (V_B, F)."""
        if box:
            self.set_box(box)
            try:
                return self.original_pimdb(pos, m, omega_P, beta)
            finally:
                self.set_box(0.0)
        pos = self._pos(pos)
        N, P, _ = pos.shape
        F = np.empty_like(pos)
        VB = np.zeros(1, dtype=self.dtype)
        self._check(self.lib().ora_original_pimdb(N, P, m, omega_P, beta, self._p(pos),
                                                  self._p(VB), self._p(F)), "original_pimdb")
        return VB[0], F

    def expected_spring_energy(self, pos, M, m, omega_P):
        pos = self._pos(pos)
        N, P, _ = pos.shape
        M = self._arr(M)
        out = np.zeros(1, dtype=self.dtype)
        self._check(self.lib().ora_expected_spring_energy(N, P, m, omega_P, self._p(pos),
                                                          self._p(M), self._p(out)),
                    "expected_spring_energy")
        return out[0]

    # ------------------------------------------------ molecular dynamics
    def philox4x32_10(self, counter, key):
        """Philox4x32-10 block: four 32-bit counter words, two key words -> four words."""
        c = (ctypes.c_uint32 * 4)(*counter)
        k = (ctypes.c_uint32 * 2)(*key)
        o = (ctypes.c_uint32 * 4)()
        self.lib().ora_philox4x32_10(c, k, o)
        return [int(x) for x in o]

    def thermostat_normals(self, seed, step, n):
        z = np.empty(n, dtype=np.float64)
        self.lib().ora_thermostat_normals(seed, step, n, z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return z

    def external_forces(self, pos, m, omega0, pair_type=0, pair_a=0.0, pair_b=1.0, pair_rc=0.0, box=0.0):
        """(U-bar, -grad U-bar) of the trap and same-bead pair potential
        (pair_type 1 Gaussian g, s; 2 Lennard-Jones eps, sigma cut and shifted at pair_rc)."""
        pos = self._pos(pos)
        N, P, _ = pos.shape
        F = np.zeros_like(pos)
        U = np.zeros(1, dtype=self.dtype)
        self._check(self.lib().ora_external_forces(N, P, m, omega0, pair_type, pair_a, pair_b, pair_rc, box,
                                                   self._p(pos), self._p(F), self._p(U)),
                    "external_forces")
        return U[0], F

    def md_run(self, pos, vel, m, omega_P, beta, dt, gamma, nsteps, omega0=0.0, pair_type=0,
               pair_a=0.0, pair_b=1.0, kT=0.0, seed=0, step0=0, pair_rc=0.0, box=0.0, elem0=0):
        """nsteps BAOAB steps; returns (pos, vel, energies[4]) as new arrays.
        elem0: element offset of the thermostat counters (a replica at that
        offset of a packed batch; 0 for a single system)."""
        pos = self._pos(pos).copy()
        vel = self._arr(vel).copy()
        N, P, _ = pos.shape
        en = np.zeros(4, dtype=self.dtype)
        self.lib().ora_set_noise_offset(int(elem0))
        self._check(self.lib().ora_md_run(N, P, m, omega_P, beta, dt, gamma, kT, omega0, pair_type,
                                          pair_a, pair_b, pair_rc, box, seed, step0, nsteps, self._p(pos),
                                          self._p(vel), self._p(en)), "md_run")
        return pos, vel, en


#: float64 oracle (the default)
float64 = _Oracle("LIB", np.float64, ctypes.c_double)
#: the same routines in long double: the higher-precision referee
long_double = _Oracle("LIB_LD", np.longdouble, ctypes.c_longdouble)


def interior_energies(pos, m, omega_P):
    return float64.interior_energies(pos, m, omega_P)


def cycle_energies(pos, m, omega_P, direct=False):
    return float64.cycle_energies(pos, m, omega_P, direct)


def forward_potentials(E, beta, shift=SHIFT_MIN_ALL):
    return float64.forward_potentials(E, beta, shift)


def backward_potentials(E, beta, shift=SHIFT_MIN_ALL):
    return float64.backward_potentials(E, beta, shift)


def backward_potentials_definition(E, beta):
    return float64.backward_potentials_definition(E, beta)


def connection_probabilities(E, V, W, beta):
    return float64.connection_probabilities(E, V, W, beta)


def forces(pos, M, m, omega_P):
    return float64.forces(pos, M, m, omega_P)


def fast_pimdb(pos, m, omega_P, beta, full=False):
    """Algorithm 1 in float64.  Returns (V_B, F) or (V_B, F, V, W, M)."""
    out = float64.fast_pimdb(pos, m, omega_P, beta, full)
    return (float(out[0]),) + tuple(out[1:])


def original_pimdb(pos, m, omega_P, beta):
    VB, F = float64.original_pimdb(pos, m, omega_P, beta)
    return float(VB), F


def expected_spring_energy(pos, M, m, omega_P):
    return float(float64.expected_spring_energy(pos, M, m, omega_P))


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle.so")
