"""Planted mistakes in the molecular-dynamics oracle must be caught by its pins.

Each mutant is oracle/md_oracle.c with one plausible slip: a generator
constant, the Box-Muller transform, a force or energy term, the minimum image,
the splitting of the BAOAB step, the thermostat's noise amplitude, or the
energy estimator.  It is compiled with the unchanged exchange oracle into a
temporary library.  The pin that should catch the slip is then run against it.
These pins are the ones in test_md_oracle_pins.py and test_pbc_oracle_pins.py,
written here as functions of the library: known answers, normal moments,
forces as minus the finite-difference gradient, central pair forces,
reversibility, second-order energy error, and equipartition with the
closed-form trapped-boson energy.  A test passes only if that pin fails on
the mutant, which shows the pin would not silently agree with such a
mistake.  Every pin also passes on the real oracle.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import build as oracle_build
from oracle import harmonic
from paper_2305_18025_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LJ = (10.22, 2.556, 2.5 * 2.556)  # eps, sigma, cutoff


# ------------------------------------------------------------------ the pins
def pin_philox(o):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    return all(o.philox4x32_10([int(x, 16) for x in r[0:4]], [int(x, 16) for x in r[4:6]])
               == [int(x, 16) for x in r[6:10]] for r in rows)


def pin_normals(o):
    z = o.thermostat_normals(seed=7, step=3, n=200_003)
    return (abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2 and abs((z ** 4).mean() - 3.0) < 6e-2
            and abs((z[:-1] * z[1:]).mean()) < 1e-2)


def pin_minus_gradient(o, omega0, pair, a=3.0, b=0.5, rc=0.0, box=0.0, spread=0.8, m=1.3):
    rng = np.random.default_rng(11)
    pos = rng.normal(0, spread, (5, 3, 3))
    if box:
        pos = rng.uniform(0, box, (5, 3, 3))
    U, F = o.external_forces(pos, m, omega0, pair, a, b, rc, box)
    h = 1e-6 * max(1.0, spread)
    for idx in [(0, 0, 0), (1, 2, 1), (4, 1, 2), (2, 0, 2), (3, 1, 0)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[idx] += h
        p2[idx] -= h
        fd = -(o.external_forces(p1, m, omega0, pair, a, b, rc, box)[0]
               - o.external_forces(p2, m, omega0, pair, a, b, rc, box)[0]) / (2 * h)
        if not abs(fd - F[idx]) < 1e-6 * max(1.0, abs(F[idx])):
            return False
    return True


def pin_gaussian_pair(o, box=0.0):
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, box, (4, 6, 3)) if box else rng.normal(0, 1.0, (4, 6, 3))
    _, Fp = o.external_forces(pos, 2.0, 0.0, 1, 3.0, 0.5 if not box else 1.5, 0.0, box)
    central = np.abs(Fp.sum(axis=0)).max() < 1e-12
    two = np.zeros((2, 2, 3))
    two[1, :, 0] = 0.8
    U2, _ = o.external_forces(two, 1.0, 0.0, 1, 3.0, 0.5)
    return central and abs(U2 - 3.0 * np.exp(-0.64 / 0.5)) < 1e-14


def _md_system(N, P, seed):
    rng = np.random.default_rng(seed)
    return inputs.trapped_positions(N, P, seed), rng.normal(0, 0.3, (N, P, 3))


def pin_reversible(o):
    N, P, beta = 4, 5, 1.5
    wP = inputs.omega_P(P, beta)
    pos, vel = _md_system(N, P, 1)
    kw = dict(omega0=1.0, pair_type=1, pair_a=3.0, pair_b=0.5)
    p1, v1, _ = o.md_run(pos, vel, 1.0, wP, beta, 0.02, 0.0, 50, **kw)
    p2, v2, _ = o.md_run(p1, -v1, 1.0, wP, beta, 0.02, 0.0, 50, **kw)
    return np.abs(p2 - pos).max() < 1e-10 and np.abs(v2 + vel).max() < 1e-10


def pin_second_order(o):
    N, P, beta = 3, 4, 1.0
    wP = inputs.omega_P(P, beta)
    pos, vel = _md_system(N, P, 2)
    kw = dict(omega0=1.0, pair_type=1, pair_a=3.0, pair_b=0.5)

    def H(p, v):
        VB, _ = o.fast_pimdb(p, 1.0, wP, beta)
        U, _ = o.external_forces(p, 1.0, 1.0, 1, 3.0, 0.5)
        return 0.5 * (v ** 2).sum() + VB + U

    H0 = H(pos, vel)
    errs = []
    for dt, n in [(0.02, 100), (0.01, 200)]:
        p, v, _ = o.md_run(pos, vel, 1.0, wP, beta, dt, 0.0, n, **kw)
        errs.append(abs(H(p, v) - H0))
    return errs[0] < 1e-3 * abs(H0) and 2.5 < errs[0] / errs[1] < 6.0


def pin_equipartition(o, nsamp=10000):
    """<KE> = 3NP/(2 beta) and <E_prim> = the closed-form trapped-boson energy,
    within four block standard errors (N = 2, P = 4, beta = 2)."""
    N, P, beta, dt, every, seed = 2, 4, 2.0, 0.1, 10, 8
    wP = inputs.omega_P(P, beta)
    rng = np.random.default_rng(seed)
    pos, vel = rng.normal(0, 0.7, (N, P, 3)), np.zeros((N, P, 3))
    pos, vel, _ = o.md_run(pos, vel, 1.0, wP, beta, dt, 1.0, 2000, seed=seed, step0=0, omega0=1.0)
    step, en = 2000, []
    for _ in range(nsamp):
        pos, vel, e = o.md_run(pos, vel, 1.0, wP, beta, dt, 1.0, every, seed=seed, step0=step, omega0=1.0)
        step += every
        en.append(e.copy())
    en = np.array(en)
    for col, exact in [(2, 1.5 * N * P / beta), (3, harmonic.mean_energy(N, P, beta, 1.0))]:
        b = en[:, col].reshape(50, -1).mean(axis=1)
        err = b.std(ddof=1) / np.sqrt(len(b))
        if not abs(b.mean() - exact) < 4 * err + 1e-3 * abs(exact):
            return False
    return True


# ---------------------------------------------------------------- the mutants
# name: (text in md_oracle.c, replacement, pin that must fail)
MUTANTS = {
    "philox_weyl_increment": ("k1 += W1;", "k1 += W0;", pin_philox),
    "philox_word_permutation": ("n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;",
                                "n1 = lo0, n2 = hi0 ^ c3 ^ k1, n3 = lo1;", pin_philox),
    "box_muller_same_angle": ("ra * sin(two_pi * u[1])", "ra * cos(two_pi * u[1])", pin_normals),
    "box_muller_radius": ("sqrt(-2.0 * log(u[0]))", "sqrt(-log(u[0]))", pin_normals),
    "trap_force_drops_one_over_P": ("for (int d = 0; d < 3; ++d) f[d] -= invP * kt * r[d];",
                                    "for (int d = 0; d < 3; ++d) f[d] -= kt * r[d];",
                                    lambda o: pin_minus_gradient(o, 1.0, 0)),
    "gaussian_force_sign": ("f[0] += invP * e * dx / (pb * pb);", "f[0] -= invP * e * dx / (pb * pb);",
                            lambda o: pin_minus_gradient(o, 0.0, 1)),
    "gaussian_energy_counts_pairs_twice": ("if (lp > l) U += invP * e;", "U += invP * e;",
                                           lambda o: pin_minus_gradient(o, 0.7, 1)),
    "lennard_jones_force_factor": ("invP * 24.0 * pa * (2.0 * s6 * s6 - s6) / r2",
                                   "invP * 12.0 * pa * (2.0 * s6 * s6 - s6) / r2",
                                   lambda o: pin_minus_gradient(o, 0.0, 2, *LJ, box=12.0, m=4.0026)),
    "minimum_image_floor": ("dz -= L * RINTR(dz / L);\n          }\n          const ora_real e = pa",
                            "dz -= L * floor(dz / L);\n          }\n          const ora_real e = pa",
                            lambda o: pin_gaussian_pair(o, box=4.0)),
    "baoab_first_kick_full_step": ("vel[i] += 0.5 * dt * F[i] / m;     /* B */",
                                   "vel[i] += dt * F[i] / m;     /* B */", pin_reversible),
    "baoab_drift_full_step": ("pos[i] += 0.5 * dt * vel[i];       /* A */\n      vel[i] = c1",
                              "pos[i] += dt * vel[i];       /* A */\n      vel[i] = c1", pin_second_order),
    "thermostat_noise_variance": ("SQRT((1.0 - c1 * c1) * kT / m)", "SQRT((1.0 - c1) * kT / m)",
                                  pin_equipartition),
    "primitive_estimator_spring_sign": ("3.0 * N * P / (2.0 * beta) - spring + ubar",
                                        "3.0 * N * P / (2.0 * beta) + spring + ubar", pin_equipartition),
}


def _oracle_from(lib_path, monkeypatch):
    """An oracle object over another library (the build step is not rerun)."""
    monkeypatch.setattr(oracle_build, "MUTANT_LIB", str(lib_path), raising=False)
    monkeypatch.setattr(oracle_build, "build", lambda *a, **k: oracle_build.LIB)
    return oracle._Oracle("MUTANT_LIB", np.float64, ctypes.c_double)


def _compile(d, md_source):
    (d / "md_oracle.c").write_text(md_source)
    shutil.copy(oracle_build.SRC, d / "bpimd_oracle.c")
    shutil.copy(os.path.join(os.path.dirname(oracle_build.SRC), "bpimd_oracle.h"), d / "bpimd_oracle.h")
    lib = d / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                    "-o", str(lib), str(d / "bpimd_oracle.c"), str(d / "md_oracle.c"), "-lm"], check=True)
    return lib


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_every_pin_holds_on_the_real_oracle(tmp_path, monkeypatch):
    lib = _compile(tmp_path, open(oracle_build.MD_SRC).read())
    o = _oracle_from(lib, monkeypatch)
    for name, (_, _, pin) in MUTANTS.items():
        assert pin(o), f"the pin used for {name} fails on the unmodified oracle"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_catches_md_mutant(tmp_path, monkeypatch, name):
    old, new, pin = MUTANTS[name]
    src = open(oracle_build.MD_SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = _compile(tmp_path, src.replace(old, new, 1))
    o = _oracle_from(lib, monkeypatch)
    assert not pin(o), f"mutant {name} was not detected by its pin"
