"""Write sampled long-double oracle outputs for the largest GPU parity case.

The float64 oracle's own rounding at N = 6912 (~1e-10 relative on forces, from
the shifted log-sum-exp of the Numerical Stability section accumulating
eps * |V| per step) is as large as the force tolerance, so the reference for
that case is the same oracle compiled in long double.  Running it takes tens
of seconds on x86-64 and much longer in software quad precision on aarch64,
so this script stores a seeded sample of its outputs.  It calls only oracle/.

Usage: python tests/golden/make_referee_samples.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2305_18025_gb300 import inputs  # noqa: E402

CASES = [
    # name, N, P, beta, generator, seed
    ("referee_N6912_P4_trapped_seed9_beta1.txt", 6912, 4, 1.0, "trapped", 9),
    # the largest N accepted (recompute mode; the oracle itself needs ~9 GB here)
    ("referee_N16384_P4_trapped_seed13_beta1.txt", 16384, 4, 1.0, "trapped", 13),
]
SAMPLES = 256


def main(only=None):
    for name, N, P, beta, gen, seed in CASES:
        if only and only not in name:
            continue
        pos = inputs.trapped_positions(N, P, seed)
        wP = inputs.omega_P(P, beta)
        VB, F, V, W, _ = oracle.long_double.fast_pimdb(pos, 1.0, wP, beta, full=True)
        rng = np.random.default_rng(12345)
        fidx = np.sort(rng.choice(F.size, size=SAMPLES, replace=False))
        # always include every exterior-bead component of a few particles
        ext = [((l * P + j) * 3 + d) for l in (0, 1, N // 2, N - 2, N - 1) for j in (0, P - 1) for d in range(3)]
        fidx = np.unique(np.concatenate([fidx, ext]))
        vidx = np.unique(np.concatenate([rng.choice(N + 1, size=64, replace=False), [0, 1, N - 1, N]]))
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
        with open(path, "w") as f:
            f.write("# Long-double run of the oracle (Algorithm 1, appendix Algorithm Pseudocode)\n")
            f.write(f"# inputs: paper_2305_18025_gb300.inputs.trapped_positions(N={N}, P={P}, seed={seed}),"
                    f" m=1, omega_P=sqrt(P)/beta, beta={beta}\n")
            f.write(f"# written by tests/golden/make_referee_samples.py; long double mantissa bits:"
                    f" {np.finfo(np.longdouble).nmant + 1}\n")
            f.write(f"N {N}\nP {P}\nbeta {beta!r}\nseed {seed}\n")
            f.write(f"VB {float(VB)!r}\n")
            f.write(f"FNORM {float(np.sqrt(np.sum(F.astype(np.float64) ** 2)))!r}\n")
            f.write(f"FMAX {float(np.abs(F).max())!r}\n")
            for i in fidx:
                f.write(f"F {int(i)} {float(F.reshape(-1)[i])!r}\n")
            for v in vidx:
                f.write(f"VF {int(v)} {float(V[v])!r}\n")
                f.write(f"VBW {int(v)} {float(W[v])!r}\n")
        print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
