"""Write pow2_table.h: T[j] = 2^(-j/256) as 64-bit fixed-point integers
(value T[j] / 2^63, rounded to nearest), j = 0..255, and ln 2 as a 64-bit
fraction (ln 2 * 2^64).  The constants are computed to 60 significant digits
with mpmath; rerun after editing nothing but this script:

    python paper_2305_18025_gb300/csrc/gen_pow2_table.py
"""
import os

from mpmath import mp, mpf, log, power, nint

mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    rows = []
    for j in range(256):
        v = int(nint(power(2, mpf(-j) / 256) * mpf(2) ** 63))
        assert 0 < v <= 2 ** 63
        rows.append(v)
    ln2 = int(nint(log(2) * mpf(2) ** 64))
    lines = ["// Generated by gen_pow2_table.py (mpmath, 60 digits): do not edit.",
             "// POW2_T63[j] = round(2^(-j/256) * 2^63), j = 0..255; LN2_Q64 = round(ln 2 * 2^64).",
             "#pragma once",
             f"#define BPIMD_LN2_Q64 0x{ln2:016X}ull",
             "#define BPIMD_POW2_T63_INIT \\"]
    for k in range(0, 256, 4):
        chunk = ", ".join(f"0x{v:016X}ull" for v in rows[k:k + 4])
        lines.append(f"  {chunk}," + " \\" if k + 4 < 256 else f"  {chunk}")
    lines.append("")
    with open(os.path.join(HERE, "pow2_table.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
