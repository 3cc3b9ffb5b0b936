"""Compile the C oracle into oracle/liboracle.so with gcc.

Test infrastructure: the oracle is the CPU reference the tests compare the CUDA
library against.  Building it is part of ``__graft_entry__.build()``; nothing on
the product path links it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bpimd_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Build liboracle.so if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB) >= os.path.getmtime(os.path.join(HERE, "bpimd_oracle.h"))):
        return LIB
    # ISO C mode and -ffp-contract=off: no fused multiply-add contraction, so
    # the oracle rounds the same way on x86-64 and aarch64 hosts.
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
