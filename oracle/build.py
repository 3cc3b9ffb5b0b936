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
MD_SRC = os.path.join(HERE, "md_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_LD = os.path.join(HERE, "liboracle_ld.so")


def _fresh(lib):
    return os.path.exists(lib) and all(
        os.path.getmtime(lib) >= os.path.getmtime(p)
        for p in (SRC, MD_SRC, os.path.join(HERE, "bpimd_oracle.h")))


def _compile(lib, extra):
    # ISO C mode and -ffp-contract=off: no fused multiply-add contraction, so
    # the float64 oracle rounds the same way on x86-64 and aarch64 hosts.
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC"] + extra + ["-o", lib + ".tmp", SRC, MD_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)


def build(force: bool = False) -> str:
    """Build liboracle.so (float64) and liboracle_ld.so (long double referee)
    if missing or older than the source; returns the float64 library path."""
    if force or not _fresh(LIB):
        _compile(LIB, [])
    if force or not _fresh(LIB_LD):
        _compile(LIB_LD, ["-DORA_LONG_DOUBLE"])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
