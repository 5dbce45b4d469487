"""Compile the oracle's plain-C direct sums (``bs_direct.c``) into a shared object.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Flags: -O2, OpenMP over
the outer target loop, and ``-ffp-contract=off`` so that no fused multiply-add
is introduced: the x86 build host and the Arm GPU host then round identically.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bs_direct.c")
LIB = os.path.join(HERE, "libbsdirect.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
