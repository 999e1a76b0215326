"""Compile the FP64 oracle (hemeoracle.c) into oracle/libhemeoracle.so.

Test infrastructure only (see oracle/__init__.py).  Plain gcc, double
precision, no FMA contraction; OpenMP when the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hemeoracle.c")
LIB = os.path.join(HERE, "libhemeoracle.so")


def _compile(extra):
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off",
           "-fno-fast-math", *extra, SRC, "-o", LIB + ".tmp", "-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    r = _compile(["-fopenmp"])
    if r.returncode != 0:
        r = _compile([])
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
