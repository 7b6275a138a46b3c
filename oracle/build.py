"""Compile the C oracle into oracle/_mclu_oracle.so (test infrastructure only).

Flags: binary64 round-to-nearest, no contraction of a*b+c into FMA
(-ffp-contract=off; fma() is only called explicitly), no fast-math, OpenMP for
outer loops.  Portable host code: no -march, no intrinsics.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mclu_oracle.c")
LIB = os.path.join(HERE, "_mclu_oracle.so")

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]


def build_oracle(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
