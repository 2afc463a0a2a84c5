"""Compile the FP64 oracle (plain C) into oracle/liboracle.so with gcc.

Test infrastructure: the oracle is built so that tests and the benchmark's CPU
baseline can call it; nothing on the product path links it.
-ffp-contract=off keeps every a*b+c a separate multiply and add on both x86 and
Arm, so the oracle gives the same FP64 results on either machine.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fdtd_oracle.c")
SRC2 = os.path.join(HERE, "split_pml.c")
HDR = os.path.join(HERE, "fdtd_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in (SRC, SRC2, HDR))


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-Wall", "-Wno-unused-function", SRC, SRC2, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
