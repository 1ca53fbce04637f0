"""Compile the FP64 oracle (plain C + OpenMP) into oracle/liboracle.so.

Test infrastructure: built next to the library so that the tests, the smoke
check and the CPU-baseline leg of the benchmark can load it.
IEEE semantics are kept (no fast-math, no FMA contraction) because the
binary32 geometry decision value must follow its written operation order.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hlbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", LIB, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
