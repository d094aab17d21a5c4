"""Compile the CPU oracle (plain C, FP64) into oracle/liboracle.so.

Test infrastructure: the oracle is built so that tests and the CPU-baseline
leg of the benchmark can run it; the product library never links it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ehc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

BASE_FLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11"]


def build(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".tmp{os.getpid()}"
    for omp in (["-fopenmp"], []):
        cmd = [cc, *BASE_FLAGS, *omp, SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
        if verbose:
            print(r.stderr, file=sys.stderr)
    raise RuntimeError(f"oracle build failed:\n{r.stderr}")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
