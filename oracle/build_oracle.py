"""Compile the oracle (plain C) into oracle/_liboracle.so with gcc.

Flags: -O2 -ffp-contract=off so that x86-64 and aarch64 builds round identically; OpenMP
over cells when the compiler supports it (results do not depend on the thread count: every
cell is computed independently and the only reduction, the CFL minimum, is order-free).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cteno_oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", SRC,
            "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
    sys.stderr.write(r.stderr)
    raise RuntimeError("oracle build failed")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
