"""Compile the oracle's C++ core into oracle/liboracle.so (g++, OpenMP when
available).  Test infrastructure: see oracle/__init__.py."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")


def stale() -> bool:
    return (not os.path.exists(LIB)) or os.path.getmtime(LIB) < os.path.getmtime(SRC)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", SRC, "-o", tmp]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:3] + extra + base[3:], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print("built", LIB, "with", extra or "no OpenMP")
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
