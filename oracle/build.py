"""Compile the FP64 oracle (test infrastructure) into ``oracle/liboracle.so``.

Plain g++, no GPU.  ``-ffp-contract=off`` keeps the arithmetic identical on
x86_64 and aarch64 hosts (GCC fuses multiply-adds by default on aarch64).
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["snh.cpp", "tet.cpp", "eigen.cpp", "sparse.cpp", "contact.cpp", "newton.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["ppn_oracle.h", "build.py"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    base = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-Wall", "-o", LIB + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES]
    # OpenMP over the independent element and SpMV-row loops when the compiler has it
    # (the results do not depend on it); otherwise a single-threaded build
    for extra in (["-fopenmp"], []):
        cmd = base + extra
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if subprocess.run(cmd).returncode == 0:
            break
    else:
        raise RuntimeError("g++ failed to build the oracle")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
