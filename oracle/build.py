"""Compile the oracle (plain C++17, CPU, FP64) into oracle/liblks_oracle.so.

Test infrastructure: the tests, the smoke check and the benchmark's CPU-baseline leg load it.
Portable host code only (no -march=native), so the same source builds on x86-64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lks_oracle.cpp")
LIB = os.path.join(HERE, "liblks_oracle.so")
# timing build: the same source with OpenMP over its independent per-node loops (bitwise the same
# results); built when the compiler supports -fopenmp
LIB_OMP = os.path.join(HERE, "liblks_oracle_omp.so")


def _compile(out: str, extra, verbose: bool) -> None:
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", *extra, "-o", out + ".tmp", SRC]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or not (os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        _compile(LIB, [], verbose)
    if force or not (os.path.exists(LIB_OMP) and os.path.getmtime(LIB_OMP) >= os.path.getmtime(SRC)):
        try:
            _compile(LIB_OMP, ["-fopenmp"], verbose)
        except (subprocess.CalledProcessError, OSError):
            pass  # no OpenMP: the single-threaded build alone
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
