"""Compiles the CPU oracle (test infrastructure) into oracle/liboracle.so, and
on request the same sources with OpenMP into oracle/liboracle_omp.so (its
parallel row loops give the same bits; used only to time the CPU baseline on
all host cores)."""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["amg_oracle.cpp", "mlp_oracle.cpp"]
TARGET = os.path.join(HERE, "liboracle.so")
TARGET_OMP = os.path.join(HERE, "liboracle_omp.so")


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t
               for s in SOURCES if os.path.exists(os.path.join(HERE, s)))


def build(force: bool = False, openmp: bool = False) -> str:
    target = TARGET_OMP if openmp else TARGET
    if force or _stale(target):
        srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
        tmp = target + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp] + (["-fopenmp"] if openmp else []) + srcs
        subprocess.run(cmd, check=True)
        os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, openmp="--openmp" in sys.argv))
