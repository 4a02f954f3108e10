"""Compiles the CPU oracle (test infrastructure) into oracle/liboracle.so."""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["amg_oracle.cpp", "mlp_oracle.cpp"]
TARGET = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(TARGET):
        return True
    t = os.path.getmtime(TARGET)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t
               for s in SOURCES if os.path.exists(os.path.join(HERE, s)))


def build(force: bool = False) -> str:
    if force or _stale():
        srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
        tmp = TARGET + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp] + srcs
        subprocess.run(cmd, check=True)
        os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
