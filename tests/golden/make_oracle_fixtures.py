"""Writes tests/golden/oracle_poisson<side>.json from the CPU oracle only.

For the 7-point Poisson problem (Sec. 3) on side^3 cells with a uniform[0,1)
right-hand side from splitmix64 seed 2: the oracle's hierarchy (rows and
stored entries per level, operator complexity), PCG iteration count and
residuals to 1e-8 (x0 = 0, V(1,1), 2 matching sweeps, coarsest <= 200 rows).
The inputs are integer-exact on every platform, and the oracle is strict IEEE
FP64 without contraction, so these values hold on any machine.

usage: python tests/golden/make_oracle_fixtures.py 256 [128 ...]
"""

from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synthetic import poisson3d, uniform01  # noqa: E402


def make(side: int, tol: float = 1e-8, seed: int = 2) -> dict:
    A = poisson3d(side)
    n = side ** 3
    b = uniform01(seed, n)
    t0 = time.time()
    H = oracle.Hierarchy(A)
    t1 = time.time()
    x, info = oracle.pcg(A, b, tol=tol, maxit=500, hier=H, history=True)
    t2 = time.time()
    levels = [dict(n=H.level_n(l), nnz=H.level_nnz(l)) for l in range(H.levels)]
    return dict(
        problem="poisson3d", side=side, rhs="uniform01", seed=seed, tol=tol, sweeps=2,
        max_coarse=200, levels=levels, operator_complexity=H.operator_complexity(),
        iterations=info["iterations"], status=info["status"], relres=info["relres"],
        true_relres=info["true_relres"], res_hist=[float(v) for v in info["res_hist"]],
        oracle_setup_s=round(t1 - t0, 2), oracle_solve_s=round(t2 - t1, 2),
        oracle_threads=1)


if __name__ == "__main__":
    for arg in sys.argv[1:] or ["256"]:
        side = int(arg)
        d = make(side)
        path = os.path.join(HERE, "oracle_poisson%d.json" % side)
        with open(path, "w") as f:
            json.dump(d, f, indent=1)
        print(path, d["iterations"], d["operator_complexity"], d["oracle_setup_s"],
              d["oracle_solve_s"])
