"""Writes tests/golden/oracle_poisson<side>.json from the CPU oracle only.

For the 7-point Poisson problem (Sec. 3) on side^3 cells with a uniform[0,1)
right-hand side from splitmix64 seed 2: the oracle's hierarchy (rows and
stored entries per level, operator complexity), PCG iteration count and
residuals to 1e-8 (x0 = 0, V(1,1), 2 matching sweeps, coarsest <= 200 rows),
and the final solution at X_SAMPLES rows (the first, the last, and rows drawn
from splitmix64 seed X_SAMPLE_SEED), so a GPU solve of the full problem can be
checked entry by entry without storing all of x.
The inputs are integer-exact on every platform, and the oracle is strict IEEE
FP64 without contraction, so these values hold on any machine.

usage: python tests/golden/make_oracle_fixtures.py 256 [128 ...]
"""

from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synthetic import poisson3d, uniform01  # noqa: E402


X_SAMPLES, X_SAMPLE_SEED = 64, 99


def sample_rows(n: int) -> list:
    """Sorted distinct rows: 0, n - 1 and X_SAMPLES - 2 uniform draws."""
    u = uniform01(X_SAMPLE_SEED, X_SAMPLES - 2)
    return sorted({0, n - 1, *[int(v * n) for v in u]})


def host_cpu() -> str:
    """CPU model of this host (for the recorded oracle timings)."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


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
    rows = sample_rows(n)
    return dict(
        problem="poisson3d", side=side, rhs="uniform01", seed=seed, tol=tol, sweeps=2,
        max_coarse=200, levels=levels, operator_complexity=H.operator_complexity(),
        iterations=info["iterations"], status=info["status"], relres=info["relres"],
        true_relres=info["true_relres"], res_hist=[float(v) for v in info["res_hist"]],
        x_rows=rows, x_values=[float(x[i]) for i in rows],
        oracle_setup_s=round(t1 - t0, 2), oracle_solve_s=round(t2 - t1, 2),
        oracle_threads=1, oracle_host=host_cpu(), oracle_host_cores=os.cpu_count())


if __name__ == "__main__":
    for arg in sys.argv[1:] or ["256", "128", "64", "32"]:
        side = int(arg)
        d = make(side)
        path = os.path.join(HERE, "oracle_poisson%d.json" % side)
        with open(path, "w") as f:
            json.dump(d, f, indent=1)
        print(path, d["iterations"], d["operator_complexity"], d["oracle_setup_s"],
              d["oracle_solve_s"])
