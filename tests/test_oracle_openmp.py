"""The OpenMP build of the oracle (used to time the CPU baseline on all host
cores) parallelises only loops whose iterations write disjoint outputs and
keeps every sum in order, so it must reproduce the single-thread oracle bit
for bit: the whole PCG residual history and the solution, on the matching
hierarchy with Cholesky, on the variable V-cycle with the PCG coarsest solve
and with smoothed prolongators (P and P^T through the parallel SpMV), with
several threads and a ragged last dot-product block."""

import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from synthetic import poisson3d, uniform01
oracle.use_openmp(sys.argv[2] == "1")
out = {"threads": oracle.threads()}
A = poisson3d(21, 19, 23)          # 9177 rows: dot products end in a ragged block
b = uniform01(5, A[0].size - 1)
for name, kw in (("v11", {}),
                 ("vmatch", dict(sweeps=3, smooth_sweeps=2, variable=True, coarse="pcg")),
                 ("smatch", dict(sweeps=3, smooth_sweeps=2, coarse="pcg", smoothed=True))):
    H = oracle.Hierarchy(A, **kw)
    x, info = oracle.pcg(A, b, tol=1e-10, hier=H, history=True,
                         beta_form=1 if kw else 0)
    out[name] = {"x": x.view(np.uint64).tolist(),
                 "res": np.asarray(info["res_hist"]).view(np.uint64).tolist(),
                 "it": info["iterations"]}
print(json.dumps(out))
"""


def _run(openmp, threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT, "1" if openmp else "0"],
                       capture_output=True, text=True, env=env, timeout=300, check=True)
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_openmp_oracle_gives_the_same_bits():
    plain = _run(False, 1)
    omp = _run(True, 4)
    assert plain["threads"] == 1
    assert omp["threads"] == 4
    for name in ("v11", "vmatch", "smatch"):
        assert omp[name]["it"] == plain[name]["it"] > 5
        assert omp[name]["res"] == plain[name]["res"]
        assert omp[name]["x"] == plain[name]["x"]
