"""The shared-memory ring streams (bulk copies into per-warp stages) against
the per-lane-load kernels and the oracle.

Per row both forms run the same FMAs in the same order, so V-cycles (no dot
products) agree bit for bit; PCG's dot products are summed in another order
(the ring kernels use another grid), so its iterates agree to rounding.
Cases cover a ragged last slice (rows not a multiple of 32), several slices
per warp, FP64 and FP32 hierarchies (the ring's kernels), FP32 with BF16
values from level 2 (per-lane kernels on both sides there), and a matrix
whose widest slice does not fit the ring (the per-lane kernels run).
"""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import random_spd_graph

pytestmark = pytest.mark.gpu


def _np(t):
    return t.cpu().numpy()


CASES = {
    "poisson37x11x23": lambda: poisson3d(37, 11, 23),  # 9,361 rows: ragged last slice
    "poisson48": lambda: poisson3d(48),
    "diffusion40": lambda: diffusion3d(np.exp(gaussian_field((40, 36, 33), 2.0, 4.0, 17))),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [dict(precision="f64"), dict(precision="f32"),
                                  dict(precision="f32", bf16_from_level=2)])
def test_ring_vcycle_bitwise(amg, case, prec):
    A = CASES[case]()
    n = len(A[0]) - 1
    Ad = amg.csr_to_device(A)
    r = torch.as_tensor(uniform01(21, n), device="cuda")
    H1 = amg.Hierarchy(*Ad, stream_ring=1, **prec)
    H0 = amg.Hierarchy(*Ad, stream_ring=0, **prec)
    assert torch.equal(H1.vcycle(r), H0.vcycle(r))
    assert torch.equal(H1.spmv(r), H0.spmv(r))


@pytest.mark.parametrize("case", sorted(CASES))
def test_ring_pcg_matches_oracle(amg, orc, case):
    A = CASES[case]()
    n = len(A[0]) - 1
    Ad = amg.csr_to_device(A)
    b = uniform01(22, n)
    H1 = amg.Hierarchy(*Ad, stream_ring=1)
    H0 = amg.Hierarchy(*Ad, stream_ring=0)
    bt = torch.as_tensor(b, device="cuda")
    x1, i1 = H1.pcg(bt, tol=1e-10, x_history=True)
    x0, i0 = H0.pcg(bt, tol=1e-10)
    assert i1["status"] == 0 and abs(i1["iterations"] - i0["iterations"]) <= 1
    xo, io = orc.pcg(A, b, tol=1e-10, hier=orc.Hierarchy(A), x_history=True)
    assert abs(i1["iterations"] - io["iterations"]) <= 1
    # every iterate against the oracle's, to 1e-12 relative
    xh = _np(i1["x_hist"])
    for k in range(1, min(len(xh), len(io["x_hist"]))):
        ref = io["x_hist"][k]
        assert np.linalg.norm(xh[k] - ref) <= 1e-12 * np.linalg.norm(ref), k
    assert np.linalg.norm(_np(x1) - _np(x0)) <= 1e-12 * np.linalg.norm(_np(x0))


def test_ring_many_slices_per_warp(amg):
    # 96^3: 27,648 slices over at most 2 x 152 x 8 warps, several per warp and
    # several trips around each ring
    A = poisson3d(96)
    n = 96 ** 3
    Ad = amg.csr_to_device(A)
    r = torch.as_tensor(uniform01(23, n), device="cuda")
    z1 = amg.Hierarchy(*Ad, stream_ring=1).vcycle(r)
    z0 = amg.Hierarchy(*Ad, stream_ring=0).vcycle(r)
    assert torch.equal(z1, z0)


def test_wide_slices_fall_back(amg, orc):
    # rows of ~60 entries: a stage would not fit twice per warp in the ring's
    # shared memory, so the per-lane-load kernels run; results as before
    A = random_spd_graph(900, 0.07, 31)
    n = 900
    Ad = amg.csr_to_device(A)
    r = torch.as_tensor(uniform01(24, n), device="cuda")
    H1 = amg.Hierarchy(*Ad, stream_ring=1, max_coarse=40)
    H0 = amg.Hierarchy(*Ad, stream_ring=0, max_coarse=40)
    assert torch.equal(H1.vcycle(r), H0.vcycle(r))
    zo = orc.Hierarchy(A, max_coarse=40).vcycle(_np(r))
    assert np.linalg.norm(_np(H1.vcycle(r)) - zo) <= 1e-13 * np.linalg.norm(zo)
