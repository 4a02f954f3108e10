"""Slice heights decoupled from threads per row (the autotuner's second axis).

A layout (C, tpr) with C != 32 / tpr lets a warp cover 32 / tpr rows of one
or several slices (C < 32 / tpr) or part of a slice (C > 32 / tpr).  Each row
still sums its entries in ascending column order, so with one thread per row
the rows are the same bits as in the default layout; with several threads per
row the partial sums split differently and agree to rounding.  Checked
against the oracle (V-cycle, SpMV, PCG iterations), against the default
layout, with a ragged last slice, FP32 values, compressed columns, the
persistent small-level launch and the multi-RHS kernels.
"""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu

LAYOUTS = [(8, 1), (16, 1), (64, 1), (8, 2), (64, 2), (16, 4), (64, 4), (8, 8), (4, 8)]


def _np(t):
    return t.cpu().numpy()


def _problem():
    # 9,361 rows: a ragged last slice for every height
    return diffusion3d(np.exp(gaussian_field((23, 11, 37), 2.0, 4.0, 31)))


@pytest.mark.parametrize("C,tpr", LAYOUTS)
def test_decoupled_layout_matches_oracle(amg, orc, C, tpr):
    A = _problem()
    n = len(A[0]) - 1
    Ad = amg.csr_to_device(A)
    H = amg.Hierarchy(*Ad, slice_height=C, threads_per_row=tpr)
    for l in range(H.levels):
        lay = H.level_layout(l)
        assert (lay["slice_height"], lay["threads_per_row"]) == (C, tpr), l
    Ho = orc.Hierarchy(A)
    r = uniform01(41, n)
    rt = torch.as_tensor(r, device="cuda")
    z, zo = _np(H.vcycle(rt)), Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-13 * np.linalg.norm(zo)
    y, yo = _np(H.spmv(rt)), orc.spmv(A, r)
    assert np.linalg.norm(y - yo) <= 1e-14 * np.linalg.norm(yo)
    x, info = H.pcg(rt, tol=1e-10)
    xo, io = orc.pcg(A, r, tol=1e-10, hier=Ho)
    assert info["status"] == 0 and abs(info["iterations"] - io["iterations"]) <= 1
    assert np.linalg.norm(_np(x) - xo) <= 1e-10 * np.linalg.norm(xo)
    if tpr == 1:  # one thread per row: the default layout's bits
        H0 = amg.Hierarchy(*Ad)
        assert torch.equal(H.vcycle(rt), H0.vcycle(rt))


@pytest.mark.parametrize("C,tpr", [(8, 1), (64, 1), (16, 4)])
def test_decoupled_layout_fp32_compressed_and_tail(amg, orc, C, tpr):
    A = poisson3d(40, 33, 29)  # 38,280 rows
    n = 40 * 33 * 29
    Ad = amg.csr_to_device(A)
    r = torch.as_tensor(uniform01(42, n), device="cuda")
    zo = orc.Hierarchy(A).vcycle(_np(r))
    # FP32 operator values
    z32 = _np(amg.Hierarchy(*Ad, slice_height=C, threads_per_row=tpr, precision="f32").vcycle(r))
    assert np.linalg.norm(z32 - zo) <= 1e-5 * np.linalg.norm(zo)
    # compressed columns: the same bits as plain int32 columns
    Hc = amg.Hierarchy(*Ad, slice_height=C, threads_per_row=tpr, compress_columns=1)
    Hp = amg.Hierarchy(*Ad, slice_height=C, threads_per_row=tpr)
    assert torch.equal(Hc.vcycle(r), Hp.vcycle(r))
    # every level as separate launches against the persistent small-level launch
    Ht = amg.Hierarchy(*Ad, slice_height=C, threads_per_row=tpr, tail_rows=0)
    assert torch.equal(Ht.vcycle(r), Hp.vcycle(r))


def test_decoupled_layout_multi_rhs(amg):
    # the blocked kernels walk the slices themselves: any height works, and with
    # one thread per row each column is the single-vector V-cycle's bits
    A = poisson3d(24)
    n = 24 ** 3
    Ad = amg.csr_to_device(A)
    H = amg.Hierarchy(*Ad, slice_height=64, threads_per_row=1)
    R = torch.as_tensor(uniform01(43, n * 8).reshape(n, 8), device="cuda")
    Z = H.vcycle_multi(R)
    for c in range(8):
        assert torch.equal(Z[:, c], H.vcycle(R[:, c].contiguous())), c


def test_autotuner_picks_from_both_axes(amg, orc):
    A = diffusion3d(np.exp(gaussian_field((30, 28, 26), 2.0, 4.0, 44)))
    n = 30 * 28 * 26
    H = amg.Hierarchy(*amg.csr_to_device(A), autotune=1, max_coarse=50)
    cands = {(32 // t, t) for t in (1, 2, 4, 8)} | {(C, t) for t in (1, 2, 4, 8)
                                                   for C in (8, 16, 32, 64)}
    chosen = [(H.level_layout(l)["slice_height"], H.level_layout(l)["threads_per_row"])
              for l in range(H.levels - 1)]
    print("autotuned (slice height, threads per row) per level:", chosen)
    assert all(c in cands for c in chosen)
    Ho = orc.Hierarchy(A, max_coarse=50)
    r = uniform01(45, n)
    z = _np(H.vcycle(torch.as_tensor(r, device="cuda")))
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-13 * np.linalg.norm(zo)


def test_batched_systems_keep_coupled_slices(amg):
    from synthetic import diffusion_problem

    systems = [diffusion_problem(s, 1.0, 4.0, 50 + s) for s in (10, 13)]
    Hb = amg.BatchHierarchy([amg.csr_to_device(S) for S in systems], slice_height=64,
                            threads_per_row=1)
    lay = Hb.level_layout(0)
    assert (lay["slice_height"], lay["threads_per_row"]) == (32, 1)
