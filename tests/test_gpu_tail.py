"""The persistent launch of the small levels (levels with at most `tail_rows`
rows and the coarsest solve between barriers) against one launch per step:
the same per-row code runs in both, so every result must agree bit for bit,
in every precision and layout and for batched systems.  The launch is one CTA
when its largest level has at most 16384 rows (__syncthreads between phases)
and a cooperative grid with the bounded grid barrier beyond; both are
covered below."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu


def _pair(amg, A, **opts):
    Ad = amg.csr_to_device(A)
    return (amg.Hierarchy(*Ad, **opts), amg.Hierarchy(*Ad, **dict(opts, tail_rows=0)))


def _kinds(H, r):
    _, recs = H.vcycle_profile(r)
    return [(x["level"], x["kind"]) for x in recs]


SMALL = (40, 36, 30)   # 43200 rows: the default tail runs in one CTA
LARGE = (64, 64, 64)   # level 1 has 65536 rows: a tail from it spans the grid
HUGE = (96, 96, 96)    # level 1 has 221184 rows: a wider grid


@pytest.mark.parametrize("shape,opts", [
    (SMALL, dict(precision="f64")),
    (SMALL, dict(precision="f32")),
    (SMALL, dict(precision="f32", bf16_from_level=2)),
    (SMALL, dict(precision="f64", threads_per_row=2)),
    (SMALL, dict(precision="f32", threads_per_row=4, slice_height=8)),
    (SMALL, dict(precision="f64", threads_per_row=16)),
    (SMALL, dict(precision="f32", threads_per_row=32, tail_rows=16384)),
    (SMALL, dict(precision="f64", tail_rows=16384)),
    (LARGE, dict(precision="f64", tail_rows=70000)),
    (LARGE, dict(precision="f32", tail_rows=70000, threads_per_row=2)),
    (LARGE, dict(precision="f32", tail_rows=20000, bf16_from_level=1)),
    # several sweeps per side, the variable V-cycle, the PCG coarsest solve
    (SMALL, dict(precision="f64", smooth_sweeps=2, variable_cycle=1, tail_rows=16384)),
    (SMALL, dict(precision="f32", smooth_sweeps=3, tail_rows=16384)),
    (SMALL, dict(precision="f64", smooth_sweeps=2, coarse_solver=1, tail_rows=16384)),
    (SMALL, dict(precision="f64", coarse_solver=1, coarse_tol=0.0, coarse_maxit=9,
                 tail_rows=16384)),
    (LARGE, dict(precision="f64", smooth_sweeps=2, variable_cycle=1, tail_rows=70000)),
    (HUGE, dict(precision="f64", tail_rows=300000)),
    (HUGE, dict(precision="f32", smooth_sweeps=2, tail_rows=300000)),
])
def test_tail_vcycle_bitwise(amg, shape, opts):
    A = diffusion3d(np.exp(gaussian_field(shape, 1.5, 4.0, 21)))
    n = shape[0] * shape[1] * shape[2]
    H, H0 = _pair(amg, A, **opts)
    assert H.levels == H0.levels >= 4
    r = torch.as_tensor(uniform01(4, n), device="cuda")
    z, z0 = H.vcycle(r), H0.vcycle(r)
    assert torch.equal(z, z0)
    kinds = _kinds(H, r)
    lt = [l for l, k in kinds if k == "tail"]
    assert len(lt) == 1 and all(k != "tail" for _, k in _kinds(H0, r))
    expect = next(l for l in range(1, H.levels) if H.level_info(l)[0] <= H.opts.tail_rows)
    assert lt[0] == expect
    # no per-step record at or below the tail level
    assert all(l < lt[0] for l, k in kinds if k != "tail")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_tail_pcg_bitwise(amg, precision):
    A = poisson3d(44)
    n = 44 ** 3
    H, H0 = _pair(amg, A, precision=precision)
    b = torch.as_tensor(uniform01(7, n), device="cuda")
    x, info = H.pcg(b, tol=1e-10, history=True)
    x0, info0 = H0.pcg(b, tol=1e-10, history=True)
    assert info["status"] == info0["status"] == 0
    assert info["iterations"] == info0["iterations"]
    assert info["res_hist"] == info0["res_hist"]
    assert torch.equal(x, x0)


@pytest.mark.parametrize("tail_rows", [8000, 30000])
def test_tail_large_coarsest_bitwise(amg, tail_rows):
    # coarsest level above 1024 rows: the two-phase row-parallel coarse solve,
    # in one CTA (tail from 6912 rows) and over the grid (from 27648 rows)
    A = poisson3d(48)
    H, H0 = _pair(amg, A, max_coarse=2000, tail_rows=tail_rows)
    assert H.levels >= 3 and H.level_info(H.levels - 1)[0] > 1024
    r = torch.as_tensor(uniform01(5, 48 ** 3), device="cuda")
    assert torch.equal(H.vcycle(r), H0.vcycle(r))
    assert any(k == "tail" for _, k in _kinds(H, r))
    x, info = H.pcg(r, tol=1e-9)
    x0, info0 = H0.pcg(r, tol=1e-9)
    assert info["iterations"] == info0["iterations"] and torch.equal(x, x0)


def test_tail_batch_bitwise(amg):
    systems = [poisson3d(20, 18, 16), diffusion3d(np.exp(gaussian_field((24, 20, 22), 2.0, 4.0, 8))),
               poisson3d(26), diffusion3d(np.exp(gaussian_field((12, 30, 14), 0.5, 2.0, 9)))]
    Ad = [amg.csr_to_device(S) for S in systems]
    H = amg.BatchHierarchy(Ad, precision="f32", max_coarse=60)
    H0 = amg.BatchHierarchy(Ad, precision="f32", max_coarse=60, tail_rows=0)
    assert H.levels == H0.levels >= 3
    b = torch.as_tensor(uniform01(11, H.n), device="cuda")
    assert torch.equal(H.vcycle(b), H0.vcycle(b))
    x, st = H.pcg(b, tol=1e-8)
    x0, st0 = H0.pcg(b, tol=1e-8)
    assert [s["iterations"] for s in st] == [s["iterations"] for s in st0]
    assert all(s["status"] == 0 for s in st)
    assert torch.equal(x, x0)


def test_tail_rows_option_checked(amg):
    A = poisson3d(10)
    with pytest.raises(amg.AmgError):
        amg.Hierarchy(*amg.csr_to_device(A), tail_rows=-1)


def test_tail_barrier_timeout_reported_and_recovered(amg):
    # Test hook: the barrier waits for an arrival that never comes; every CTA
    # gives up after 10 ms (bounded, no fault), the solve reports
    # AMG_ERR_DEVICE_CHECK, and the handle works again once the hook is off.
    from paper_2406_19754_gb300 import _lib

    A = poisson3d(48)  # level 1 has 27648 rows: the tail spans the grid
    n = 48 ** 3
    Ad = amg.csr_to_device(A)
    H = amg.Hierarchy(*Ad, tail_rows=30000)
    b = torch.as_tensor(uniform01(3, n), device="cuda")
    x_ref, info_ref = amg.Hierarchy(*Ad, tail_rows=30000).pcg(b, tol=1e-8)
    lib = _lib.load()
    for use_graph in (True, False):
        assert lib.amg_debug_tail_timeout(H.h, 1) == 0
        with pytest.raises(amg.AmgError) as e:
            H.pcg(b, tol=1e-8, use_graph=use_graph)
        assert e.value.status == _lib.AMG_ERR_DEVICE_CHECK
        assert lib.amg_debug_tail_timeout(H.h, 0) == 0
        x, info = H.pcg(b, tol=1e-8, use_graph=use_graph)
        assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
        assert torch.equal(x, x_ref)
