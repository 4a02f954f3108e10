"""GPU path against the CPU oracle, through the C ABI.

Bit-exact: matchings, aggregates, coarse-level structure and values, smoother
scales.  FP64 kernels: SpMV and V-cycle to 1e-13 relative (summation order
and FMA differ); PCG iterates to 1e-12 relative at every step and the same
iteration count +-1.
"""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import random_spd_graph

pytestmark = pytest.mark.gpu


def _cases():
    yield "poisson32", poisson3d(32)
    yield "poisson_ragged", poisson3d(37, 11, 23)  # N not a multiple of the slice height
    yield "diffusion20", diffusion3d(np.exp(gaussian_field((20, 20, 20), 2.0, 4.0, 3)))
    yield "random300", random_spd_graph(300, 0.03, 9, positive_offdiag=True)


CASES = list(_cases())


def _dev(A):
    import paper_2406_19754_gb300 as amg

    return amg.csr_to_device(A)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_matching_bit_exact(amg, orc, case):
    _, A = case
    mate, rounds = amg.pairwise_match(*_dev(A))
    want = orc.match(A)
    assert np.array_equal(_np(mate), want)
    assert rounds >= 1


@pytest.mark.parametrize("sweeps", [1, 2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hierarchy_bit_exact(amg, orc, case, sweeps):
    _, A = case
    H = amg.Hierarchy(*_dev(A), sweeps=sweeps, max_coarse=50)
    Ho = orc.Hierarchy(A, sweeps=sweeps, max_coarse=50, max_dense=2048)
    assert Ho.status == 0
    assert H.levels == Ho.levels
    for l in range(H.levels):
        n, nnz = H.level_info(l)
        assert (n, nnz) == (Ho.level_n(l), Ho.level_nnz(l))
        ex = H.level_export(l)
        assert np.array_equal(_np(ex["sscale"]), Ho.level_dinv(l))
        if l > 0:
            rp, ci, v = Ho.level_csr(l)
            assert np.array_equal(_np(ex["rowptr"]), rp)
            assert np.array_equal(_np(ex["col"]), ci)
            assert np.array_equal(_np(ex["val"]), v)  # bitwise, canonical order
        if l < H.levels - 1:
            assert np.array_equal(_np(ex["agg"]), Ho.level_agg(l))


@pytest.mark.parametrize("tpr", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c[0])
def test_spmv_every_level(amg, orc, case, tpr):
    _, A = case
    H = amg.Hierarchy(*_dev(A), threads_per_row=tpr, max_coarse=50)
    Ho = orc.Hierarchy(A, max_coarse=50)
    for l in range(H.levels):
        Al = A if l == 0 else Ho.level_csr(l)
        n = H.level_info(l)[0]
        x = uniform01(40 + l, n) - 0.5
        y0 = uniform01(80 + l, n)
        want = 2.0 * orc.spmv(Al, x) - 0.5 * y0
        y = torch.as_tensor(y0, device="cuda")
        got = _np(H.spmv(torch.as_tensor(x, device="cuda"), y, level=l, alpha=2.0, beta=-0.5))
        scale = np.abs(want).max() + 1e-300
        assert np.max(np.abs(got - want)) <= 1e-13 * scale


@pytest.mark.parametrize("tpr", [1, 4, 32])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_vcycle_fp64_matches_oracle(amg, orc, case, tpr):
    _, A = case
    n = len(A[0]) - 1
    H = amg.Hierarchy(*_dev(A), threads_per_row=tpr)
    Ho = orc.Hierarchy(A)
    for seed in (1, 2):
        r = uniform01(seed, n) - 0.3
        z = _np(H.vcycle(torch.as_tensor(r, device="cuda")))
        zo = Ho.vcycle(r)
        assert np.linalg.norm(z - zo) <= 1e-13 * np.linalg.norm(zo)


def test_vcycle_single_level_is_cholesky(amg, orc):
    A = poisson3d(5)
    H = amg.Hierarchy(*_dev(A))
    assert H.levels == 1
    b = uniform01(4, 125)
    z = _np(H.vcycle(torch.as_tensor(b, device="cuda")))
    Ho = orc.Hierarchy(A)
    np.testing.assert_allclose(z, Ho.vcycle(b), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_pcg_iterates_match_oracle(amg, orc, case, use_graph):
    _, A = case
    n = len(A[0]) - 1
    b = uniform01(1, n)
    H = amg.Hierarchy(*_dev(A))
    Ho = orc.Hierarchy(A)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, maxit=200, history=True,
                    x_history=True, use_graph=use_graph)
    xo, io = orc.pcg(A, b, tol=1e-6, maxit=200, hier=Ho, history=True, x_history=True)
    assert info["status"] == 0 and io["status"] == 0
    assert abs(info["iterations"] - io["iterations"]) <= 1
    k = min(info["iterations"], io["iterations"])
    xh = _np(info["x_hist"])
    for j in range(1, k + 1):
        d = np.linalg.norm(xh[j] - io["x_hist"][j]) / np.linalg.norm(io["x_hist"][j])
        assert d <= 1e-12, (j, d)
    np.testing.assert_allclose(info["res_hist"][:k + 1], io["res_hist"][:k + 1], rtol=1e-10)
    assert info["true_relres"] <= 1.01e-6


def test_pcg_flexible_beta_matches_oracle(amg, orc):
    A = poisson3d(24)
    b = uniform01(3, 24 ** 3)
    H = amg.Hierarchy(*_dev(A))
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-8, beta_form="flexible",
                    x_history=True)
    xo, io = orc.pcg(A, b, tol=1e-8, hier=orc.Hierarchy(A), beta_form=1, x_history=True)
    assert abs(info["iterations"] - io["iterations"]) <= 1
    k = min(info["iterations"], io["iterations"])
    d = np.linalg.norm(_np(info["x_hist"])[k] - io["x_hist"][k]) / np.linalg.norm(io["x_hist"][k])
    assert d <= 1e-12


def test_pcg_f32_hierarchy(amg, orc):
    A = diffusion3d(np.exp(gaussian_field((24, 24, 24), 2.0, 4.0, 3)))
    n = 24 ** 3
    b = uniform01(4, n)
    H64 = amg.Hierarchy(*_dev(A))
    H32 = amg.Hierarchy(*_dev(A), precision="f32")
    Hbf = amg.Hierarchy(*_dev(A), precision="f32", bf16_from_level=2)
    bt = torch.as_tensor(b, device="cuda")
    x64, i64 = H64.pcg(bt, tol=1e-8)
    x32, i32 = H32.pcg(bt, tol=1e-8)
    xbf, ibf = Hbf.pcg(bt, tol=1e-8)
    xo, io = orc.pcg(A, b, tol=1e-8, hier=orc.Hierarchy(A))
    for info in (i64, i32, ibf):
        assert info["status"] == 0 and info["true_relres"] <= 1.05e-8
    assert abs(i32["iterations"] - i64["iterations"]) <= 1
    assert ibf["iterations"] <= i64["iterations"] + 3
    for x in (x32, xbf):
        err = np.linalg.norm(_np(x) - xo) / np.linalg.norm(xo)
        assert err < 1e-6


def test_smoother_weights_roundtrip(amg, orc):
    A = poisson3d(12)
    n = 12 ** 3
    om = (0.2 + 0.8 * uniform01(7, n)).astype(np.float32)
    H = amg.Hierarchy(*_dev(A))
    H.set_smoother_weights(torch.as_tensor(om, device="cuda"))
    Ho = orc.Hierarchy(A, omega=om.astype(np.float64))
    assert np.array_equal(_np(H.level_export(0)["sscale"]), Ho.level_dinv(0))
    r = uniform01(8, n)
    z = _np(H.vcycle(torch.as_tensor(r, device="cuda")))
    assert np.linalg.norm(z - Ho.vcycle(r)) <= 1e-13 * np.linalg.norm(z)
    H.set_smoother_weights(None)
    assert np.array_equal(_np(H.level_export(0)["sscale"]), orc.Hierarchy(A).level_dinv(0))


# ------------------------------------------------------------------ edge cases and errors

def test_one_by_one_and_tiny(amg, orc):
    A = (np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([4.0]))
    H = amg.Hierarchy(*_dev(A))
    x, info = H.pcg(torch.tensor([2.0], dtype=torch.float64, device="cuda"), tol=1e-12)
    assert info["status"] == 0 and abs(x.item() - 0.5) < 1e-15


def test_zero_rhs_converges_immediately(amg):
    H = amg.Hierarchy(*_dev(poisson3d(8)))
    x, info = H.pcg(torch.zeros(512, dtype=torch.float64, device="cuda"))
    assert info["iterations"] == 0 and info["status"] == 0 and float(x.abs().max()) == 0.0


def test_maxit_reported(amg):
    H = amg.Hierarchy(*_dev(poisson3d(16)))
    b = torch.as_tensor(uniform01(2, 4096), device="cuda")
    _, info = H.pcg(b, tol=1e-14, maxit=3)
    assert info["status"] == 1 and info["iterations"] == 3


def test_not_spd_is_reported(amg):
    import paper_2406_19754_gb300 as m

    # -Poisson is negative definite: the coarse Cholesky must refuse it
    rp, ci, v = poisson3d(4)
    with pytest.raises(m.AmgError) as e:
        m.Hierarchy(*_dev((rp, ci, -v)))
    assert e.value.status == m._lib.AMG_ERR_NOT_SPD


def test_bad_arguments_rejected(amg):
    import paper_2406_19754_gb300 as m

    A = _dev(poisson3d(4))
    with pytest.raises(m.AmgError) as e:
        m.Hierarchy(*A, sweeps=5)
    assert e.value.status == m._lib.AMG_ERR_ARG
    with pytest.raises(m.AmgError):
        m.Hierarchy(*A, slice_height=128, threads_per_row=1)  # heights 1..64
    with pytest.raises(m.AmgError):
        m.Hierarchy(*A, slice_height=12, threads_per_row=4)  # powers of two only
    with pytest.raises(m.AmgError):
        m.Hierarchy(*A, threads_per_row=3)
    H = m.Hierarchy(*A)
    with pytest.raises(m.AmgError):
        H.spmv(torch.zeros(64, dtype=torch.float64, device="cuda"), level=7)


def test_allocation_failure_is_clean(amg):
    import paper_2406_19754_gb300 as m

    lib = m._lib.load()
    A = _dev(poisson3d(10))
    for k in (0, 3, 17):
        lib.amg_debug_fail_alloc_after(k)
        with pytest.raises(m.AmgError) as e:
            m.Hierarchy(*A)
        assert e.value.status == m._lib.AMG_ERR_OOM
    lib.amg_debug_fail_alloc_after(-1)
    H = m.Hierarchy(*A)  # the library still works afterwards
    assert H.levels >= 2


def test_autotuned_layouts_keep_results(amg, orc):
    # the autotuner only changes slice height / threads per row: the hierarchy
    # stays bit-exact and the V-cycle agrees to rounding
    A = diffusion3d(np.exp(gaussian_field((24, 20, 16), 2.0, 4.0, 13)))
    n = 24 * 20 * 16
    H = amg.Hierarchy(*_dev(A), autotune=1, max_coarse=50)
    Ho = orc.Hierarchy(A, max_coarse=50)
    assert H.levels == Ho.levels
    for l in range(1, H.levels):
        assert np.array_equal(_np(H.level_export(l)["val"]), Ho.level_csr(l)[2])
    r = uniform01(5, n)
    z = _np(H.vcycle(torch.as_tensor(r, device="cuda")))
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-13 * np.linalg.norm(zo)
    _, info = H.pcg(torch.as_tensor(r, device="cuda"), tol=1e-8)
    _, io = orc.pcg(A, r, tol=1e-8, hier=Ho)
    assert info["status"] == 0 and abs(info["iterations"] - io["iterations"]) <= 1
