"""Multi-RHS V-cycle and PCG against the single-RHS path and the oracle.

The blocked V-cycle must reproduce every column's single V-cycle bit for bit
(same per-column operation order).  Blocked PCG: per column, the iteration
count +-1 and the solution to 1e-10 relative against the oracle's PCG.

Column counts cover both kernel forms: 16-byte column vectors when 4 (FP32)
or 2 (FP64) divides K -- K = 2, 4, 8, 12, 32, 48, 64, including lane layouts
that leave lanes idle (12, 48) -- and per-column lanes otherwise (1, 5, 33)
or when a vector is not 16-byte aligned."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("K", [1, 2, 4, 5, 8, 12, 32, 33, 48, 64])
def test_vcycle_multi_equals_single_columns(amg, precision, K):
    A = poisson3d(19, 13, 11)  # ragged slices
    n = 19 * 13 * 11
    H = amg.Hierarchy(*amg.csr_to_device(A), precision=precision, max_coarse=60)
    R = torch.as_tensor(uniform01(K, n * K).reshape(n, K) - 0.4, device="cuda")
    Z = H.vcycle_multi(R)
    for c in range(K):
        zc = H.vcycle(R[:, c].contiguous())
        assert torch.equal(Z[:, c], zc), c


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_vcycle_multi_unaligned_vectors(amg, precision):
    # R and Z 8 bytes past a 16-byte boundary: the per-column kernels run,
    # with the same bits as the vector kernels on aligned copies
    A = poisson3d(19, 13, 11)
    n, K = 19 * 13 * 11, 8
    H = amg.Hierarchy(*amg.csr_to_device(A), precision=precision, max_coarse=60)
    buf = torch.as_tensor(uniform01(9, n * K + 1), device="cuda")
    R = buf[1:].view(n, K)
    zbuf = torch.zeros(n * K + 1, dtype=torch.float64, device="cuda")
    Z = zbuf[1:].view(n, K)
    assert R.data_ptr() % 16 == 8 and Z.data_ptr() % 16 == 8
    H.vcycle_multi(R, Z)
    assert torch.equal(Z, H.vcycle_multi(R.clone()))
    assert torch.equal(Z[:, 5], H.vcycle(R[:, 5].contiguous()))


def test_vcycle_multi_bf16_levels(amg):
    A = diffusion3d(np.exp(gaussian_field((16, 16, 16), 2.0, 3.0, 2)))
    H = amg.Hierarchy(*amg.csr_to_device(A), precision="f32", bf16_from_level=1)
    R = torch.as_tensor(uniform01(3, 4096 * 7).reshape(4096, 7), device="cuda")
    Z = H.vcycle_multi(R)
    for c in range(7):
        assert torch.equal(Z[:, c], H.vcycle(R[:, c].contiguous()))


@pytest.mark.parametrize("K", [12, 7])  # vector-column and per-column kernels
def test_pcg_multi_matches_oracle_per_column(amg, orc, K):
    A = poisson3d(20)
    n = 8000
    H = amg.Hierarchy(*amg.csr_to_device(A))
    Bh = uniform01(100, n * K).reshape(n, K)
    Bh[:, 3] = 0.0  # converged before the first step
    X, stats = H.pcg_multi(torch.as_tensor(Bh, device="cuda"), tol=1e-8)
    X = X.cpu().numpy()
    Ho = orc.Hierarchy(A)
    for c in range(K):
        xo, io = orc.pcg(A, Bh[:, c].copy(), tol=1e-8, hier=Ho)
        st = stats[c]
        assert st["status"] == 0 and abs(st["iterations"] - io["iterations"]) <= 1, (c, st, io)
        if c == 3:
            assert st["iterations"] == 0 and np.all(X[:, c] == 0.0)
            continue
        assert np.linalg.norm(X[:, c] - xo) <= 1e-10 * np.linalg.norm(xo), c
        assert st["true_relres"] <= 1.05e-8


def test_pcg_multi_f32_and_columns_stop_independently(amg):
    A = diffusion3d(np.exp(gaussian_field((20, 20, 20), 1.5, 4.0, 8)))
    n, K = 8000, 40
    H = amg.Hierarchy(*amg.csr_to_device(A), precision="f32")
    Bh = uniform01(7, n * K).reshape(n, K)
    Bh[:, ::2] *= 1e-3  # scaling a column must not change its relative convergence
    X, stats = H.pcg_multi(torch.as_tensor(Bh, device="cuda"), tol=1e-8)
    its = [s["iterations"] for s in stats]
    assert all(s["status"] == 0 and s["true_relres"] <= 1.05e-8 for s in stats)
    assert max(its) - min(its) <= 3
    # against single-RHS solves of two columns
    for c in (0, 1):
        xs, si = H.pcg(torch.as_tensor(Bh[:, c].copy(), device="cuda"), tol=1e-8)
        assert abs(si["iterations"] - its[c]) <= 1
        rel = float((X[:, c] - xs).norm() / xs.norm())
        assert rel < 1e-6


def test_multi_rejects_bad_shapes(amg):
    import paper_2406_19754_gb300 as m

    H = m.Hierarchy(*m.csr_to_device(poisson3d(10)))
    with pytest.raises(m.AmgError):
        H.vcycle_multi(torch.zeros((1000, 65), dtype=torch.float64, device="cuda"))
