"""Compressed column indices in the sliced-ELL kernels (2-byte offsets from a
4-byte base per slice column) against plain 4-byte indices: the same slots
and the same order of operations, so every result must agree bit for bit;
a matrix whose offsets do not fit keeps plain indices and stays correct."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu


def _pair(amg, A, **opts):
    Ad = amg.csr_to_device(A)
    return (amg.Hierarchy(*Ad, compress_columns=1, **opts),
            amg.Hierarchy(*Ad, compress_columns=0, **opts))


@pytest.mark.parametrize("opts", [
    dict(precision="f64"),
    dict(precision="f32"),
    dict(precision="f32", bf16_from_level=1),
    dict(precision="f64", threads_per_row=2),
    dict(precision="f64", threads_per_row=4),
    dict(precision="f32", threads_per_row=8),
    dict(precision="f64", tail_rows=0),
])
def test_compressed_matches_plain_bitwise(amg, opts):
    shape = (36, 34, 32)
    n = shape[0] * shape[1] * shape[2]
    A = diffusion3d(np.exp(gaussian_field(shape, 2.0, 5.0, 31)))
    H, H0 = _pair(amg, A, **opts)
    assert H.levels == H0.levels
    for l in range(H.levels):
        assert H.level_layout(l)["compressed"] and not H0.level_layout(l)["compressed"]
        assert H.level_layout(l)["slots"] == H0.level_layout(l)["slots"]
        if l + 1 < H.levels:
            assert H.level_layout(l, ap=True)["compressed"]
    r = torch.as_tensor(uniform01(6, n), device="cuda")
    assert torch.equal(H.spmv(r), H0.spmv(r))
    assert torch.equal(H.vcycle(r), H0.vcycle(r))
    x, info = H.pcg(r, tol=1e-9)
    x0, info0 = H0.pcg(r, tol=1e-9)
    assert info["iterations"] == info0["iterations"] and torch.equal(x, x0)


def _chain_with_chords(n, d):
    """1-D chain plus a coupling i <-> i + d: diag 4, off-diagonals -1.
    Strictly diagonally dominant (SPD); rows around d mix column offsets
    near 0 and near d in one slice column."""
    rows = [[] for _ in range(n)]
    for i in range(n):
        for j in (i - d, i - 1, i + 1, i + d):
            if 0 <= j < n and (abs(i - j) == 1 or (abs(i - j) == d)):
                rows[i].append((j, -1.0))
        rows[i].append((i, 4.0))
        rows[i].sort()
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([j for r in rows for j, _ in r], dtype=np.int32)
    va = np.array([v for r in rows for _, v in r], dtype=np.float64)
    return rp, ci, va


def test_wide_offsets_fall_back_to_plain_indices(amg, orc):
    n, d = 140000, 70000
    A = _chain_with_chords(n, d)
    H = amg.Hierarchy(*amg.csr_to_device(A), compress_columns=1)
    assert not H.level_layout(0)["compressed"]
    x = uniform01(12, n)
    rp, ci, va = A
    y_ref = np.array([np.dot(va[rp[i]:rp[i + 1]], x[ci[rp[i]:rp[i + 1]]]) for i in range(n)])
    y = H.spmv(torch.as_tensor(x, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(y, y_ref, rtol=1e-14, atol=1e-14)
    Ho = orc.Hierarchy(A)
    z = H.vcycle(torch.as_tensor(x, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(x)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


def test_poisson_level0_is_compressed(amg):
    Ad = amg.csr_to_device(poisson3d(48))
    H = amg.Hierarchy(*Ad, compress_columns=1)
    lay = H.level_layout(0)
    assert lay["compressed"] and lay["slice_height"] == 32 and lay["threads_per_row"] == 1
    assert H.level_layout(0, ap=True)["compressed"]
    assert not amg.Hierarchy(*Ad).level_layout(0)["compressed"]  # off by default
    with pytest.raises(amg.AmgError):
        H.level_layout(H.levels - 1, ap=True)
