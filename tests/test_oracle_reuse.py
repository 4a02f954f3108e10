"""Pins for rebuilding a hierarchy on new matrix values with the aggregates of
an existing one (the paper's coefficient update with preserved structure,
Sec. 2.2): the new level matrices are P^T A P with the old P (dense numpy),
the smoother scales 1/sum|a_ij|, and the same matrix reproduces the original
hierarchy exactly."""

import numpy as np

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import dense, dense_operator, prolongator


def test_reuse_same_matrix_reproduces_the_hierarchy(orc):
    A = diffusion3d(np.exp(gaussian_field((9, 8, 7), 1.5, 2.0, 4)))
    H = orc.Hierarchy(A, max_coarse=20)
    R = H.reuse(A)
    assert R.status == 0 and R.levels == H.levels
    for l in range(H.levels):
        for a, b in zip(H.level_csr(l), R.level_csr(l)):
            assert np.array_equal(a, b)
        assert np.array_equal(H.level_dinv(l), R.level_dinv(l))
    b = uniform01(1, 9 * 8 * 7)
    assert np.array_equal(H.vcycle(b), R.vcycle(b))


def test_reuse_new_values_is_galerkin_with_the_old_aggregates(orc):
    shape = (10, 9, 8)
    n = 10 * 9 * 8
    A1 = diffusion3d(np.exp(gaussian_field(shape, 1.0, 2.0, 7)))
    A2 = diffusion3d(np.exp(gaussian_field(shape, 2.5, 3.0, 8)))  # same sparsity
    assert np.array_equal(A1[0], A2[0]) and np.array_equal(A1[1], A2[1])
    H = orc.Hierarchy(A1, max_coarse=15)
    R = H.reuse(A2)
    assert R.status == 0 and R.levels == H.levels >= 3
    Ad = dense(A2)
    for l in range(H.levels - 1):
        agg = H.level_agg(l)
        assert np.array_equal(agg, R.level_agg(l))
        P = prolongator(agg, H.level_n(l + 1))
        Ac = P.T @ Ad @ P
        assert np.abs(dense(R.level_csr(l + 1)) - Ac).max() <= 1e-13 * np.abs(Ac).max()
        d = np.abs(Ad).sum(axis=1)
        assert np.allclose(R.level_dinv(l), 1.0 / d, rtol=1e-15, atol=0)
        Ad = dense(R.level_csr(l + 1))
    # the rebuilt V-cycle is symmetric positive definite (usable by PCG)
    B = dense_operator(R.vcycle, n)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    # and differs from a fresh hierarchy of A2 only through the aggregates
    F = orc.Hierarchy(A2, max_coarse=15)
    same = all(np.array_equal(F.level_agg(l), H.level_agg(l)) for l in range(F.levels - 1))
    if same and F.levels == H.levels:
        assert np.array_equal(F.vcycle(uniform01(3, n)), R.vcycle(uniform01(3, n)))


def test_reuse_rejects_another_structure(orc):
    H = orc.Hierarchy(poisson3d(6, 5, 4), max_coarse=10)
    R = H.reuse(poisson3d(5, 6, 4))
    assert R.status == -1
