"""Pins for the input generators, SpMV, the l1 diagonal and Cholesky.

Every check compares against something other than the oracle itself: the
published splitmix64 sequence, closed-form Laplacian eigenpairs, a library
routine (scipy, numpy), or an invariant the paper states.
"""

import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from synthetic import (csr_nnz_poisson3d, diffusion3d, gaussian_field, poisson3d, splitmix64,
                       standard_normal, uniform01)
from tests.helpers import dense, lap1d, random_spd_graph, to_scipy

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLD, name)) as f:
        return [int(s) for s in f.read().split() if not s.startswith("#") and s.isdigit()]


# ------------------------------------------------------------------ generators

def test_splitmix64_published_sequence(orc):
    want = _golden_ints("splitmix64.txt")
    got = [int(v) for v in splitmix64(1234567, 5)]
    assert got == want
    gamma = 0x9E3779B97F4A7C15
    assert orc.mix64(1234567 + gamma) == want[0]
    assert orc.mix64(1234567 + 2 * gamma) == want[1]


def test_uniform_and_normal_moments():
    u = uniform01(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    z = standard_normal(8, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 1, 1), (4, 4, 4), (3, 5, 7), (16, 16, 16)])
def test_poisson_structure(shape):
    nx, ny, nz = shape
    rp, ci, v = poisson3d(nx, ny, nz)
    n = nx * ny * nz
    assert len(rp) == n + 1 and rp[-1] == csr_nnz_poisson3d(nx, ny, nz)
    M = dense((rp, ci, v))
    assert np.array_equal(M, M.T)
    assert np.all(np.diag(M) == 6.0)
    off = M - np.diag(np.diag(M))
    assert set(np.unique(off)) <= {0.0, -1.0}
    for i in range(n):  # ascending columns in every row
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


def test_diffusion_unit_coefficient_is_poisson():
    A = poisson3d(5, 4, 3)
    B = diffusion3d(np.ones((3, 4, 5)))
    for a, b in zip(A, B):
        assert np.array_equal(a, b)


def test_diffusion_bitwise_symmetric_and_dominant():
    k = np.exp(gaussian_field((6, 7, 8), 2.0, 2.0, 11))
    A = diffusion3d(k)
    M = dense(A)
    assert np.array_equal(M, M.T)
    off = np.abs(M - np.diag(np.diag(M))).sum(axis=1)
    nnb = (M != 0).sum(axis=1) - 1
    assert np.all(np.diag(M) >= off * (1 - 1e-14))  # interior rows: weakly dominant
    assert np.all(np.diag(M)[nnb < 6] > off[nnb < 6])  # boundary faces: strictly dominant
    # harmonic-mean face between cells 0 and 1 (x neighbours)
    k0, k1 = k[0, 0, 0], k[0, 0, 1]
    assert math.isclose(-M[0, 1], 2 * k0 * k1 / (k0 + k1), rel_tol=1e-15)


def test_gaussian_field_covariance():
    # Cov(r) = sigma^2 exp(-r^2 / (2 ell^2)); estimated over independent seeds
    sigma, ell = 1.5, 2.0
    fs = np.stack([gaussian_field((8, 8, 8), sigma, ell, 100 + s) for s in range(300)])
    var = fs[:, 4, 4, 4].var()
    assert abs(var / sigma ** 2 - 1.0) < 0.2
    c2 = np.mean(fs[:, 4, 4, 2] * fs[:, 4, 4, 4]) / sigma ** 2
    assert abs(c2 - math.exp(-4.0 / (2 * ell * ell))) < 0.12


# ------------------------------------------------------------------ SpMV

def test_spmv_matches_scipy(orc):
    for A in (poisson3d(7, 5, 3), random_spd_graph(40, 0.2, 3, positive_offdiag=True),
              diffusion3d(np.exp(gaussian_field((5, 6, 7), 1.0, 2.0, 4)))):
        x = uniform01(5, len(A[0]) - 1) - 0.5
        y = orc.spmv(A, x)
        np.testing.assert_allclose(y, to_scipy(A) @ x, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("n,ks", [(9, (1, 1, 1)), (9, (2, 5, 9)), (12, (3, 7, 1))])
def test_poisson_eigenvector_closed_form(orc, n, ks):
    # A v = (6 - 2 sum_d cos(k_d pi / (n + 1))) v for v = prod_d sin(k_d pi x_d / (n + 1))
    t = np.arange(1, n + 1)
    s = [np.sin(k * math.pi * t / (n + 1)) for k in ks]
    v = np.einsum("k,j,i->kji", s[2], s[1], s[0]).reshape(-1)
    lam = 6.0 - 2.0 * sum(math.cos(k * math.pi / (n + 1)) for k in ks)
    y = orc.spmv(poisson3d(n), v)
    np.testing.assert_allclose(y, lam * v, atol=1e-12)


def test_laplacian_extreme_eigenvalues(orc):
    n = 16
    A = poisson3d(n)
    N = n ** 3
    op = spla.LinearOperator((N, N), matvec=lambda x: orc.spmv(A, x), dtype=np.float64)
    c = math.cos(math.pi / (n + 1))
    lam_min, lam_max = 6 - 6 * c, 6 + 6 * c
    big = spla.eigsh(op, k=1, which="LA", tol=1e-12, return_eigenvectors=False)[0]
    small = spla.eigsh(op, k=1, sigma=0.0, which="LM", tol=1e-12, return_eigenvectors=False,
                       OPinv=spla.LinearOperator((N, N), matvec=lambda b: spla.spsolve(
                           to_scipy(A).tocsc(), b)))[0]
    assert abs(big - lam_max) < 1e-10
    assert abs(small - lam_min) < 1e-10
    # 1D Laplacian tridiag(-1, 2, -1): eigenvalues 2 - 2 cos(k pi / (n + 1))
    L = lap1d(10)
    ev = np.sort(np.linalg.eigvalsh(dense(L)))
    want = np.sort(2 - 2 * np.cos(np.arange(1, 11) * math.pi / 11))
    np.testing.assert_allclose(ev, want, atol=1e-13)
    y = orc.spmv(L, np.sin(3 * math.pi * np.arange(1, 11) / 11))
    np.testing.assert_allclose(y, want[2] * np.sin(3 * math.pi * np.arange(1, 11) / 11),
                               atol=1e-13)


def test_dot_blocked_exact_integers(orc):
    x = np.arange(10000, dtype=np.float64)
    assert orc.dot(x, np.ones(10000)) == 10000 * 9999 / 2
    y = uniform01(3, 9000)
    assert abs(orc.dot(y, y) - math.fsum(y * y)) < 1e-11


# ------------------------------------------------------------------ l1 diagonal

def test_l1_diagonal_poisson_closed_form(orc):
    A = poisson3d(5)
    d = orc.l1_scale(A)
    rp = A[0]
    for i in range(125):
        nnb = rp[i + 1] - rp[i] - 1
        assert d[i] == 1.0 / (6.0 + nnb)  # interior rows: 1/12, l1-Jacobi = Jacobi w = 1/2
    assert d[62] == 1.0 / 12.0


@pytest.mark.parametrize("which", ["poisson", "diffusion", "random"])
def test_l1_jacobi_is_A_convergent(orc, which):
    # Sec. 2.3: ||I - M^-1 A||_A < 1 without damping; also for any omega in (0, 1]
    if which == "poisson":
        A = poisson3d(6)
    elif which == "diffusion":
        A = diffusion3d(np.exp(gaussian_field((6, 6, 6), 2.0, 2.0, 9)))
    else:
        A = random_spd_graph(60, 0.15, 12, positive_offdiag=True)
    M = dense(A)
    n = M.shape[0]
    for omega in (None, 0.05 + 0.95 * uniform01(77, n)):
        s = orc.l1_scale(A, omega)
        Ssq = np.sqrt(s)
        ev = np.linalg.eigvalsh(Ssq[:, None] * M * Ssq[None, :])  # eig(S A), S = M^-1
        rho = np.max(np.abs(1.0 - ev))
        assert ev.min() > 0 and rho < 1.0


# ------------------------------------------------------------------ Cholesky

def test_cholesky_matches_numpy(orc):
    A = dense(random_spd_graph(30, 0.3, 21, positive_offdiag=True))
    L, st = orc.cholesky(A)
    assert st == 0
    np.testing.assert_allclose(L @ L.T, A, rtol=0, atol=1e-14 * np.abs(A).max())
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-13, atol=1e-14)
    b = uniform01(4, 30)
    np.testing.assert_allclose(orc.chol_solve(L, b), np.linalg.solve(A, b), rtol=1e-12)


def test_cholesky_rejects_indefinite(orc):
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    _, st = orc.cholesky(A)
    assert st == -2
