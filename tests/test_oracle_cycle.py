"""Pins for the oracle's V(nu, nu) cycle, the variable V-cycle and the PCG
coarsest solver (the VBM / VMATCH configurations of Sec. 3).

Independent checks: the V-cycle's error-propagation recursion assembled with
dense numpy matrices (E = K^nu (I - P B_c P^T A) K^nu, K = I - S A,
B = (I - E) A^-1), and a textbook preconditioned CG written here in numpy.
"""

import numpy as np
import pytest

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import dense, dense_operator, prolongator


def _levels(Ho, A0):
    mats, S, P = [], [], []
    for l in range(Ho.levels):
        A = dense(A0) if l == 0 else dense(Ho.level_csr(l))
        mats.append(A)
        S.append(np.diag(Ho.level_dinv(l)))
        if l + 1 < Ho.levels:
            agg = Ho.level_agg(l)
            P.append(prolongator(agg, Ho.level_n(l + 1)))
    return mats, S, P


def _recursive_B(mats, S, P, nu0, variable, Bc):
    """B_0 of the V(nu_l, nu_l) cycle by the error-propagation recursion."""
    B = Bc
    for l in range(len(mats) - 2, -1, -1):
        A = mats[l]
        n = A.shape[0]
        nu = nu0 * 2 ** l if variable else nu0
        K = np.eye(n) - S[l] @ A
        Kn = np.linalg.matrix_power(K, nu)
        E = Kn @ (np.eye(n) - P[l] @ B @ P[l].T @ A) @ Kn
        B = (np.eye(n) - E) @ np.linalg.inv(A)
    return B


@pytest.mark.parametrize("nu0,variable", [(1, False), (2, False), (3, False), (1, True),
                                          (2, True)])
@pytest.mark.parametrize("sweeps", [2, 3])
def test_vcycle_sweeps_match_error_propagation(orc, nu0, variable, sweeps):
    A = diffusion3d(np.exp(gaussian_field((7, 6, 5), 1.5, 2.0, 13)))
    n = 7 * 6 * 5
    Ho = orc.Hierarchy(A, sweeps=sweeps, max_coarse=6, smooth_sweeps=nu0, variable=variable)
    assert Ho.status == 0 and Ho.levels >= 3
    mats, S, P = _levels(Ho, A)
    B = _recursive_B(mats, S, P, nu0, variable, np.linalg.inv(mats[-1]))
    Bo = dense_operator(Ho.vcycle, n)
    assert np.abs(Bo - B).max() <= 1e-10 * np.abs(B).max()
    assert np.abs(Bo - Bo.T).max() <= 1e-10 * np.abs(Bo).max()  # symmetric: PCG applies
    assert np.linalg.eigvalsh(0.5 * (Bo + Bo.T)).min() > 0


def test_one_sweep_is_the_v11_cycle(orc):
    A = poisson3d(9, 8, 7)
    b = uniform01(3, 9 * 8 * 7)
    z1 = orc.Hierarchy(A, max_coarse=20).vcycle(b)
    z2 = orc.Hierarchy(A, max_coarse=20, smooth_sweeps=1, variable=False).vcycle(b)
    assert np.array_equal(z1, z2)
    # the variable cycle with nu_0 = 1 differs once a coarser level sweeps twice
    z3 = orc.Hierarchy(A, max_coarse=20, variable=True).vcycle(b)
    assert not np.array_equal(z1, z3)


def _numpy_pcg(A, dinv, b, maxit, tol):
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for _ in range(maxit):
        q = A @ p
        pq = p @ q
        if not pq > 0:
            break
        a = rz / pq
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * bn:
            break
        z = dinv * r
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    return x


@pytest.mark.parametrize("maxit", [1, 3, 7])
def test_coarse_pcg_matches_textbook_pcg(orc, maxit):
    # one level: the whole V-cycle is the coarsest solve
    A = diffusion3d(np.exp(gaussian_field((5, 4, 3), 1.0, 2.0, 2)))
    b = uniform01(4, 60) - 0.3
    Ho = orc.Hierarchy(A, max_levels=1, coarse="pcg", coarse_maxit=maxit, coarse_tol=0.0)
    assert Ho.levels == 1
    x = Ho.vcycle(b)
    xr = _numpy_pcg(dense(A), Ho.level_dinv(0), b, maxit, 0.0)
    assert np.linalg.norm(x - xr) <= 1e-12 * np.linalg.norm(xr)


def test_coarse_pcg_finite_termination_and_tolerance(orc):
    A = poisson3d(4, 3, 3)  # 36 rows, well conditioned
    n = 36
    b = uniform01(9, n)
    Ho = orc.Hierarchy(A, max_levels=1, coarse="pcg", coarse_maxit=n, coarse_tol=1e-14)
    x = Ho.vcycle(b)
    xs = np.linalg.solve(dense(A), b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    # a loose tolerance stops early, with the residual it promised
    Ho2 = orc.Hierarchy(A, max_levels=1, coarse="pcg", coarse_maxit=n, coarse_tol=1e-2)
    x2 = Ho2.vcycle(b)
    assert np.linalg.norm(b - dense(A) @ x2) <= 1e-2 * np.linalg.norm(b)
    assert np.linalg.norm(x2 - xs) > 1e-8 * np.linalg.norm(xs)
    # zero right-hand side: zero solution, no iterations
    assert not np.any(Ho.vcycle(np.zeros(n)))


def test_vmatch_configuration_converges(orc):
    """The paper's VMATCH choices (aggregates <= 8, variable V-cycle from two
    sweeps, PCG-l1 coarsest solve, at most 40 iterations) inside flexible CG."""
    A = poisson3d(24)
    n = 24 ** 3
    b = np.ones(n)
    Ho = orc.Hierarchy(A, sweeps=3, smooth_sweeps=2, variable=True, coarse="pcg",
                       coarse_maxit=40, coarse_tol=1e-4)
    x, info = orc.pcg(A, b, tol=1e-6, hier=Ho, beta_form=1)
    assert info["status"] == 0 and info["iterations"] <= 20
    assert np.linalg.norm(b - dense(A) @ x) <= 1.1e-6 * np.linalg.norm(b)
