"""Pins for the oracle's smoothed prolongator (Sec. 2.3, SMATCH):
P = (I - w D^-1 A) P_hat, w = 1 / ||D^-1 A||_inf, coarse matrices P^T A P,
and the V-cycle that restricts with P^T and prolongs with P -- all checked
against dense numpy written here."""

import numpy as np
import pytest

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import dense, dense_operator, prolongator


def _rect(csr, ncols):
    rp, ci, v = csr
    M = np.zeros((len(rp) - 1, ncols))
    for i in range(len(rp) - 1):
        for e in range(rp[i], rp[i + 1]):
            M[i, ci[e]] += v[e]
    return M


def _problem():
    return diffusion3d(np.exp(gaussian_field((9, 8, 7), 1.5, 2.0, 21)))


def test_prolongator_and_galerkin_match_dense(orc):
    A = _problem()
    H = orc.Hierarchy(A, sweeps=3, max_coarse=12, smoothed=True)
    assert H.status == 0 and H.levels >= 3
    Ad = dense(A)
    for l in range(H.levels - 1):
        (rp, ci, v), w = H.level_prolongator(l)
        D = np.diag(Ad)
        assert w == pytest.approx(1.0 / np.max(np.abs(Ad).sum(axis=1) / D), rel=1e-15)
        Ph = prolongator(H.level_agg(l), H.level_n(l + 1))
        P = Ph - w * (Ad / D[:, None]) @ Ph
        Pg = _rect((rp, ci, v), P.shape[1])
        assert np.abs(Pg - P).max() <= 1e-15 * np.abs(P).max()
        assert all(np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0) for i in range(len(rp) - 1))
        Ac = P.T @ Ad @ P
        Ad = dense(H.level_csr(l + 1))
        assert np.abs(Ad - Ac).max() <= 1e-13 * np.abs(Ac).max()


@pytest.mark.parametrize("nu0", [1, 2, 4])
def test_smoothed_vcycle_matches_error_propagation(orc, nu0):
    A = _problem()
    n = 9 * 8 * 7
    H = orc.Hierarchy(A, sweeps=2, max_coarse=20, smoothed=True, smooth_sweeps=nu0)
    mats, S, P = [], [], []
    for l in range(H.levels):
        mats.append(dense(A) if l == 0 else dense(H.level_csr(l)))
        S.append(np.diag(H.level_dinv(l)))
        if l + 1 < H.levels:
            Pcsr, _ = H.level_prolongator(l)
            P.append(_rect(Pcsr, H.level_n(l + 1)))
    B = np.linalg.inv(mats[-1])
    for l in range(len(mats) - 2, -1, -1):
        Al = mats[l]
        K = np.linalg.matrix_power(np.eye(len(Al)) - S[l] @ Al, nu0)
        E = K @ (np.eye(len(Al)) - P[l] @ B @ P[l].T @ Al) @ K
        B = (np.eye(len(Al)) - E) @ np.linalg.inv(Al)
    Bo = dense_operator(H.vcycle, n)
    assert np.abs(Bo - B).max() <= 1e-10 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (Bo + Bo.T)).min() > 0


def test_smatch_configuration(orc):
    """Aggregates <= 8, smoothed P, 4 l1-Jacobi sweeps, PCG-l1 coarsest solve
    (<= 40 iterations): fewer iterations and a larger operator complexity
    than the unsmoothed VMATCH-style hierarchy, as the paper reports."""
    A = poisson3d(24)
    b = np.ones(24 ** 3)
    Hs = orc.Hierarchy(A, sweeps=3, smoothed=True, smooth_sweeps=4, coarse="pcg")
    Hu = orc.Hierarchy(A, sweeps=3, smooth_sweeps=4, coarse="pcg")
    _, i_s = orc.pcg(A, b, tol=1e-6, hier=Hs, beta_form=1)
    _, i_u = orc.pcg(A, b, tol=1e-6, hier=Hu, beta_form=1)
    assert i_s["status"] == 0 and i_u["status"] == 0
    assert i_s["iterations"] < i_u["iterations"]
    assert Hs.operator_complexity() > Hu.operator_complexity()


def test_smoothed_reuse_recomputes_the_prolongator(orc):
    A1 = _problem()
    A2 = diffusion3d(np.exp(gaussian_field((9, 8, 7), 2.5, 3.0, 22)))
    H = orc.Hierarchy(A1, sweeps=2, max_coarse=20, smoothed=True)
    R = H.reuse(A2)
    F = orc.Hierarchy(A2, sweeps=2, max_coarse=20, smoothed=True)
    assert R.status == 0
    (_, _, v1), w1 = H.level_prolongator(0)
    (_, _, v2), w2 = R.level_prolongator(0)
    assert not np.array_equal(v1, v2)  # (w is 1/2 for both: diagonally dominant rows)
    b = uniform01(5, 9 * 8 * 7)
    if all(np.array_equal(F.level_agg(l), H.level_agg(l)) for l in range(F.levels - 1)):
        assert np.array_equal(F.vcycle(b), R.vcycle(b))


def test_matching_takes_each_edge_from_its_upper_row(orc):
    """Smoothed coarse matrices are symmetric only up to rounding; the matching
    reads edge {i, j} from row min(i, j), so replacing every value below the
    diagonal changes nothing, while changing the values above it does."""
    rp, ci, v = poisson3d(12)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    u = uniform01(12, len(v))
    lower = (rp, ci, np.where(ci < rows, v * (1.0 + 1e-3 * u), v))
    upper = (rp, ci, np.where(ci > rows, v * (1.0 + 1e-3 * u), v))
    assert np.array_equal(orc.match(lower), orc.match((rp, ci, v)))
    assert not np.array_equal(orc.match(upper), orc.match((rp, ci, v)))


def test_filtered_prolongator_smoothing_matches_dense(orc):
    """With pfilter > 0 the prolongator is smoothed with A_F: entries with
    |a_ij| < theta sqrt(a_ii a_jj) dropped and lumped into the diagonal (row
    sums kept), P = P_hat - w D^-1 A_F P_hat with D and w from A; the coarse
    matrix stays P^T A P with the unfiltered A."""
    A = diffusion3d(np.exp(gaussian_field((12, 10, 9), 2.5, 2.0, 23)))
    theta = 0.08
    H = orc.Hierarchy(A, sweeps=2, max_coarse=12, smoothed=True, pfilter=theta)
    assert H.status == 0 and H.levels >= 3
    Ad = dense(A)
    dropped_somewhere = False
    for l in range(H.levels - 1):
        d = np.diag(Ad)
        weak = (np.abs(Ad) < theta * np.sqrt(np.outer(d, d))) & ~np.eye(len(d), dtype=bool)
        dropped_somewhere |= bool(weak.any())
        AF = np.where(weak, 0.0, Ad)
        AF[np.diag_indices(len(d))] += np.where(weak, Ad, 0.0).sum(axis=1)
        assert np.allclose(AF.sum(axis=1), Ad.sum(axis=1), rtol=1e-13, atol=1e-13)
        (rp, ci, v), w = H.level_prolongator(l)
        assert w == pytest.approx(1.0 / np.max(np.abs(Ad).sum(axis=1) / d), rel=1e-14)
        Ph = prolongator(H.level_agg(l), H.level_n(l + 1))
        P = Ph - w * (AF / d[:, None]) @ Ph
        assert np.abs(_rect((rp, ci, v), P.shape[1]) - P).max() <= 1e-14 * np.abs(P).max()
        Ac = P.T @ Ad @ P
        Ad = dense(H.level_csr(l + 1))
        assert np.abs(Ad - Ac).max() <= 1e-13 * np.abs(Ac).max()
    assert dropped_somewhere


def test_filtered_smatch_is_sparser(orc):
    # on Poisson every level-0 coupling is strong; the coarse levels lose their
    # weak entries, so the hierarchy is sparser and converges as fast
    A = poisson3d(24)
    b = np.ones(24 ** 3)
    Hu = orc.Hierarchy(A, sweeps=3, smoothed=True, smooth_sweeps=4, coarse="pcg")
    Hf = orc.Hierarchy(A, sweeps=3, smoothed=True, smooth_sweeps=4, coarse="pcg", pfilter=0.01)
    assert Hf.operator_complexity() < Hu.operator_complexity()
    _, iu = orc.pcg(A, b, tol=1e-6, hier=Hu, beta_form=1)
    _, i_f = orc.pcg(A, b, tol=1e-6, hier=Hf, beta_form=1)
    assert i_f["iterations"] <= iu["iterations"] + 1
