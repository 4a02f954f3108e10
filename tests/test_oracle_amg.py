"""Pins for matching, aggregation, the Galerkin product, the V-cycle and PCG.

Independent checks: brute-force maximum-weight matchings on tiny graphs, a
separate round-based locally-dominant matcher written here in plain Python,
closed-form coarse stencils, dense P^T A P by numpy, dense Eq. (amg) by
numpy, and CG step counts fixed by the spectrum.
"""

import itertools
import math
import os

import numpy as np
import pytest

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import (dense, dense_operator, from_dense, lap1d, prolongator,
                           random_spd_graph, to_scipy)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _graphs():
    yield "poisson5", poisson3d(5)
    yield "poisson_ragged", poisson3d(7, 3, 4)
    yield "diffusion", diffusion3d(np.exp(gaussian_field((6, 5, 4), 2.0, 2.0, 5)))
    for s in range(4):
        yield "random%d" % s, random_spd_graph(25 + 7 * s, 0.15, 40 + s, positive_offdiag=(s % 2))


# ------------------------------------------------------------------ weights

def test_weights_poisson_all_tie(orc):
    A = poisson3d(4)
    c = orc.match_weights(A)
    rp, ci, _ = A
    off = np.array([ci[e] != i for i in range(64) for e in range(rp[i], rp[i + 1])])
    # c = 1 - 2(-1)/(6 + 6) = 7/6 on every edge
    assert np.all(np.abs(c[off] - 7.0 / 6.0) <= 2.3e-16)
    assert len(np.unique(c[off])) == 1


def test_weights_of_spd_matrices_lie_in_0_2(orc):
    # for SPD A, |a_ij| < sqrt(a_ii a_jj) <= (a_ii + a_jj)/2, so 0 < c_ij < 2 (w = 1)
    for name, A in _graphs():
        c = orc.match_weights(A)
        rp, ci, _ = A
        off = np.array([ci[e] != i for i in range(len(rp) - 1) for e in range(rp[i], rp[i + 1])])
        assert np.all(c[off] > 0) and np.all(c[off] < 2), name


def test_weights_invariant_under_diagonal_scaling(orc):
    # c_ij(D A D, D^-1 w) = c_ij(A, w): the weights only see the scaled pair
    A = random_spd_graph(30, 0.2, 3, positive_offdiag=True)
    d = 0.5 + uniform01(9, 30)
    M = dense(A)
    B = from_dense(d[:, None] * M * d[None, :])
    c0 = orc.match_weights(A)
    c1 = orc.match_weights(B, 1.0 / d)
    np.testing.assert_allclose(c1, c0, rtol=1e-14, atol=1e-15)


# ------------------------------------------------------------------ matching

def _edges(orc, A):
    rp, ci, _ = A
    c = orc.match_weights(A)
    E = {}
    for i in range(len(rp) - 1):
        for e in range(rp[i], rp[i + 1]):
            j = int(ci[e])
            if j > i and c[e] > 0:
                E[(i, j)] = c[e]
    return E


def _check_matching(orc, A, mate):
    n = len(mate)
    E = _edges(orc, A)
    for i in range(n):
        m = mate[i]
        if m >= 0:
            assert mate[m] == i and m != i
            assert (min(i, m), max(i, m)) in E
    for (i, j) in E:  # maximal: no eligible edge with both ends free
        assert mate[i] >= 0 or mate[j] >= 0


@pytest.mark.parametrize("name_A", list(_graphs()), ids=lambda t: t[0])
def test_matching_valid_and_maximal(orc, name_A):
    _, A = name_A
    _check_matching(orc, A, orc.match(A))


def _rounds_locally_dominant(orc, A):
    """Independent statement: rounds of mutual heaviest-neighbour pointers."""
    n = len(A[0]) - 1
    E = _edges(orc, A)
    adj = {i: [] for i in range(n)}
    for (i, j), c in E.items():
        key = (c, -i, -j)
        adj[i].append((key, j))
        adj[j].append((key, i))
    mate = [-1] * n
    rounds = 0
    while True:
        cand = {}
        for i in range(n):
            if mate[i] >= 0:
                continue
            opts = [(k, j) for (k, j) in adj[i] if mate[j] < 0]
            if opts:
                cand[i] = max(opts)[1]
        if not cand:
            break
        rounds += 1
        for i, j in cand.items():
            if cand.get(j) == i:
                mate[i] = j
    return np.array(mate), rounds


@pytest.mark.parametrize("name_A", list(_graphs()), ids=lambda t: t[0])
def test_greedy_equals_locally_dominant_rounds(orc, name_A):
    _, A = name_A
    ld, rounds = _rounds_locally_dominant(orc, A)
    assert np.array_equal(orc.match(A), ld)
    assert rounds < len(ld)


def _max_weight_matching(n, E):
    best = 0.0
    edges = list(E.items())

    def rec(k, used, tot):
        nonlocal best
        best = max(best, tot)
        for t in range(k, len(edges)):
            (i, j), c = edges[t]
            if i not in used and j not in used:
                rec(t + 1, used | {i, j}, tot + c)

    rec(0, frozenset(), 0.0)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_matching_half_approximation_bruteforce(orc, seed):
    n = 8 + seed % 4
    A = random_spd_graph(n, 0.45, 300 + seed, positive_offdiag=True)
    E = _edges(orc, A)
    mate = orc.match(A)
    got = sum(c for (i, j), c in E.items() if mate[i] == j)
    assert got >= 0.5 * _max_weight_matching(n, E) - 1e-12


# ------------------------------------------------------------------ aggregation

def test_number_pairs_by_smallest_member(orc):
    mate = np.array([3, -1, 4, 0, 2, -1], dtype=np.int32)
    agg, nc = orc.number_pairs(mate)
    assert nc == 4
    assert list(agg) == [0, 1, 2, 0, 2, 3]


@pytest.mark.parametrize("name_A", list(_graphs())[:3], ids=lambda t: t[0])
def test_hierarchy_aggregates(orc, name_A):
    _, A = name_A
    H = orc.Hierarchy(A, sweeps=2, max_coarse=4)
    assert H.status == 0
    for l in range(H.levels - 1):
        agg = H.level_agg(l)
        nc = H.level_n(l + 1)
        sizes = np.bincount(agg, minlength=nc)
        assert sizes.min() >= 1 and sizes.max() <= 4
        firsts = np.array([np.flatnonzero(agg == I)[0] for I in range(nc)])
        assert np.all(np.diff(firsts) > 0)  # numbered by smallest member
        S = to_scipy(H.level_csr(l))
        for I in range(nc):  # every aggregate is connected in the level graph
            mem = np.flatnonzero(agg == I)
            sub = S[mem][:, mem].toarray() != 0
            seen, todo = {0}, [0]
            while todo:
                k = todo.pop()
                for m in np.flatnonzero(sub[k]):
                    if m not in seen:
                        seen.add(m)
                        todo.append(m)
            assert len(seen) == len(mem)


# ------------------------------------------------------------------ Galerkin

def test_galerkin_1d_pairs_reproduce_laplacian(orc):
    n = 16
    agg = np.arange(n) // 2
    Ac = orc.galerkin(lap1d(n), agg, n // 2)
    assert np.array_equal(dense(Ac), dense(lap1d(n // 2)))


def test_galerkin_poisson_x_pairs_closed_form(orc):
    nx = 6
    A = poisson3d(nx, 3, 2)
    x = np.arange(nx * 6) % nx
    rest = np.arange(nx * 6) // nx
    agg = (x // 2 + (nx // 2) * rest).astype(np.int32)
    C = dense(orc.galerkin(A, agg, (nx // 2) * 6))
    # coarse stencil: diagonal 6+6-1-1 = 10, x neighbours -1, y/z neighbours -2
    W = dense(poisson3d(nx // 2, 3, 2))
    want = np.where(W == 6, 10.0, 0.0)
    m = nx // 2
    for I in range(m * 6):
        for J in range(m * 6):
            if W[I, J] == -1:
                want[I, J] = -1.0 if abs(I - J) == 1 else -2.0
    assert np.array_equal(C, want)


@pytest.mark.parametrize("name_A", list(_graphs()), ids=lambda t: t[0])
def test_galerkin_equals_dense_triple_product(orc, name_A):
    _, A = name_A
    n = len(A[0]) - 1
    agg, nc = orc.number_pairs(orc.match(A))
    Ac = orc.galerkin(A, agg, nc)
    P = prolongator(agg, nc)
    M = dense(A)
    want = P.T @ M @ P
    got = dense(Ac)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-13 * np.abs(M).max())
    assert np.array_equal(got, got.T)  # bitwise symmetric
    # row-sum invariant and energy identity x_c^T A_c x_c = (P x_c)^T A (P x_c)
    np.testing.assert_allclose(got.sum(axis=1), P.T @ M.sum(axis=1), rtol=1e-13, atol=1e-12)
    xc = uniform01(13, nc) - 0.5
    assert math.isclose(xc @ got @ xc, (P @ xc) @ M @ (P @ xc), rel_tol=1e-12)
    assert n >= nc


def test_hierarchy_levels_bitwise_symmetric(orc):
    A = diffusion3d(np.exp(gaussian_field((10, 10, 10), 2.0, 3.0, 8)))
    H = orc.Hierarchy(A, max_coarse=10)
    assert H.levels >= 3
    for l in range(H.levels):
        M = dense(H.level_csr(l))
        assert np.array_equal(M, M.T)


def test_hierarchy_integer_poisson_levels_exact(orc):
    H = orc.Hierarchy(poisson3d(8), max_coarse=8)
    for l in range(1, H.levels):
        M = dense(H.level_csr(l))
        assert np.array_equal(M, np.round(M))  # 0/1 P keeps integer stencils
        P = prolongator(H.level_agg(l - 1), H.level_n(l))
        assert np.array_equal(M, P.T @ dense(H.level_csr(l - 1)) @ P)


# ------------------------------------------------------------------ V-cycle

def _vcycle_dense(orc, H, n):
    return dense_operator(H.vcycle, n)


@pytest.mark.parametrize("side,max_coarse", [(4, 8), (6, 8), (8, 8), (8, 40)])
def test_vcycle_symmetric_positive_definite(orc, side, max_coarse):
    A = poisson3d(side)
    n = side ** 3
    # plain l1-Jacobi, random under-relaxation, and random over-relaxation below 2
    # (2 diag(d/omega) - A > 0 keeps the smoother A-convergent, so B stays SPD)
    for omega in (None, 0.05 + 0.95 * uniform01(side, n), 1.0 + 0.95 * uniform01(side + 1, n)):
        H = orc.Hierarchy(A, max_coarse=max_coarse, omega=omega)
        assert H.levels >= 2
        B = _vcycle_dense(orc, H, n)
        assert np.linalg.norm(B - B.T) <= 1e-14 * np.linalg.norm(B)
        np.linalg.cholesky(0.5 * (B + B.T))
        ev = np.linalg.eigvals(B @ dense(A))
        assert np.abs(ev.imag).max() < 1e-10
        assert ev.real.min() > 0 and ev.real.max() <= 1.0 + 1e-12


def test_vcycle_two_level_matches_eq_amg(orc):
    # I - B A = (I - M^-T A)(I - P A_c^-1 P^T A)(I - M^-1 A), M^-1 = diag(s)
    A = diffusion3d(np.exp(gaussian_field((5, 5, 5), 1.5, 2.0, 6)))
    n = 125
    H = orc.Hierarchy(A, max_coarse=60)
    assert H.levels == 2
    M = dense(A)
    S = np.diag(H.level_dinv(0))
    P = prolongator(H.level_agg(0), H.level_n(1))
    Ac = P.T @ M @ P
    I = np.eye(n)
    E = (I - S @ M) @ (I - P @ np.linalg.solve(Ac, P.T @ M)) @ (I - S @ M)
    B_formula = (I - E) @ np.linalg.inv(M)
    B = _vcycle_dense(orc, H, n)
    np.testing.assert_allclose(B, B_formula, rtol=0, atol=1e-12 * np.abs(B).max())


def test_vcycle_single_level_is_exact_solve(orc):
    A = poisson3d(5)
    H = orc.Hierarchy(A, max_coarse=200)
    assert H.levels == 1
    b = uniform01(3, 125)
    np.testing.assert_allclose(H.vcycle(b), np.linalg.solve(dense(A), b), rtol=1e-13)
    L = H.coarse_factor()
    np.testing.assert_allclose(L, np.linalg.cholesky(dense(A)), rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ PCG

@pytest.mark.parametrize("seed", range(5))
def test_cg_exact_in_n_steps(orc, seed):
    n = 6 + 3 * seed
    A = random_spd_graph(n, 0.5, 500 + seed, positive_offdiag=True)
    b = uniform01(seed, n)
    x, info = orc.pcg(A, b, tol=1e-12, maxit=n)
    assert info["status"] == 0 and info["iterations"] <= n
    np.testing.assert_allclose(x, np.linalg.solve(dense(A), b), rtol=1e-9)


def test_cg_poisson_2x2x2_four_distinct_eigenvalues(orc):
    with open(os.path.join(GOLD, "poisson2x2x2_cg.txt")) as f:
        rows = dict(l.split(None, 1) for l in f if l.strip() and not l.startswith("#"))
    A = poisson3d(2)
    ev = sorted(set(np.round(np.linalg.eigvalsh(dense(A)), 12)))
    assert ev == [float(s) for s in rows["eigenvalues"].split()]
    b = uniform01(17, 8) + 0.1
    _, info = orc.pcg(A, b, tol=1e-13, maxit=20)
    assert info["status"] == 0 and info["iterations"] == int(rows["cg_iterations"])


def test_pcg_with_exact_inverse_takes_one_step(orc):
    A = random_spd_graph(15, 0.4, 8)
    Ainv = np.linalg.inv(dense(A))
    b = uniform01(2, 15)
    _, info = orc.pcg(A, b, tol=1e-12, binv=Ainv)
    assert info["iterations"] == 1 and info["status"] == 0


@pytest.mark.parametrize("beta_form", [0, 1])
def test_pcg_amg_poisson_32(orc, beta_form):
    A = poisson3d(32)
    b = uniform01(1, 32 ** 3)
    H = orc.Hierarchy(A)
    x, info = orc.pcg(A, b, tol=1e-6, hier=H, beta_form=beta_form, history=True)
    assert info["status"] == 0 and info["true_relres"] <= 1.01e-6
    r = b - to_scipy(A) @ x
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6
    assert 10 <= info["iterations"] <= 40


# ------------------------------------------------------------------ batched systems

def _batch_systems():
    return [poisson3d(5, 4, 3), diffusion3d(np.exp(gaussian_field((4, 5, 6), 1.5, 2.0, 31))),
            poisson3d(6), random_spd_graph(40, 0.1, 77, positive_offdiag=True)]


def test_block_diagonal_hierarchy_gives_block_diagonal_vcycle(orc):
    A, offs = orc.block_diag(_batch_systems())
    H = orc.Hierarchy(A, max_coarse=8)
    assert H.levels >= 3
    B = dense_operator(H.vcycle, offs[-1])
    for a in range(len(offs) - 1):
        for c in range(len(offs) - 1):
            blk = B[offs[a]:offs[a + 1], offs[c]:offs[c + 1]]
            if a != c:
                assert np.all(blk == 0.0)  # exactly: every operator is block diagonal
    for l in range(H.levels - 1):  # no aggregate spans two systems
        agg = H.level_agg(l)
        sysof = np.searchsorted(offs[1:], np.arange(offs[-1]), side="right") if l == 0 else None
        if sysof is not None:
            for I in range(H.level_n(l + 1)):
                assert len(set(sysof[agg == I])) == 1


def test_block_pcg_solves_each_block(orc):
    systems = _batch_systems()
    A, offs = orc.block_diag(systems)
    H = orc.Hierarchy(A, max_coarse=8)
    for k, S in enumerate(systems):
        n = offs[k + 1] - offs[k]
        b = uniform01(50 + k, n)
        x, info = orc.pcg_block(H, offs[k], offs[k + 1], b, tol=1e-10)
        assert info["status"] == 0
        np.testing.assert_allclose(x, np.linalg.solve(dense(S), b), rtol=1e-8)
    # a single block is the plain solve
    S = systems[2]
    b = uniform01(9, 216)
    Hs = orc.Hierarchy(S, max_coarse=8)
    A1, o1 = orc.block_diag([S])
    H1 = orc.Hierarchy(A1, max_coarse=8)
    xa, ia = orc.pcg(S, b, tol=1e-10, hier=Hs)
    xb, ib = orc.pcg_block(H1, 0, 216, b, tol=1e-10)
    assert ia["iterations"] == ib["iterations"]
    np.testing.assert_allclose(xa, xb, rtol=1e-13)
