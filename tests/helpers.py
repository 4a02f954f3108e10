"""Small dense/sparse helpers for the tests (no solver arithmetic)."""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from synthetic import uniform01


def to_scipy(A):
    rp, ci, v = A
    n = len(rp) - 1
    return sp.csr_matrix((np.asarray(v), np.asarray(ci), np.asarray(rp)), shape=(n, n))


def dense(A):
    return to_scipy(A).toarray()


def from_dense(M):
    S = sp.csr_matrix(M)
    S.sort_indices()
    return (S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


def lap1d(n):
    M = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return from_dense(M)


def random_spd_graph(n, p, seed, positive_offdiag=False):
    """Symmetric random sparsity with off-diagonal values in [-1, 0) (or mixed
    sign), diagonal = row sum of |off| plus a margin: strictly diagonally
    dominant, hence SPD, and bitwise symmetric."""
    u = uniform01(seed, n * n * 3).reshape(3, n, n)
    mask = np.triu(u[0] < p, 1)
    vals = -(0.1 + u[1])
    if positive_offdiag:
        vals = np.where(u[2] < 0.3, -vals, vals)
    U = np.where(mask, vals, 0.0)
    M = U + U.T
    M[np.diag_indices(n)] = np.abs(M).sum(axis=1) + 0.5 + u[2].diagonal()
    return from_dense(M)


def dense_operator(apply, n):
    B = np.empty((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[:] = 0.0
        e[k] = 1.0
        B[:, k] = apply(e)
    return B


def prolongator(agg, nc):
    P = np.zeros((len(agg), nc))
    P[np.arange(len(agg)), agg] = 1.0
    return P
