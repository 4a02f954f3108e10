"""Batched solves of independent uneven systems against the oracle.

The oracle builds its hierarchy from the same block-diagonal matrix and runs
one PCG per diagonal block with that hierarchy's (block-diagonal) V-cycle.
Hierarchy: bit-exact.  Per system: iteration count +-1 and the solution to
1e-10 relative (different reduction order over many iterations)."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import random_spd_graph

pytestmark = pytest.mark.gpu


def _systems():
    return [poisson3d(9, 8, 7), diffusion3d(np.exp(gaussian_field((10, 10, 10), 2.0, 3.0, 5))),
            poisson3d(12), diffusion3d(np.exp(gaussian_field((7, 9, 11), 0.5, 2.0, 6))),
            random_spd_graph(300, 0.03, 12, positive_offdiag=True), poisson3d(3, 2, 1)]


def _dev_systems(amg, systems):
    return [amg.csr_to_device(S) for S in systems]


@pytest.fixture(scope="module")
def batch_case(amg, orc):
    systems = _systems()
    A, offs = orc.block_diag(systems)
    H = amg.BatchHierarchy(_dev_systems(amg, systems), max_coarse=40)
    Ho = orc.Hierarchy(A, max_coarse=40, systems=offs)
    return systems, A, offs, H, Ho


def test_batch_offsets_and_hierarchy_bit_exact(amg, orc, batch_case):
    systems, A, offs, H, Ho = batch_case
    assert H.offsets == offs and H.nsys == len(systems)
    assert H.levels == Ho.levels
    for l in range(H.levels):
        assert H.level_info(l) == (Ho.level_n(l), Ho.level_nnz(l))
        ex = H.level_export(l)
        if l > 0:
            rp, ci, v = Ho.level_csr(l)
            assert np.array_equal(ex["rowptr"].cpu().numpy(), rp)
            assert np.array_equal(ex["col"].cpu().numpy(), ci)
            assert np.array_equal(ex["val"].cpu().numpy(), v)
        if l < H.levels - 1:
            assert np.array_equal(ex["agg"].cpu().numpy(), Ho.level_agg(l))


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_pcg_matches_per_block_oracle(amg, orc, batch_case, use_graph):
    systems, A, offs, H, Ho = batch_case
    b = uniform01(3, offs[-1])
    x, stats = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-8, use_graph=use_graph)
    x = x.cpu().numpy()
    for k in range(len(systems)):
        bk = b[offs[k]:offs[k + 1]]
        xo, io = orc.pcg_block(Ho, offs[k], offs[k + 1], bk, tol=1e-8)
        st = stats[k]
        assert st["status"] == 0 and io["status"] == 0, (k, st, io)
        assert abs(st["iterations"] - io["iterations"]) <= 1, (k, st, io)
        xk = x[offs[k]:offs[k + 1]]
        assert np.linalg.norm(xk - xo) <= 1e-10 * np.linalg.norm(xo), k
        assert st["true_relres"] <= 1.05e-8


def test_batch_f32_and_maxit(amg, orc):
    systems = _systems()[:4]
    A, offs = orc.block_diag(systems)
    H = amg.BatchHierarchy(_dev_systems(amg, systems), precision="f32")
    b = torch.as_tensor(uniform01(4, offs[-1]), device="cuda")
    x, stats = H.pcg(b, tol=1e-8)
    for st in stats:
        assert st["status"] == 0 and st["true_relres"] <= 1.05e-8
    _, stats = H.pcg(b, tol=1e-15, maxit=4)
    assert all(st["status"] == 1 and st["iterations"] == 4 for st in stats)


def test_batch_coarsest_level_is_per_system(amg, orc):
    # systems of very different sizes: each stops coarsening at <= max_coarse
    # rows of its own, so the coarsest level is block diagonal, one block each
    systems = [poisson3d(24), poisson3d(6), diffusion3d(np.exp(gaussian_field((16, 12, 10), 2.0,
                                                                              4.0, 9)))]
    A, offs = orc.block_diag(systems)
    H = amg.BatchHierarchy(_dev_systems(amg, systems), max_coarse=30)
    Ho = orc.Hierarchy(A, max_coarse=30, systems=offs)
    assert Ho.status == 0 and H.levels == Ho.levels
    nl = H.levels
    assert H.level_info(nl - 1) == (Ho.level_n(nl - 1), Ho.level_nnz(nl - 1))
    b = uniform01(8, offs[-1])
    x, stats = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-10)
    for k in range(3):
        xo, io = orc.pcg_block(Ho, offs[k], offs[k + 1], b[offs[k]:offs[k + 1]], tol=1e-10)
        assert abs(stats[k]["iterations"] - io["iterations"]) <= 1
        xk = x[offs[k]:offs[k + 1]].cpu().numpy()
        assert np.linalg.norm(xk - xo) <= 1e-10 * np.linalg.norm(xo)


def test_batch_of_one_equals_single_solve(amg):
    S = poisson3d(20)
    b = torch.as_tensor(uniform01(5, 8000), device="cuda")
    Hb = amg.BatchHierarchy([amg.csr_to_device(S)])
    Hs = amg.Hierarchy(*amg.csr_to_device(S))
    xb, sb = Hb.pcg(b, tol=1e-8)
    xs, ss = Hs.pcg(b, tol=1e-8)
    assert sb[0]["iterations"] == ss["iterations"]
    assert float((xb - xs).norm() / xs.norm()) <= 1e-12
