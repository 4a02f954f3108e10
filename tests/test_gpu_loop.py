"""The PCG loop as one graph (device-side stopping test in a conditional
while node) against the host-driven loop (one graph per iteration, or plain
launches): same decisions, same iterates bit for bit."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("maxit,tol", [(500, 1e-9), (7, 1e-12), (1, 1e-12)])
def test_loop_graph_matches_host_loop(amg, precision, maxit, tol):
    A = diffusion3d(np.exp(gaussian_field((30, 28, 26), 1.0, 4.0, 12)))
    n = 30 * 28 * 26
    H = amg.Hierarchy(*amg.csr_to_device(A), precision=precision)
    b = torch.as_tensor(uniform01(8, n), device="cuda")
    x1, i1 = H.pcg(b, tol=tol, maxit=maxit)                 # loop graph
    x2, i2 = H.pcg(b, tol=tol, maxit=maxit, history=True)   # graph per iteration
    x3, i3 = H.pcg(b, tol=tol, maxit=maxit, use_graph=False)
    for x, i in ((x2, i2), (x3, i3)):
        assert i["iterations"] == i1["iterations"] and i["status"] == i1["status"]
        assert i["relres"] == i1["relres"]
        assert torch.equal(x, x1)
    if maxit < 100:
        assert i1["status"] == 1 and i1["iterations"] == maxit
    else:
        assert i1["status"] == 0 and i1["relres"] <= tol
        assert i2["res_hist"][-1] == i1["relres"]


def test_loop_graph_reused_and_rebuilt(amg):
    A = poisson3d(32)
    n = 32 ** 3
    H = amg.Hierarchy(*amg.csr_to_device(A))
    b = torch.as_tensor(uniform01(2, n), device="cuda")
    xa, ia = H.pcg(b, tol=1e-8)
    xb, ib = H.pcg(2.0 * b, tol=1e-8)           # new x buffer: graph rebuilt
    x = torch.zeros_like(b)
    xc, ic = H.pcg(b, x, tol=1e-8)
    xd, id_ = H.pcg(b, x.zero_(), tol=1e-8)     # same x buffer: graph reused
    assert ia["iterations"] == ic["iterations"] == id_["iterations"]
    assert torch.equal(xa, xc) and torch.equal(xc, xd)
    assert torch.allclose(xb, 2.0 * xa, rtol=1e-6)
    # a zero right-hand side stops before the first iteration
    x0, i0 = H.pcg(torch.zeros_like(b), tol=1e-8)
    assert i0["iterations"] == 0 and i0["status"] == 0 and not torch.any(x0)


def _batch_systems():
    return [poisson3d(14, 12, 10), diffusion3d(np.exp(gaussian_field((16, 14, 12), 1.5, 3.0, 3))),
            poisson3d(9), diffusion3d(np.exp(gaussian_field((20, 10, 8), 0.7, 2.0, 4)))]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_loop_graph_matches_host_loop(amg, precision):
    Ad = [amg.csr_to_device(S) for S in _batch_systems()]
    H = amg.BatchHierarchy(Ad, precision=precision, max_coarse=30)
    b = torch.as_tensor(uniform01(5, H.n), device="cuda")
    x1, s1 = H.pcg(b, tol=1e-9)                    # loop graph
    x2, s2 = H.pcg(b, tol=1e-9, use_graph=False)   # host loop, plain launches
    assert [s["iterations"] for s in s1] == [s["iterations"] for s in s2]
    assert [s["status"] for s in s1] == [s["status"] for s in s2] == [0] * 4
    assert torch.equal(x1, x2)
    # the same output buffer with another tolerance and cap: nothing stale
    x = torch.zeros_like(b)
    _, sa = H.pcg(b, x, tol=1e-4)
    _, sb = H.pcg(b, x.zero_(), tol=1e-9, maxit=6)
    assert all(s["iterations"] <= t["iterations"] for s, t in zip(sa, s1))
    assert all(s["iterations"] == min(6, t["iterations"]) for s, t in zip(sb, s1))
