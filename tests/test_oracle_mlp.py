"""Pins for the learned-smoother oracle: features from closed-form stencils,
the MLP against PyTorch's CPU float64 layers and autograd, Adam against
torch.optim.Adam, and the two-grid loss against a dense evaluation of
E = S (I - P A_c^-1 P^T A) S with central finite differences for its
gradient."""

import math

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, standard_normal, uniform01
from tests.helpers import dense, prolongator

NF, NH = 9, 32


def _params(seed, scale=0.5):
    return scale * standard_normal(seed, 1409)


def _torch_mlp(p):
    p = torch.as_tensor(p, dtype=torch.float64)
    o = 0
    W1 = p[o:o + NH * NF].reshape(NH, NF); o += NH * NF
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    W3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def _torch_forward(params, feat, omega_max=1.0):
    W1, b1, W2, b2, W3, b3 = _torch_mlp(params)
    f = torch.as_tensor(feat, dtype=torch.float64)
    h1 = torch.nn.functional.gelu(f @ W1.T + b1)
    h2 = torch.nn.functional.gelu(h1 @ W2.T + b2)
    z = h2 @ W3 + b3
    return torch.clamp(omega_max * torch.sigmoid(z), min=1e-3)


def test_features_poisson_closed_form(orc):
    A = poisson3d(5, 4, 3)
    f = orc.mlp_features(A, (3, 4, 5))
    i = 1 + 5 * (1 + 4 * 1)  # interior cell (1, 1, 1)
    np.testing.assert_array_equal(f[i], [-1 / 6] * 6 + [1.0, 0.0, 1.0])
    # corner (0, 0, 0): only +x, +y, +z neighbours
    np.testing.assert_array_equal(f[0], [0, -1 / 6, 0, -1 / 6, 0, -1 / 6, 0.5, 0.0, 0.5])


def test_features_diffusion_harmonic_faces(orc):
    k = np.exp(gaussian_field((4, 5, 6), 1.0, 2.0, 3))
    A = diffusion3d(k)
    f = orc.mlp_features(A, k.shape)
    z, y, x = 2, 2, 3
    i = x + 6 * (y + 5 * z)
    h = lambda a, b: 2 * a * b / (a + b)
    faces = [h(k[z, y, x], k[z, y, x - 1]), h(k[z, y, x], k[z, y, x + 1]),
             h(k[z, y, x], k[z, y - 1, x]), h(k[z, y, x], k[z, y + 1, x]),
             h(k[z, y, x], k[z - 1, y, x]), h(k[z, y, x], k[z + 1, y, x])]
    diag = sum(faces)
    np.testing.assert_allclose(f[i, :6], [-fc / diag for fc in faces], rtol=1e-14)
    assert math.isclose(f[i, 6], 1.0, rel_tol=1e-14)  # interior rows: zero row sum
    assert math.isclose(f[i, 7], math.log(max(faces) / min(faces)), rel_tol=1e-12)


def test_forward_matches_torch(orc):
    feat = orc.mlp_features(diffusion3d(np.exp(gaussian_field((6, 6, 6), 2.0, 2.0, 4))),
                            (6, 6, 6))
    p = _params(11)
    om, _ = orc.mlp_forward(p, feat)
    np.testing.assert_allclose(om, _torch_forward(p, feat).numpy(), rtol=1e-13, atol=1e-15)
    assert np.all(om >= 1e-3) and np.all(om < 1.0)
    om0, z0 = orc.mlp_forward(np.zeros(1409), feat)  # zero network: sigmoid(0)
    assert np.all(om0 == 0.5) and np.all(z0 == 0.0)


@pytest.mark.parametrize("omega_max", [1.5, 1.9])
def test_forward_backward_with_omega_cap(orc, omega_max):
    # omega = max(omega_max sigmoid(z), 1e-3): over-relaxation up to omega_max < 2
    feat = orc.mlp_features(diffusion3d(np.exp(gaussian_field((5, 6, 4), 2.0, 2.0, 9))),
                            (5, 6, 4))
    p = _params(14)
    om, _ = orc.mlp_forward(p, feat, omega_max)
    want = _torch_forward(p, feat, omega_max).numpy()
    np.testing.assert_allclose(om, want, rtol=1e-13, atol=1e-15)
    assert np.all(om >= 1e-3) and np.all(om < omega_max) and om.max() > 1.0
    om0, _ = orc.mlp_forward(np.zeros(1409), feat, omega_max)
    assert np.all(om0 == 0.5 * omega_max)  # zero network: omega_max sigmoid(0)
    g_out = uniform01(15, len(om)) - 0.5
    grad = orc.mlp_backward(p, feat, g_out, omega_max)
    pt = torch.as_tensor(p, dtype=torch.float64).requires_grad_(True)
    (_torch_forward(pt, feat, omega_max) * torch.as_tensor(g_out)).sum().backward()
    np.testing.assert_allclose(grad, pt.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_backward_matches_autograd_and_differences(orc):
    feat = orc.mlp_features(poisson3d(4, 3, 5), (5, 3, 4)) + 0.1 * uniform01(2, 60 * 9).reshape(
        60, 9)
    p = _params(12)
    g_out = uniform01(3, 60) - 0.5
    grad = orc.mlp_backward(p, feat, g_out)
    pt = torch.as_tensor(p, dtype=torch.float64).requires_grad_(True)
    (_torch_forward(pt, feat) * torch.as_tensor(g_out)).sum().backward()
    np.testing.assert_allclose(grad, pt.grad.numpy(), rtol=1e-10, atol=1e-14)
    h = 1e-6
    for k in (0, 100, 300, 700, 1343, 1400, 1408):
        e = np.zeros(1409)
        e[k] = h
        fd = (orc.mlp_forward(p + e, feat)[0] - orc.mlp_forward(p - e, feat)[0]) @ g_out / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1e-8, abs(grad[k])) + 1e-9, k


def test_adam_matches_torch(orc):
    p = _params(13)
    m, v = np.zeros(1409), np.zeros(1409)
    pt = torch.nn.Parameter(torch.as_tensor(p.copy()))
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = standard_normal(100 + t, 1409)
        orc.mlp_adam(p, g, m, v, t)
        pt.grad = torch.as_tensor(g)
        opt.step()
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)


def _two_grid_setup(orc, side=6, sigma=1.5):
    A = diffusion3d(np.exp(gaussian_field((side,) * 3, sigma, 2.0, 21)))
    H = orc.Hierarchy(A, max_coarse=1)  # only level 0's aggregates and level 1 are used
    agg = H.level_agg(0)
    return A, agg, H.level_csr(1)


def test_two_grid_loss_matches_dense(orc):
    A, agg, Ac = _two_grid_setup(orc)
    n = len(agg)
    om = 0.3 + 0.7 * uniform01(5, n)
    e0 = standard_normal(6, 2 * n).reshape(2, n)
    loss, _ = orc.twogrid_loss(A, agg, Ac, om, e0, K=2)
    M = dense(A)
    d = np.abs(M).sum(axis=1)
    S = np.eye(n) - (om / d)[:, None] * M
    P = prolongator(agg, len(Ac[0]) - 1)
    E = S @ (np.eye(n) - P @ np.linalg.solve(P.T @ M @ P, P.T @ M)) @ S
    want = 0.0
    for e in e0:
        eK = E @ (E @ e)
        want += math.log(math.sqrt(eK @ M @ eK) / math.sqrt(e @ M @ e)) / 2
    assert math.isclose(loss, want / 2, rel_tol=1e-11)
    assert loss < 0.0  # omega in (0, 1]: each cycle contracts the A-norm


def test_two_grid_loss_over_relaxed_contracts(orc):
    # omega in (1, 2): 2 diag(d / omega) - A = (2/omega - 1) diag(d) + (diag(d) - A) > 0
    # keeps S = I - diag(omega / d) A an A-norm contraction, so the loss stays negative
    A, agg, Ac = _two_grid_setup(orc)
    n = len(agg)
    om = 1.0 + 0.95 * uniform01(9, n)
    M = dense(A)
    d = np.abs(M).sum(axis=1)
    ev = np.linalg.eigvals((om / d)[:, None] * M).real  # eig(diag(s) A) in (0, 2)
    assert ev.min() > 0.0 and ev.max() < 2.0
    e0 = standard_normal(10, 2 * n).reshape(2, n)
    loss, _ = orc.twogrid_loss(A, agg, Ac, om, e0, K=2)
    assert loss < 0.0


def test_two_grid_gradient_central_differences(orc):
    A, agg, Ac = _two_grid_setup(orc)
    n = len(agg)
    om = 0.3 + 0.7 * uniform01(7, n)
    e0 = standard_normal(8, 3 * n).reshape(3, n)
    _, g = orc.twogrid_loss(A, agg, Ac, om, e0, K=2)
    h = 1e-6
    for i in (0, 17, 55, 101, n - 1):
        e = np.zeros(n)
        e[i] = h
        lp, _ = orc.twogrid_loss(A, agg, Ac, om + e, e0, K=2)
        lm, _ = orc.twogrid_loss(A, agg, Ac, om - e, e0, K=2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-10, (i, fd, g[i])
