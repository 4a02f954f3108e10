"""Learned-smoother kernels against the FP64 oracle: features, forward,
backward (gradients), Adam, and the two-grid loss with its gradient."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, standard_normal, uniform01

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm(amg):
    from paper_2406_19754_gb300 import learned

    return learned


def _problem(shape=(10, 9, 8), sigma=2.0, seed=3):
    return diffusion3d(np.exp(gaussian_field(shape, sigma, 3.0, seed)))


def test_features_match_oracle(amg, orc, lm):
    for A, shape in ((_problem(), (10, 9, 8)), (poisson3d(7, 6, 5), (5, 6, 7))):
        m = lm.Mlp(0)
        f = m.features(amg.csr_to_device(A), shape).cpu().numpy()
        np.testing.assert_allclose(f, orc.mlp_features(A, shape), rtol=2e-6, atol=1e-7)


def test_forward_backward_match_oracle(amg, orc, lm):
    A, shape = _problem(), (10, 9, 8)
    n = 720
    m = lm.Mlp(1)
    p = (0.5 * standard_normal(21, m.nparam)).astype(np.float32)
    m.set_params(p)
    feat = m.features(amg.csr_to_device(A), shape)
    m.set_exact_forward(True)  # FP32 on the CUDA cores
    om = m.forward(feat).cpu().numpy()
    m.set_exact_forward(False)
    f64 = feat.cpu().numpy().astype(np.float64)
    om_o, _ = orc.mlp_forward(p.astype(np.float64), f64)
    np.testing.assert_allclose(om, om_o, rtol=2e-5, atol=1e-6)
    g_out = (uniform01(5, n) - 0.5).astype(np.float32)
    m.backward(feat, torch.as_tensor(g_out, device="cuda"), accumulate=False)
    g = m.grad()
    g_o = orc.mlp_backward(p.astype(np.float64), f64, g_out.astype(np.float64))
    assert np.linalg.norm(g - g_o) <= 1e-5 * np.linalg.norm(g_o)
    # accumulate adds; a second pass doubles the gradient
    m.backward(feat, torch.as_tensor(g_out, device="cuda"), accumulate=True)
    np.testing.assert_allclose(m.grad(), 2 * g, rtol=1e-12)


@pytest.mark.parametrize("shape,omega_max", [((10, 9, 8), 1.0), ((7, 6, 5), 1.0),
                                             ((7, 6, 5), 1.9)])
def test_tensor_core_forward_matches_oracle(amg, orc, lm, shape, omega_max):
    # FP16 operands keep 10 mantissa bits: omega within 3e-3 of the FP64 network
    # (210 rows: a ragged last tile of 16)
    A = _problem(shape)
    n = shape[0] * shape[1] * shape[2]
    m = lm.Mlp(2, omega_max)
    p = (0.5 * standard_normal(23, m.nparam)).astype(np.float32)
    p[-1] = 1.0
    m.set_params(p)
    feat = m.features(amg.csr_to_device(A), shape)
    om = m.forward(feat).cpu().numpy()
    om_o, _ = orc.mlp_forward(p.astype(np.float64), feat.cpu().numpy().astype(np.float64),
                              omega_max)
    err = np.abs(om - om_o).max()
    print("tensor-core forward: max |omega - omega_oracle| = %.2e over %d rows" % (err, n))
    assert err <= 3e-3
    assert om.min() > 0.0 and om.max() <= omega_max


def test_fast_gelu_error_bound(amg):
    # the tensor-core forward's GELU (erf by Abramowitz & Stegun 7.1.26, within
    # 1.5e-7 of erf) against the exact GELU in float64
    import ctypes as C

    from paper_2406_19754_gb300 import _lib

    u = torch.linspace(-9.0, 9.0, 200001, dtype=torch.float32, device="cuda")
    out = torch.empty_like(u)
    lib = _lib.load()
    assert lib.mlp_debug_gelu(C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()), u.numel(),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    ud = u.double().cpu()
    exact = torch.nn.functional.gelu(ud)
    err = (out.double().cpu() - exact).abs() / ud.abs().clamp(min=1.0)
    print("fast GELU: max |error| / max(1, |u|) = %.2e" % float(err.max()))
    assert float(err.max()) <= 3e-7


@pytest.mark.parametrize("omega_max", [1.5, 1.9])
def test_forward_backward_with_omega_cap(amg, orc, lm, omega_max):
    # omega = max(omega_max sigmoid(z), 1e-3): the over-relaxing form of the network
    A, shape = _problem(), (10, 9, 8)
    n = 720
    m = lm.Mlp(4, omega_max)
    m.set_exact_forward(True)
    p = (0.5 * standard_normal(22, m.nparam)).astype(np.float32)
    p[-1] = 3.0  # output bias: most rows above omega = 1
    m.set_params(p)
    feat = m.features(amg.csr_to_device(A), shape)
    om = m.forward(feat).cpu().numpy()
    f64 = feat.cpu().numpy().astype(np.float64)
    om_o, _ = orc.mlp_forward(p.astype(np.float64), f64, omega_max)
    np.testing.assert_allclose(om, om_o, rtol=2e-5, atol=1e-6)
    assert om.max() > 1.0 and om.max() < omega_max
    g_out = (uniform01(6, n) - 0.5).astype(np.float32)
    m.backward(feat, torch.as_tensor(g_out, device="cuda"), accumulate=False)
    g_o = orc.mlp_backward(p.astype(np.float64), f64, g_out.astype(np.float64), omega_max)
    assert np.linalg.norm(m.grad() - g_o) <= 1e-5 * np.linalg.norm(g_o)


def test_omega_cap_checked(amg, lm):
    from paper_2406_19754_gb300 import _lib

    m = lm.Mlp(0)
    for bad in (0.5, 2.0, float("nan")):
        assert m._lib.mlp_set_omega_max(m.h, bad) == _lib.AMG_ERR_ARG
    assert m._lib.mlp_set_omega_max(m.h, 1.9) == 0


def test_adam_matches_oracle(amg, orc, lm):
    m = lm.Mlp(2)
    p0 = m.params().astype(np.float64)
    po, mo, vo = p0.copy(), np.zeros(m.nparam), np.zeros(m.nparam)
    A, shape = _problem((6, 6, 6)), (6, 6, 6)
    feat = m.features(amg.csr_to_device(A), shape)
    for t in range(1, 4):
        g_out = torch.as_tensor((uniform01(30 + t, 216) - 0.3).astype(np.float32), device="cuda")
        m.backward(feat, g_out, accumulate=False)
        g = m.grad()
        m.adam(lr=1e-2, grad_scale=0.5)
        orc.mlp_adam(po, 0.5 * g, mo, vo, t, lr=1e-2)
        # the oracle follows the float32 parameters the GPU uses for the next gradient
        np.testing.assert_allclose(m.params(), po, rtol=1e-6, atol=1e-7)
        po = m.params().astype(np.float64)


@pytest.mark.parametrize("max_coarse", [10 ** 6, 20])
def test_twogrid_loss_matches_oracle(amg, orc, lm, max_coarse):
    # max_coarse large: level 1 is the coarsest (exact coarse solve);
    # small: A_1^-1 by inner PCG-AMG to 1e-12
    A = _problem((12, 11, 10))
    n = 1320
    Ad = amg.csr_to_device(A)
    H = amg.Hierarchy(*Ad, max_coarse=min(max_coarse, 400))
    assert H.levels >= 2
    om = (0.2 + 0.8 * uniform01(4, n)).astype(np.float32)
    H.set_smoother_weights(torch.as_tensor(om, device="cuda"))
    e0 = standard_normal(9, 3 * n).reshape(3, n)
    loss, dom = lm.twogrid_loss(H, torch.as_tensor(e0, device="cuda"), 2)
    Ho = orc.Hierarchy(A, max_coarse=1)
    agg, Ac = Ho.level_agg(0), Ho.level_csr(1)
    loss_o, dom_o = orc.twogrid_loss(A, agg, Ac, om.astype(np.float64), e0, K=2)
    tol = 1e-12 if H.levels == 2 else 1e-9
    assert abs(loss - loss_o) <= tol * abs(loss_o)
    np.testing.assert_allclose(dom.cpu().numpy(), dom_o, rtol=2e-6,
                               atol=1e-6 * np.abs(dom_o).max())


def test_training_steps_reduce_loss(amg, lm):
    # repeated Adam steps on one problem must lower its two-grid loss
    A, shape = _problem((12, 12, 12), 2.5, 7), (12, 12, 12)
    Ad = amg.csr_to_device(A)
    m = lm.Mlp(3)
    e0 = torch.as_tensor(standard_normal(11, 2 * 1728).reshape(2, 1728), device="cuda")
    losses = []
    for _ in range(25):
        H = amg.Hierarchy(*Ad)
        feat = m.features(Ad, shape)
        H.set_smoother_weights(m.forward(feat))
        loss, dom = lm.twogrid_loss(H, e0, 2)
        m.backward(feat, dom, accumulate=False)
        m.adam(lr=3e-2)
        losses.append(loss)
    assert min(losses[-5:]) < losses[0] - 1e-3


def test_trained_network_against_plain_smoother(amg, lm):
    """The committed network (trained on 4000 generated 48^3 problems) on
    held-out problems: its two-grid loss and PCG iterations against plain
    l1-Jacobi (omega = 1) on the same hierarchy.  Within omega in (0, 1] the
    training drives omega to 1, so the network may not lose to the plain
    smoother; the measured difference is printed."""
    from synthetic import diffusion_problem

    m = lm.Mlp(0)
    m.load(lm.DEFAULT_WEIGHTS)
    side = 40
    n = side ** 3
    for sigma, seed in ((2.5, 5), (1.0, 77)):
        Ad = amg.csr_to_device(diffusion_problem(side, sigma, 8.0, seed))
        H = amg.Hierarchy(*Ad)
        e0 = torch.as_tensor(standard_normal(seed + 7919, 4 * n).reshape(4, n), device="cuda")
        b = torch.as_tensor(uniform01(seed + 1, n), device="cuda")
        loss_p, _ = lm.twogrid_loss(H, e0, 2, gradient=False)
        _, ip = H.pcg(b, tol=1e-8)
        om = m.forward(m.features(Ad, (side, side, side)))
        assert float(om.min()) > 0.0 and float(om.max()) <= 1.0
        H.set_smoother_weights(om)
        loss_l, _ = lm.twogrid_loss(H, e0, 2, gradient=False)
        _, il = H.pcg(b, tol=1e-8)
        print("sigma %.1f: two-grid loss plain %.5f learned %.5f; PCG iterations plain %d "
              "learned %d; mean omega %.5f" % (sigma, loss_p, loss_l, ip["iterations"],
                                              il["iterations"], float(om.mean())))
        assert loss_l <= loss_p + 1e-3 * abs(loss_p)
        assert il["iterations"] <= ip["iterations"] + 1


def test_over_relaxing_network_against_plain_smoother(amg, lm):
    """The network trained with the output cap omega_max = 1.9 (the same 4000
    problems; omega may exceed 1) on held-out problems: two-grid loss and PCG
    iterations against plain l1-Jacobi and against the constant omega equal
    to the network's mean.  The two-grid loss the network was trained on must
    improve clearly; PCG iterations must not get worse; all numbers are
    printed."""
    from synthetic import diffusion_problem

    m = lm.Mlp(0, 1.9)
    m.load(lm.weights_path(1.9))
    side = 40
    n = side ** 3
    for sigma, seed in ((2.5, 5), (1.0, 77), (0.0, 78)):
        Ad = amg.csr_to_device(diffusion_problem(side, sigma, 8.0, seed))
        H = amg.Hierarchy(*Ad)
        e0 = torch.as_tensor(standard_normal(seed + 7919, 4 * n).reshape(4, n), device="cuda")
        b = torch.as_tensor(uniform01(seed + 1, n), device="cuda")
        loss_p, _ = lm.twogrid_loss(H, e0, 2, gradient=False)
        _, ip = H.pcg(b, tol=1e-8)
        om = m.forward(m.features(Ad, (side, side, side)))
        assert float(om.min()) > 0.0 and float(om.max()) < 1.9
        H.set_smoother_weights(om)
        loss_l, _ = lm.twogrid_loss(H, e0, 2, gradient=False)
        _, il = H.pcg(b, tol=1e-8)
        H.set_smoother_weights(torch.full_like(om, float(om.mean())))
        loss_c, _ = lm.twogrid_loss(H, e0, 2, gradient=False)
        _, ic = H.pcg(b, tol=1e-8)
        print("cap 1.9, sigma %.1f: two-grid loss plain %.5f learned %.5f constant %.5f; PCG "
              "iterations plain %d learned %d constant %d; omega mean %.4f min %.4f max %.4f"
              % (sigma, loss_p, loss_l, loss_c, ip["iterations"], il["iterations"],
                 ic["iterations"], float(om.mean()), float(om.min()), float(om.max())))
        assert loss_l < loss_p - 0.05 * abs(loss_p)
        assert il["iterations"] <= ip["iterations"]
