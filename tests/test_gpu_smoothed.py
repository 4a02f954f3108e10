"""Smoothed prolongators on the GPU (Sec. 2.3, SMATCH) against the oracle.

P = (I - w D^-1 A) P_hat, A P and the coarse matrices P^T (A P) sum every
entry in ascending inner index with separately rounded products and sums on
both sides, so prolongators and level matrices agree bit for bit; the
V-cycle (SELL sums, the residual recurrence between sweeps) agrees to
rounding (1e-11 relative)."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu


def _pair(amg, orc, A, sweeps=2, max_coarse=40, nu0=1, coarse="cholesky", pfilter=0.0,
          **extra):
    H = amg.Hierarchy(*amg.csr_to_device(A), sweeps=sweeps, max_coarse=max_coarse,
                      smooth_sweeps=nu0, coarse_solver=1 if coarse == "pcg" else 0,
                      smooth_prolongator=1, prolongator_filter=pfilter, **extra)
    Ho = orc.Hierarchy(A, sweeps=sweeps, max_coarse=max_coarse, smooth_sweeps=nu0,
                       coarse=coarse, smoothed=True, pfilter=pfilter)
    return H, Ho


def _same_levels(H, Ho):
    assert H.levels == Ho.levels
    for l in range(H.levels - 1):
        (rp, ci, v), w = H.level_prolongator(l)
        (orp, oci, ov), ow = Ho.level_prolongator(l)
        assert w == ow
        assert np.array_equal(rp.cpu().numpy(), orp)
        assert np.array_equal(ci.cpu().numpy(), oci)
        assert np.array_equal(v.cpu().numpy(), ov)  # bit for bit
    for l in range(1, H.levels):
        got = H.level_export(l)
        rp, ci, v = Ho.level_csr(l)
        assert np.array_equal(got["rowptr"].cpu().numpy(), rp)
        assert np.array_equal(got["col"].cpu().numpy(), ci)
        assert np.array_equal(got["val"].cpu().numpy(), v)


@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_prolongators_and_coarse_matrices_bitwise(amg, orc, sweeps):
    A = diffusion3d(np.exp(gaussian_field((22, 20, 18), 1.5, 3.0, 41)))
    H, Ho = _pair(amg, orc, A, sweeps=sweeps)
    assert H.levels >= 3
    _same_levels(H, Ho)


@pytest.mark.parametrize("pfilter", [0.02, 0.08])
def test_filtered_smoothing_bitwise(amg, orc, pfilter):
    # P smoothed with A_F (weak entries lumped into the diagonal)
    A = diffusion3d(np.exp(gaussian_field((22, 20, 18), 2.5, 2.0, 43)))
    H, Ho = _pair(amg, orc, A, sweeps=2, pfilter=pfilter)
    assert H.levels >= 3
    _same_levels(H, Ho)
    r = uniform01(9, 22 * 20 * 18) - 0.5
    z = H.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)


def test_filtered_smatch_solves(amg, orc):
    A = poisson3d(40)
    b = np.ones(40 ** 3)
    H, Ho = _pair(amg, orc, A, sweeps=3, max_coarse=200, nu0=4, coarse="pcg", pfilter=0.01)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, beta_form="flexible")
    _, io = orc.pcg(A, b, tol=1e-6, hier=Ho, beta_form=1)
    assert info["status"] == 0 and info["true_relres"] <= 1.1e-6
    assert abs(info["iterations"] - io["iterations"]) <= 1
    assert H.operator_complexity() == pytest.approx(Ho.operator_complexity(), rel=1e-15)


def _bitwise_unsymmetric(side, seed):
    """poisson3d(side) with the entries below the diagonal scaled by
    1 + 1e-3 u: symmetric pattern, values that differ across the diagonal
    (as in a smoothed coarse matrix, at a larger scale)."""
    rp, ci, v = poisson3d(side)
    v = v.copy()
    u = uniform01(seed, len(v))
    for i in range(len(rp) - 1):
        for e in range(rp[i], rp[i + 1]):
            if ci[e] < i:
                v[e] *= 1.0 + 1e-3 * u[e]
    return rp, ci, v


def test_matching_reads_each_edge_from_its_upper_row(amg, orc):
    # the oracle takes edge {i, j}'s value from row min(i, j); so must the GPU
    A = _bitwise_unsymmetric(14, 12)
    mate, _ = amg.pairwise_match(*amg.csr_to_device(A))
    assert np.array_equal(mate.cpu().numpy(), orc.match(A))


def test_wide_coarse_rows_bitwise(amg, orc):
    # level 3 of 64^3 with aggregates <= 8 has rows of more than 512 distinct
    # columns: the products take the large-table path
    A = poisson3d(64)
    H, Ho = _pair(amg, orc, A, sweeps=3, max_coarse=200)
    rp, _, _ = Ho.level_csr(3)
    assert np.diff(rp).max() > 512
    _same_levels(H, Ho)


@pytest.mark.parametrize("nu0,coarse", [(1, "cholesky"), (2, "cholesky"), (4, "pcg"),
                                        (3, "cholesky")])
def test_smoothed_vcycle_matches_oracle(amg, orc, nu0, coarse):
    A = diffusion3d(np.exp(gaussian_field((20, 18, 16), 1.5, 3.0, 17)))
    n = 20 * 18 * 16
    H, Ho = _pair(amg, orc, A, sweeps=3, max_coarse=30, nu0=nu0, coarse=coarse)
    assert H.levels == Ho.levels >= 3
    r = uniform01(5, n) - 0.4
    z = H.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    # every level restricts through R = P^T and prolongs through P
    _, recs = H.vcycle_profile(torch.as_tensor(r, device="cuda"))
    assert not any(x["kind"] == "tail" for x in recs)
    assert sum(1 for x in recs if x["kind"] == "restrict") == H.levels - 1


def test_smatch_configuration_solves(amg, orc):
    """Aggregates <= 8, smoothed P, 4 l1-Jacobi sweeps, PCG-l1 coarsest solve
    (<= 40 iterations), flexible CG to 1e-6 on b = 1."""
    A = poisson3d(40)
    n = 40 ** 3
    H, Ho = _pair(amg, orc, A, sweeps=3, max_coarse=200, nu0=4, coarse="pcg")
    b = np.ones(n)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, beta_form="flexible")
    _, io = orc.pcg(A, b, tol=1e-6, hier=Ho, beta_form=1)
    assert info["status"] == 0 and info["true_relres"] <= 1.1e-6
    assert abs(info["iterations"] - io["iterations"]) <= 1
    assert H.operator_complexity() == pytest.approx(Ho.operator_complexity(), rel=1e-15)
    # every graph mode gives the same iterate
    x2, i2 = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, beta_form="flexible",
                   use_graph=False)
    assert i2["iterations"] == info["iterations"] and torch.equal(x, x2)


@pytest.mark.parametrize("agg,extra", [("matching", dict(sweeps=3)),
                                       ("vbm", dict()),
                                       ("matching", dict(sweeps=3, bf16_from_level=2))])
def test_fp32_vcycle_solves(amg, orc, agg, extra):
    """SMATCH / VBM with the V-cycle in FP32 (BF16 values below level 2 as an
    option), FCG in FP64: same convergence as the FP64 oracle within 2
    iterations, and the FP32 V-cycle within FP32 rounding of the oracle's."""
    A = poisson3d(40)
    n = 40 ** 3
    H = amg.Hierarchy(*amg.csr_to_device(A), aggregation=agg, smooth_prolongator=1,
                      smooth_sweeps=4, coarse_solver=1, precision="f32", **extra)
    Ho = orc.Hierarchy(A, aggregation=agg, smoothed=True, smooth_sweeps=4, coarse="pcg",
                       sweeps=extra.get("sweeps", 2))
    b = np.ones(n)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, beta_form="flexible")
    _, io = orc.pcg(A, b, tol=1e-6, hier=Ho, beta_form=1)
    assert info["status"] == 0 and info["true_relres"] <= 1.1e-6
    assert abs(info["iterations"] - io["iterations"]) <= 2
    if "bf16_from_level" not in extra:
        r = uniform01(7, n) - 0.4
        z = H.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
        zo = Ho.vcycle(r)
        assert np.linalg.norm(z - zo) <= 1e-4 * np.linalg.norm(zo)


def test_update_values_recomputes_the_prolongators(amg, orc):
    shape = (22, 20, 18)
    A1 = diffusion3d(np.exp(gaussian_field(shape, 1.0, 3.0, 31)))
    A2 = diffusion3d(np.exp(gaussian_field(shape, 2.5, 4.0, 32)))
    H, Ho = _pair(amg, orc, A1, sweeps=2)
    H.update_values(*amg.csr_to_device(A2))
    R = Ho.reuse(A2)
    assert R.status == 0
    _same_levels(H, R)
    b = uniform01(4, A1[0].size - 1)
    z = H.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
    zo = R.vcycle(b)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)


def test_smoothed_layouts_and_limits(amg):
    Ad = amg.csr_to_device(poisson3d(16))
    H = amg.Hierarchy(*Ad, sweeps=2, max_coarse=40, smooth_prolongator=1)
    n0, _ = H.level_info(0)
    n1, _ = H.level_info(1)
    lp = H.level_layout(0, 2)
    lr = H.level_layout(0, 3)
    assert lp["slice_height"] == H.level_layout(0, 1)["slice_height"]
    assert lp["slots"] >= H.level_prolongator(0)[0][1].numel()
    assert lr["slots"] >= H.level_prolongator(0)[0][1].numel()
    b = torch.ones(n0, dtype=torch.float64, device="cuda")
    with pytest.raises(amg.AmgError):  # several right-hand sides: not implemented
        H.vcycle_multi(torch.ones((n0, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(amg.AmgError):
        H.level_prolongator(H.levels - 1)
    with pytest.raises(amg.AmgError):
        amg.Hierarchy(*Ad, smooth_prolongator=1, autotune=1)
    with pytest.raises(amg.AmgError):
        amg.Hierarchy(*Ad, smooth_prolongator=2)
    with pytest.raises(amg.AmgError):
        amg.BatchHierarchy([Ad, Ad], smooth_prolongator=1)
    with pytest.raises(amg.AmgError):  # P of a hierarchy without smoothing
        amg.Hierarchy(*Ad).level_prolongator(0)
    assert H.pcg(b, tol=1e-8)[1]["status"] == 0
    assert n1 < n0
