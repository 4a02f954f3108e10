"""Coefficient updates on an assembled hierarchy (amg_update_values) against
the oracle's rebuild on the same aggregates."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu

SHAPE = (22, 20, 18)
N = 22 * 20 * 18


def _two():
    A1 = diffusion3d(np.exp(gaussian_field(SHAPE, 1.0, 3.0, 31)))
    A2 = diffusion3d(np.exp(gaussian_field(SHAPE, 2.5, 4.0, 32)))
    return A1, A2


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_update_matches_oracle_rebuild(amg, orc, precision):
    A1, A2 = _two()
    H = amg.Hierarchy(*amg.csr_to_device(A1), max_coarse=40, precision=precision)
    Ho = orc.Hierarchy(A1, max_coarse=40)
    H.update_values(*amg.csr_to_device(A2))
    R = Ho.reuse(A2)
    assert R.status == 0 and H.levels == R.levels
    for l in range(1, H.levels):
        got = H.level_export(l)
        rp, ci, v = R.level_csr(l)
        assert np.array_equal(got["rowptr"].cpu().numpy(), rp)
        assert np.array_equal(got["col"].cpu().numpy(), ci)
        assert np.array_equal(got["val"].cpu().numpy(), v)  # bit for bit
    b = uniform01(4, N)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-8)
    _, io = orc.pcg(A2, b, tol=1e-8, hier=R, beta_form=1 if precision == "f32" else 0)
    assert info["status"] == 0 and abs(info["iterations"] - io["iterations"]) <= 1
    if precision == "f64":
        z = H.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
        zo = R.vcycle(b)
        assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


def test_update_with_the_same_values_changes_nothing(amg):
    A1, _ = _two()
    Ad = amg.csr_to_device(A1)
    H = amg.Hierarchy(*Ad)
    b = torch.as_tensor(uniform01(5, N), device="cuda")
    x0, i0 = H.pcg(b, tol=1e-9)
    z0 = H.vcycle(b)
    H.update_values(*Ad)
    assert torch.equal(H.vcycle(b), z0)
    x1, i1 = H.pcg(b, tol=1e-9)  # graphs captured before the update are rebuilt
    assert i0["iterations"] == i1["iterations"] and torch.equal(x0, x1)


def test_update_rejects_another_pattern(amg):
    H = amg.Hierarchy(*amg.csr_to_device(poisson3d(12, 10, 8)))
    b = torch.as_tensor(uniform01(6, 960), device="cuda")
    z0 = H.vcycle(b)
    for other in (poisson3d(10, 12, 8), poisson3d(12, 10, 9)):
        with pytest.raises(amg.AmgError):
            H.update_values(*amg.csr_to_device(other))
    assert torch.equal(H.vcycle(b), z0)  # unchanged after a rejected update
