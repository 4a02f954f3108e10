"""Large coarsest levels (blocked multi-kernel Cholesky and the two-phase
coarse solve) against the oracle's textbook Cholesky."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import dense

pytestmark = pytest.mark.gpu


def test_single_level_large_dense_solve(amg, orc):
    A = diffusion3d(np.exp(gaussian_field((11, 12, 13), 1.0, 3.0, 4)))  # 1716 rows, one level
    n = 11 * 12 * 13
    H = amg.Hierarchy(*amg.csr_to_device(A), max_coarse=2000)
    assert H.levels == 1
    b = uniform01(6, n)
    z = H.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(z, orc.Hierarchy(A, max_coarse=2000).vcycle(b), rtol=1e-12,
                               atol=1e-14)
    np.testing.assert_allclose(z, np.linalg.solve(dense(A), b), rtol=1e-10)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_large_coarsest_level_in_vcycle_and_pcg(amg, orc, precision):
    A = poisson3d(24)  # level 1 has 3456 rows and is the coarsest
    n = 24 ** 3
    H = amg.Hierarchy(*amg.csr_to_device(A), max_coarse=4000, precision=precision)
    Ho = orc.Hierarchy(A, max_coarse=4000)
    assert H.levels == Ho.levels == 2 and H.level_info(1)[0] > 1024
    r = uniform01(9, n)
    if precision == "f64":
        z = H.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
        zo = Ho.vcycle(r)
        assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    R = torch.as_tensor(np.stack([r, 2 * r + 1], axis=1), device="cuda")
    Z = H.vcycle_multi(R)
    for c in range(2):
        assert torch.equal(Z[:, c], H.vcycle(R[:, c].contiguous()))
    x, info = H.pcg(torch.as_tensor(r, device="cuda"), tol=1e-8)
    _, io = orc.pcg(A, r, tol=1e-8, hier=Ho)
    assert info["status"] == 0 and abs(info["iterations"] - io["iterations"]) <= 1
