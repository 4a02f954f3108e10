"""Decoupled Vanek-Mandel-Brezina aggregation on the GPU (Sec. 2.3, VBM)
against the oracle.  The phase-1 roots come out of parallel rounds whose
decisions depend only on smaller rows, so aggregates, level matrices and
prolongators are bit-identical to the oracle's sequential pass; V-cycles agree
to rounding (1e-11 relative)."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01
from tests.helpers import from_dense, random_spd_graph

pytestmark = pytest.mark.gpu


def _aniso2d(nx, ny, eps):
    n = nx * ny
    M = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            i = y * nx + x
            M[i, i] = 2.0 + 2.0 * eps
            for dx, c in ((-1, 1.0), (1, 1.0)):
                if 0 <= x + dx < nx:
                    M[i, i + dx] = -c
            for dy in (-1, 1):
                if 0 <= y + dy < ny:
                    M[i, i + dy * nx] = -eps
    return from_dense(M)


CASES = [
    ("poisson20", lambda: poisson3d(20), 0.01),
    ("poisson_box", lambda: poisson3d(23, 17, 11), 0.2),
    ("diffusion", lambda: diffusion3d(np.exp(gaussian_field((24, 20, 18), 2.0, 3.0, 5))), 0.05),
    ("diffusion_strong", lambda: diffusion3d(np.exp(gaussian_field((20, 20, 20), 2.5, 2.0, 6))),
     0.15),
    ("aniso2d", lambda: _aniso2d(40, 30, 0.01), 0.25),
    ("random", lambda: random_spd_graph(400, 0.02, 7), 0.1),
    ("random_mixed", lambda: random_spd_graph(300, 0.03, 8, positive_offdiag=True), 0.05),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_level0_aggregates_bitwise(amg, orc, case):
    _, make, theta = case
    A = make()
    H = amg.Hierarchy(*amg.csr_to_device(A), aggregation="vbm", vbm_theta=theta, max_coarse=10,
                      max_levels=2)
    want, nc = orc.vbm_aggregate(A, theta=theta)
    if H.levels == 1:  # coarsening stalled: the oracle must find the same
        assert nc > 0.9 * (len(A[0]) - 1)
        return
    assert H.level_info(1)[0] == nc
    assert np.array_equal(H.level_export(0)["agg"].cpu().numpy(), want)


@pytest.mark.parametrize("smoothed", [False, True])
def test_hierarchy_bitwise(amg, orc, smoothed):
    A = diffusion3d(np.exp(gaussian_field((26, 22, 20), 1.5, 3.0, 9)))
    kw = dict(max_coarse=30)
    H = amg.Hierarchy(*amg.csr_to_device(A), aggregation="vbm", smooth_prolongator=int(smoothed),
                      **kw)
    Ho = orc.Hierarchy(A, aggregation="vbm", smoothed=smoothed, **kw)
    assert H.levels == Ho.levels >= 3
    for l in range(H.levels):
        ex = H.level_export(l)
        if l > 0:
            rp, ci, v = Ho.level_csr(l)
            assert np.array_equal(ex["rowptr"].cpu().numpy(), rp)
            assert np.array_equal(ex["col"].cpu().numpy(), ci)
            assert np.array_equal(ex["val"].cpu().numpy(), v)
        if l + 1 < H.levels:
            assert np.array_equal(ex["agg"].cpu().numpy(), Ho.level_agg(l))
            if smoothed:
                (prp, pci, pv), w = H.level_prolongator(l)
                (orp, oci, ov), ow = Ho.level_prolongator(l)
                assert w == ow and np.array_equal(pv.cpu().numpy(), ov)
    n = len(A[0]) - 1
    r = uniform01(3, n) - 0.3
    z = H.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)


def test_vbm_configuration_solves(amg, orc):
    """VBM (Sec. 3): VBM aggregation, smoothed prolongators, 4 l1-Jacobi sweeps,
    PCG-l1 coarsest solve (<= 40 iterations), FCG to 1e-6 on b = 1."""
    A = poisson3d(40)
    n = 40 ** 3
    H = amg.Hierarchy(*amg.csr_to_device(A), aggregation="vbm", smooth_prolongator=1,
                      smooth_sweeps=4, coarse_solver=1)
    Ho = orc.Hierarchy(A, aggregation="vbm", smoothed=True, smooth_sweeps=4, coarse="pcg")
    b = np.ones(n)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, beta_form="flexible")
    _, io = orc.pcg(A, b, tol=1e-6, hier=Ho, beta_form=1)
    assert info["status"] == 0 and info["true_relres"] <= 1.1e-6
    assert abs(info["iterations"] - io["iterations"]) <= 1
    assert H.operator_complexity() == pytest.approx(Ho.operator_complexity(), rel=1e-15)


def test_unsmoothed_vbm_with_the_persistent_tail(amg):
    # the small-level launch restricts through the (wider) member tables
    A = poisson3d(36, 30, 28)
    Ad = amg.csr_to_device(A)
    H = amg.Hierarchy(*Ad, aggregation="vbm", tail_rows=4096)
    H0 = amg.Hierarchy(*Ad, aggregation="vbm", tail_rows=0)
    r = torch.as_tensor(uniform01(2, len(A[0]) - 1), device="cuda")
    assert torch.equal(H.vcycle(r), H0.vcycle(r))
    _, recs = H.vcycle_profile(r)
    assert any(x["kind"] == "tail" for x in recs)


def test_batched_vbm_matches_single_systems(amg, orc):
    systems = [poisson3d(14, 12, 10),
               diffusion3d(np.exp(gaussian_field((16, 14, 12), 1.2, 3.0, 4)))]
    Hb = amg.BatchHierarchy([amg.csr_to_device(S) for S in systems], aggregation="vbm",
                            max_coarse=30)
    offs = [0]
    for S in systems:
        offs.append(offs[-1] + len(S[0]) - 1)
    b = uniform01(6, offs[-1])
    _, st = Hb.pcg(torch.as_tensor(b, device="cuda"), tol=1e-8)
    for k, S in enumerate(systems):
        Ho = orc.Hierarchy(S, aggregation="vbm", max_coarse=30)
        _, io = orc.pcg(S, b[offs[k]:offs[k + 1]], tol=1e-8, hier=Ho)
        assert st[k]["status"] == 0 and abs(st[k]["iterations"] - io["iterations"]) <= 1


def test_vbm_options_checked(amg):
    Ad = amg.csr_to_device(poisson3d(8))
    for bad in (dict(aggregation=2), dict(aggregation="vbm", vbm_theta=1.0),
                dict(aggregation="vbm", vbm_theta=-0.1)):
        with pytest.raises(amg.AmgError):
            amg.Hierarchy(*Ad, **bad)


def test_update_values_on_a_vbm_hierarchy(amg, orc):
    # new coefficients, the VBM aggregates kept: bit-identical to the oracle's rebuild
    shape = (22, 20, 18)
    A1 = diffusion3d(np.exp(gaussian_field(shape, 1.0, 3.0, 51)))
    A2 = diffusion3d(np.exp(gaussian_field(shape, 2.0, 3.0, 52)))
    for smoothed in (False, True):
        H = amg.Hierarchy(*amg.csr_to_device(A1), aggregation="vbm", max_coarse=30,
                          smooth_prolongator=int(smoothed))
        Ho = orc.Hierarchy(A1, aggregation="vbm", max_coarse=30, smoothed=smoothed)
        H.update_values(*amg.csr_to_device(A2))
        R = Ho.reuse(A2)
        assert R.status == 0 and H.levels == R.levels
        for l in range(1, H.levels):
            got = H.level_export(l)
            rp, ci, v = R.level_csr(l)
            assert np.array_equal(got["col"].cpu().numpy(), ci)
            assert np.array_equal(got["val"].cpu().numpy(), v)
        b = uniform01(8, len(A1[0]) - 1)
        z = H.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
        zo = R.vcycle(b)
        assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
