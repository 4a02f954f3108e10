"""V(nu, nu) cycles, the variable V-cycle and the PCG coarsest solver (the
VBM / VMATCH choices of Sec. 3) against the oracle.

The GPU steps the residual recurrence r' = r - (A S) r between sweeps where
the oracle recomputes b - A x, so V-cycle outputs agree to rounding (1e-11
relative), not bit for bit."""

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d, uniform01

pytestmark = pytest.mark.gpu


def _pair(amg, orc, A, coarse="cholesky", **cyc):
    gpu = dict(smooth_sweeps=cyc.get("nu0", 1), variable_cycle=int(cyc.get("variable", False)),
               coarse_solver=1 if coarse == "pcg" else 0,
               coarse_maxit=cyc.get("maxit", 40), coarse_tol=cyc.get("tol", 1e-4))
    H = amg.Hierarchy(*amg.csr_to_device(A), sweeps=cyc.get("sweeps", 2),
                      max_coarse=cyc.get("max_coarse", 200), max_levels=cyc.get("max_levels", 30),
                      precision=cyc.get("precision", "f64"), **gpu)
    Ho = orc.Hierarchy(A, sweeps=cyc.get("sweeps", 2), max_coarse=cyc.get("max_coarse", 200),
                       max_levels=cyc.get("max_levels", 30), smooth_sweeps=cyc.get("nu0", 1),
                       variable=cyc.get("variable", False), coarse=coarse,
                       coarse_maxit=cyc.get("maxit", 40), coarse_tol=cyc.get("tol", 1e-4))
    return H, Ho


@pytest.mark.parametrize("nu0,variable,sweeps", [(2, False, 2), (3, False, 2), (1, True, 2),
                                                 (2, True, 3), (2, True, 2)])
def test_sweeps_vcycle_matches_oracle(amg, orc, nu0, variable, sweeps):
    A = diffusion3d(np.exp(gaussian_field((20, 18, 16), 1.5, 3.0, 17)))
    n = 20 * 18 * 16
    H, Ho = _pair(amg, orc, A, nu0=nu0, variable=variable, sweeps=sweeps, max_coarse=30)
    assert H.levels == Ho.levels >= 3
    r = uniform01(5, n) - 0.4
    z = H.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    _, recs = H.vcycle_profile(torch.as_tensor(r, device="cuda"))
    nsweep = sum(1 for x in recs if x["kind"] == "sweep")
    # levels from the persistent small-level launch on sweep inside it
    tail = [x["level"] for x in recs if x["kind"] == "tail"]
    lt = tail[0] if tail else H.levels - 1
    nus = [nu0 * 2 ** l if variable else nu0 for l in range(lt)]
    assert nsweep == sum(2 * (nu - 1) for nu in nus)


@pytest.mark.parametrize("maxit", [1, 4, 25])
def test_pcg_coarse_solver_matches_oracle(amg, orc, maxit):
    # one level: the V-cycle is the coarsest solve; tol 0 runs maxit iterations
    A = diffusion3d(np.exp(gaussian_field((9, 8, 7), 1.0, 2.0, 3)))
    n = 9 * 8 * 7
    H, Ho = _pair(amg, orc, A, coarse="pcg", max_levels=1, maxit=maxit, tol=0.0)
    assert H.levels == 1
    b = uniform01(2, n)
    z = H.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(b)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)


def test_pcg_coarse_in_a_hierarchy(amg, orc):
    A = poisson3d(20)
    n = 20 ** 3
    H, Ho = _pair(amg, orc, A, coarse="pcg", max_coarse=150, maxit=12, tol=0.0, nu0=2)
    assert H.levels == Ho.levels >= 3
    b = uniform01(8, n)
    z = H.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
    zo = Ho.vcycle(b)
    assert np.linalg.norm(z - zo) <= 1e-11 * np.linalg.norm(zo)
    assert not torch.any(H.vcycle(torch.zeros(n, dtype=torch.float64, device="cuda")))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_vmatch_configuration_solves(amg, orc, precision):
    """Aggregates <= 8, variable V-cycle from 2 sweeps, PCG-l1 coarsest solve
    (<= 40 iterations, 1e-4), flexible CG to 1e-6 on b = 1 (Sec. 3)."""
    A = poisson3d(40)
    n = 40 ** 3
    cyc = dict(nu0=2, variable=True, sweeps=3, maxit=40, tol=1e-4, precision=precision)
    H, Ho = _pair(amg, orc, A, coarse="pcg", **cyc)
    b = np.ones(n)
    x, info = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-6, beta_form="flexible")
    _, io = orc.pcg(A, b, tol=1e-6, hier=Ho, beta_form=1)
    assert info["status"] == 0 and info["true_relres"] <= 1.1e-6
    slack = 1 if precision == "f64" else 2
    assert abs(info["iterations"] - io["iterations"]) <= slack
    assert H.operator_complexity() == pytest.approx(Ho.operator_complexity(), rel=1e-12)


def test_batch_with_sweeps(amg, orc):
    systems = [poisson3d(12, 10, 9), diffusion3d(np.exp(gaussian_field((14, 12, 10), 1.2, 3.0, 6)))]
    A, offs = orc.block_diag(systems)
    H = amg.BatchHierarchy([amg.csr_to_device(S) for S in systems], max_coarse=30,
                           smooth_sweeps=2)
    Ho = orc.Hierarchy(A, max_coarse=30, systems=offs, smooth_sweeps=2)
    b = uniform01(3, offs[-1])
    x, st = H.pcg(torch.as_tensor(b, device="cuda"), tol=1e-8)
    for k in range(len(systems)):
        _, io = orc.pcg_block(Ho, offs[k], offs[k + 1], b[offs[k]:offs[k + 1]], tol=1e-8)
        assert st[k]["status"] == 0 and abs(st[k]["iterations"] - io["iterations"]) <= 1


def test_cycle_options_checked(amg):
    Ad = amg.csr_to_device(poisson3d(8))
    for bad in (dict(smooth_sweeps=0), dict(smooth_sweeps=9), dict(variable_cycle=2),
                dict(coarse_solver=2), dict(coarse_maxit=-1), dict(coarse_tol=-1.0)):
        with pytest.raises(amg.AmgError):
            amg.Hierarchy(*Ad, **bad)
    with pytest.raises(amg.AmgError):  # the PCG coarsest solve is for one system
        amg.BatchHierarchy([Ad, Ad], coarse_solver=1)
