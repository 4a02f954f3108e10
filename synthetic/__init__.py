"""Seeded synthetic inputs shared by the CPU oracle and the GPU library.

This module only *creates inputs* (matrices, right-hand sides, coefficient
fields).  It holds none of the solver's arithmetic: no matching, no Galerkin
product, no smoothing and no Krylov step.  Both sides of every parity test
read the same arrays produced here.
"""

from .problems import (  # noqa: F401
    GAMMA,
    splitmix64,
    uniform01,
    standard_normal,
    poisson3d,
    diffusion3d,
    gaussian_field,
    diffusion_problem,
    batch_specs,
    csr_nnz_poisson3d,
)
