"""Problem generators: 7-point Poisson and variable-coefficient diffusion on
structured 3D grids, Gaussian random fields and uniform right-hand sides.

Numbering: a grid of ``nx * ny * nz`` cells stores cell ``(x, y, z)`` in row
``x + nx * (y + ny * z)`` (x fastest).  Every row lists its entries in
ascending column order: ``-z, -y, -x, diagonal, +x, +y, +z``.  The CSR arrays
are ``rowptr`` int64 (n + 1), ``col`` int32, ``val`` float64.

Poisson (Sec. 3 of the paper): the 7-point finite-difference Laplacian on
the unit cube with homogeneous Dirichlet data, scaled by h^2, so the diagonal
is 6 and every in-grid neighbour is -1; neighbours outside the grid are
dropped.

Diffusion, -div(k grad u): the coefficient between two neighbouring cells is
the harmonic mean 2 k_i k_j / (k_i + k_j); the face towards a Dirichlet
boundary uses k_i (the harmonic mean with a ghost cell of the same k); the
diagonal is the sum of the six face coefficients.  With k == 1 this is
exactly the Poisson matrix above.

Random numbers come from splitmix64 (Steele, Lea, Flood, OOPSLA 2014): the
i-th draw of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``.  Uniforms in
[0, 1) take the top 53 bits; normals use the Box-Muller transform.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset + count - 1`` of the splitmix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        return _mix(state)


def uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` float64 uniforms in [0, 1): (u >> 11) * 2^-53."""
    u = splitmix64(seed, count)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def standard_normal(seed: int, count: int) -> np.ndarray:
    """``count`` N(0, 1) draws by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = u[0::2]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))  # log(1 - u1), u1 < 1
    ang = 2.0 * math.pi * u2
    out = np.empty(2 * m, dtype=np.float64)
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:count]


def csr_nnz_poisson3d(nx: int, ny: int | None = None, nz: int | None = None) -> int:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    return 7 * n - 2 * (ny * nz + nx * nz + nx * ny)


def _stencil_csr(nx, ny, nz, off_vals, diag):
    """Assembles CSR from per-direction off-diagonal values.

    ``off_vals[d]`` (d = -z, -y, -x, +x, +y, +z) is an (nz, ny, nx) array of
    the entry towards that neighbour (ignored where the neighbour is outside
    the grid); ``diag`` is an (nz, ny, nx) array.
    """
    n = nx * ny * nz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    valid = [z > 0, y > 0, x > 0, None, x < nx - 1, y < ny - 1, z < nz - 1]
    step = [-nx * ny, -nx, -1, 0, 1, nx, nx * ny]
    rows = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    cols = np.empty((n, 7), dtype=np.int32)
    vals = np.empty((n, 7), dtype=np.float64)
    mask = np.empty((n, 7), dtype=bool)
    k = 0
    for d in range(7):
        cols[:, d] = (rows + step[d]).reshape(-1)
        if d == 3:
            vals[:, d] = diag.reshape(-1)
            mask[:, d] = True
        else:
            vals[:, d] = off_vals[k].reshape(-1)
            mask[:, d] = valid[d].reshape(-1)
            k += 1
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[mask]
    val = vals[mask]
    return rowptr, col, val


def poisson3d(nx: int, ny: int | None = None, nz: int | None = None):
    """7-point Poisson CSR (diag 6, neighbours -1, Dirichlet rows trimmed)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    shape = (nz, ny, nx)
    off = [np.full(shape, -1.0) for _ in range(6)]
    return _stencil_csr(nx, ny, nz, off, np.full(shape, 6.0))


def _harmonic(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (2.0 * (a * b)) / (a + b)


def diffusion3d(k: np.ndarray):
    """Variable-coefficient 7-point diffusion CSR from a cell field k (nz, ny, nx)."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    nz, ny, nx = k.shape
    # face coefficient towards each neighbour; boundary faces take k itself
    fmz = k.copy()
    fpz = k.copy()
    fmy = k.copy()
    fpy = k.copy()
    fmx = k.copy()
    fpx = k.copy()
    hz = _harmonic(k[:-1], k[1:])
    fpz[:-1] = hz
    fmz[1:] = hz
    hy = _harmonic(k[:, :-1], k[:, 1:])
    fpy[:, :-1] = hy
    fmy[:, 1:] = hy
    hx = _harmonic(k[:, :, :-1], k[:, :, 1:])
    fpx[:, :, :-1] = hx
    fmx[:, :, 1:] = hx
    diag = fmz + fmy + fmx + fpx + fpy + fpz
    off = [-fmz, -fmy, -fmx, -fpx, -fpy, -fpz]
    return _stencil_csr(nx, ny, nz, off, diag)


def gaussian_field(shape, sigma: float, ell: float, seed: int) -> np.ndarray:
    """Stationary Gaussian field with Cov(r) = sigma^2 exp(-r^2 / (2 ell^2)).

    White N(0, 1) noise on the grid padded by R = ceil(4 ell) cells per side is
    convolved separably with a Gaussian kernel of standard deviation
    ell / sqrt(2), normalised so that the 3D kernel has unit sum of squares
    (unit variance).  Returns an array of ``shape`` = (nz, ny, nx).
    """
    from scipy.ndimage import convolve1d

    nz, ny, nx = shape
    if sigma == 0.0:
        return np.zeros(shape, dtype=np.float64)
    s = ell / math.sqrt(2.0)
    R = int(math.ceil(4.0 * ell))
    t = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * s * s))
    g /= math.sqrt(float(np.sum(g * g)))
    P = (nz + 2 * R, ny + 2 * R, nx + 2 * R)
    f = standard_normal(seed, P[0] * P[1] * P[2]).reshape(P)
    f = convolve1d(f, g, axis=0, mode="constant")[R:R + nz]
    f = convolve1d(f, g, axis=1, mode="constant")[:, R:R + ny]
    f = convolve1d(f, g, axis=2, mode="constant")[:, :, R:R + nx]
    return sigma * np.ascontiguousarray(f)


def diffusion_problem(side: int, sigma: float, ell: float, seed: int):
    """Diffusion CSR with k = exp(g), g a Gaussian field (sigma, ell, seed)."""
    g = gaussian_field((side, side, side), sigma, ell, seed)
    return diffusion3d(np.exp(g))


def batch_specs(count: int, seed0: int, side_lo: int = 24, side_hi: int = 96,
                sigma_lo: float = 0.5, sigma_hi: float = 2.0):
    """Sides U{side_lo..side_hi} and sigmas U[sigma_lo, sigma_hi] for a batch.

    System ``s`` draws from stream ``seed0 + s``: draw 0 picks the side, draw 1
    sigma; its field uses that same seed.
    """
    specs = []
    for s in range(count):
        u = uniform01(seed0 + s, 2)
        side = side_lo + int(u[0] * (side_hi - side_lo + 1))
        sigma = sigma_lo + u[1] * (sigma_hi - sigma_lo)
        specs.append((side, float(sigma), seed0 + s))
    return specs
