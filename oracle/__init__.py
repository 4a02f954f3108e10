"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C++ statement of the method (CSR SpMV, l1-Jacobi diagonal,
matching weights, greedy matching, aggregation, Galerkin product, Cholesky,
the V(1,1) cycle of Eq. (amg) and PCG), wrapped here with ctypes and numpy.
Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It imports nothing from the GPU
library and the GPU library imports nothing from it.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None
_openmp = False


def use_openmp(on: bool = True) -> None:
    """Load the OpenMP build (the same sources; its parallel row loops give
    the same bits) instead of the single-thread one.  Call before the first
    oracle call of the process; OMP_NUM_THREADS sets the thread count."""
    global _openmp
    if _lib is not None and on != _openmp:
        raise RuntimeError("the oracle library is already loaded")
    _openmp = on


def threads() -> int:
    """Threads the loaded oracle's parallel row loops use (1: plain build)."""
    return int(lib().orc_threads())


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build(openmp=_openmp))
        _declare(_lib)
    return _lib


_P = C.c_void_p
_I64 = C.c_int64


def _declare(L):
    L.orc_threads.restype = C.c_int
    L.orc_dot.restype = C.c_double
    L.orc_dot.argtypes = [_I64, _P, _P]
    L.orc_spmv.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.orc_l1_scale.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.orc_match_weights.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.orc_mix64.restype = C.c_uint64
    L.orc_mix64.argtypes = [C.c_uint64]
    L.orc_match.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.orc_number_pairs.restype = _I64
    L.orc_number_pairs.argtypes = [_I64, _P, _P]
    L.orc_galerkin.argtypes = [_I64, _P, _P, _P, _P, _I64, _P, _P, _P]
    L.orc_cholesky.restype = C.c_int
    L.orc_cholesky.argtypes = [_I64, _P, _P]
    L.orc_chol_solve.argtypes = [_I64, _P, _P, _P]
    L.orc_setup.restype = _P
    L.orc_setup.argtypes = [_I64, _P, _P, _P, C.c_int, _I64, C.c_int, C.c_double, _I64, _P,
                            C.POINTER(C.c_int)]
    L.orc_setup_systems.restype = _P
    L.orc_setup_systems.argtypes = [_I64, _P, _P, _P, C.c_int, _P, C.c_int, _I64, C.c_int,
                                    C.c_double, _I64, C.POINTER(C.c_int)]
    L.orc_free.argtypes = [_P]
    L.orc_set_cycle.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double]
    L.orc_setup_smoothed.restype = _P
    L.orc_setup_smoothed.argtypes = [_I64, _P, _P, _P, C.c_int, _I64, C.c_int, C.c_double, _I64,
                                     _P]
    L.orc_setup_general.restype = _P
    L.orc_setup_general.argtypes = [_I64, _P, _P, _P, C.c_int, _I64, C.c_int, C.c_double, _I64,
                                    C.c_int, C.c_int, C.c_double, C.c_double, _P]
    L.orc_vbm_aggregate.restype = _I64
    L.orc_vbm_aggregate.argtypes = [_I64, _P, _P, _P, C.c_double, _P]
    L.orc_level_prolongator.restype = _I64
    L.orc_level_prolongator.argtypes = [_P, C.c_int, _P, _P, _P, _P]
    L.orc_setup_reuse.restype = _P
    L.orc_setup_reuse.argtypes = [_I64, _P, _P, _P, _P, _I64, _P]
    L.orc_levels.restype = C.c_int
    L.orc_levels.argtypes = [_P]
    L.orc_level_n.restype = _I64
    L.orc_level_n.argtypes = [_P, C.c_int]
    L.orc_level_nnz.restype = _I64
    L.orc_level_nnz.argtypes = [_P, C.c_int]
    L.orc_level_csr.argtypes = [_P, C.c_int, _P, _P, _P]
    L.orc_level_agg.argtypes = [_P, C.c_int, _P]
    L.orc_level_dinv.argtypes = [_P, C.c_int, _P]
    L.orc_coarse_factor.argtypes = [_P, _P]
    L.orc_vcycle.argtypes = [_P, _P, _P]
    L.orc_pcg.argtypes = [_P, _I64, _P, _P, _P, _P, _P, _P, C.c_double, C.c_int, C.c_int,
                          _P, _P, _P]
    L.orc_pcg_block.argtypes = [_P, _I64, _I64, _P, _P, C.c_double, C.c_int, C.c_int, _P]
    if hasattr(L, "mlp_orc_forward"):
        _declare_mlp(L)


def _declare_mlp(L):
    L.mlp_orc_nparam.restype = C.c_int
    L.mlp_orc_features.argtypes = [_I64, _I64, _I64, _P, _P, _P, _P]
    L.mlp_orc_forward.argtypes = [_I64, _P, _P, C.c_double, _P, _P]
    L.mlp_orc_backward.argtypes = [_I64, _P, _P, C.c_double, _P, _P]
    L.mlp_orc_adam.argtypes = [C.c_int, _P, _P, _P, _P, C.c_int, C.c_double, C.c_double,
                               C.c_double, C.c_double]
    L.tg_orc_loss.restype = C.c_int
    L.tg_orc_loss.argtypes = [_I64, _P, _P, _P, _P, _I64, _P, _P, _P, _P, C.c_int, C.c_int, _P,
                              _P, _P]


# ---------------------------------------------------------------- learned smoother

def mlp_nparam():
    return lib().mlp_orc_nparam()


def mlp_features(A, shape):
    """Nine features per row of a 7-point operator on a grid shape (nz, ny, nx)."""
    nz, ny, nx = shape
    n, rp, ci, v = csr_args(A)
    f = np.empty((n, 9))
    lib().mlp_orc_features(nx, ny, nz, _p(rp), _p(ci), _p(v), _p(f))
    return f


def mlp_forward(params, feat, omega_max=1.0):
    """omega = max(omega_max * sigmoid(z), 1e-3) per row, and z."""
    p, f = _f64(params), _f64(feat)
    n = f.shape[0]
    om, z = np.empty(n), np.empty(n)
    lib().mlp_orc_forward(n, _p(p), _p(f), omega_max, _p(om), _p(z))
    return om, z


def mlp_backward(params, feat, domega, omega_max=1.0):
    p, f, d = _f64(params), _f64(feat), _f64(domega)
    g = np.empty(mlp_nparam())
    lib().mlp_orc_backward(f.shape[0], _p(p), _p(f), omega_max, _p(d), _p(g))
    return g


def mlp_adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays params, m, v."""
    g = _f64(grad)
    lib().mlp_orc_adam(len(params), _p(params), _p(g), _p(m), _p(v), t, lr, b1, b2, eps)


def twogrid_loss(A, agg, Ac, omega, e0, K=2):
    """Two-grid error-reduction loss and d loss / d omega (exact coarse solve)."""
    n, rp, ci, v = csr_args(A)
    nc, rpc, cic, vc = csr_args(Ac)
    ag, om, e = _i32(agg), _f64(omega), _f64(e0)
    ns = e.shape[0]
    loss = np.zeros(1)
    dom = np.empty(n)
    st = lib().tg_orc_loss(n, _p(rp), _p(ci), _p(v), _p(ag), nc, _p(rpc), _p(cic), _p(vc),
                           _p(om), ns, K, _p(e), _p(loss), _p(dom))
    if st != 0:
        raise RuntimeError("coarse matrix not SPD")
    return float(loss[0]), dom


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def csr_args(A):
    rp, ci, v = A
    return len(rp) - 1, _i64(rp), _i32(ci), _f64(v)


def dot(x, y):
    x, y = _f64(x), _f64(y)
    return lib().orc_dot(len(x), _p(x), _p(y))


def spmv(A, x):
    n, rp, ci, v = csr_args(A)
    x = _f64(x)
    y = np.empty(n)
    lib().orc_spmv(n, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def l1_scale(A, omega=None):
    n, rp, ci, v = csr_args(A)
    om = None if omega is None else _f64(omega)
    d = np.empty(n)
    lib().orc_l1_scale(n, _p(rp), _p(ci), _p(v), _p(om), _p(d))
    return d


def match_weights(A, w=None):
    n, rp, ci, v = csr_args(A)
    w = None if w is None else _f64(w)
    c = np.empty(len(v))
    lib().orc_match_weights(n, _p(rp), _p(ci), _p(v), _p(w), _p(c))
    return c


def mix64(z: int) -> int:
    return int(lib().orc_mix64(C.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def match(A, w=None):
    n, rp, ci, v = csr_args(A)
    w = None if w is None else _f64(w)
    mate = np.empty(n, dtype=np.int32)
    lib().orc_match(n, _p(rp), _p(ci), _p(v), _p(w), _p(mate))
    return mate


def vbm_aggregate(A, theta=0.01):
    """Decoupled Vanek-Mandel-Brezina aggregates of A: (agg, nc)."""
    n, rp, ci, v = csr_args(A)
    agg = np.empty(n, dtype=np.int32)
    nc = lib().orc_vbm_aggregate(n, _p(rp), _p(ci), _p(v), theta, _p(agg))
    return agg, int(nc)


def number_pairs(mate):
    mate = _i32(mate)
    agg = np.empty(len(mate), dtype=np.int32)
    nc = lib().orc_number_pairs(len(mate), _p(mate), _p(agg))
    return agg, int(nc)


def galerkin(A, agg, nc):
    n, rp, ci, v = csr_args(A)
    agg = _i32(agg)
    rpc = np.empty(nc + 1, dtype=np.int64)
    lib().orc_galerkin(n, _p(rp), _p(ci), _p(v), _p(agg), nc, _p(rpc), None, None)
    nnz = int(rpc[-1])
    cc = np.empty(nnz, dtype=np.int32)
    vc = np.empty(nnz)
    lib().orc_galerkin(n, _p(rp), _p(ci), _p(v), _p(agg), nc, _p(rpc), _p(cc), _p(vc))
    return rpc, cc, vc


def cholesky(a):
    a = _f64(a)
    n = a.shape[0]
    L = np.empty((n, n))
    st = lib().orc_cholesky(n, _p(a), _p(L))
    return L, st


def chol_solve(L, b):
    L = _f64(L)
    b = _f64(b)
    x = np.empty(len(b))
    lib().orc_chol_solve(len(b), _p(L), _p(b), _p(x))
    return x


class Hierarchy:
    """The oracle's AMG hierarchy (levels, aggregates, smoother scales, coarse factor)."""

    def __init__(self, A, sweeps=2, max_coarse=200, max_levels=30, stall=0.9,
                 max_dense=8192, omega=None, systems=None, smooth_sweeps=1, variable=False,
                 coarse="cholesky", coarse_maxit=40, coarse_tol=1e-4, smoothed=False,
                 aggregation="matching", theta=0.01, pfilter=0.0):
        """systems: row offsets (nsys + 1) of independent systems stacked block
        diagonally in A; coarsening then stops when each has <= max_coarse rows.
        smooth_sweeps: l1-Jacobi sweeps nu_0 before and after the coarse
        correction; variable: nu_l = nu_0 * 2^l (variable V-cycle, Sec. 3);
        coarse: "cholesky" (dense) or "pcg" (PCG with l1-Jacobi, at most
        coarse_maxit iterations, stop at ||r|| <= coarse_tol ||b||).
        aggregation: "matching" (`sweeps` matching sweeps) or "vbm" (decoupled
        Vanek-Mandel-Brezina with strength threshold theta).  pfilter > 0:
        smoothed prolongators built from the filtered matrix A_F."""
        n, rp, ci, v = csr_args(A)
        self._keep = (rp, ci, v)
        st = C.c_int(0)
        agg = {"matching": 0, "vbm": 1}[aggregation]
        if smoothed or agg:
            assert systems is None and omega is None
            self.h = lib().orc_setup_general(n, _p(rp), _p(ci), _p(v), sweeps, max_coarse,
                                             max_levels, stall, max_dense, 1 if smoothed else 0,
                                             agg, theta, pfilter, C.byref(st))
        elif systems is not None:
            so = _i64(systems)
            self.h = lib().orc_setup_systems(n, _p(rp), _p(ci), _p(v), len(so) - 1, _p(so),
                                             sweeps, max_coarse, max_levels, stall, max_dense,
                                             C.byref(st))
        else:
            om = None if omega is None else _f64(omega)
            self.h = lib().orc_setup(n, _p(rp), _p(ci), _p(v), sweeps, max_coarse, max_levels,
                                     stall, max_dense, _p(om), C.byref(st))
        self.status = st.value
        self.n = n
        self.sweeps = sweeps
        lib().orc_set_cycle(self.h, smooth_sweeps, 1 if variable else 0,
                            {"cholesky": 0, "pcg": 1}[coarse], coarse_maxit, coarse_tol)

    def reuse(self, A, max_dense=8192):
        """A hierarchy for new values of the matrix this one was built from
        (same sparsity): these aggregates on every level, new Galerkin values,
        smoother scales and coarse factor, the same cycle parameters."""
        n, rp, ci, v = csr_args(A)
        st = C.c_int(0)
        H = Hierarchy.__new__(Hierarchy)
        H._keep = (rp, ci, v)
        H.h = lib().orc_setup_reuse(n, _p(rp), _p(ci), _p(v), self.h, max_dense, C.byref(st))
        H.status = st.value
        H.n = n
        H.sweeps = self.sweeps
        return H

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    @property
    def levels(self):
        return lib().orc_levels(self.h)

    def level_n(self, l):
        return lib().orc_level_n(self.h, l)

    def level_nnz(self, l):
        return lib().orc_level_nnz(self.h, l)

    def level_csr(self, l):
        n, nnz = self.level_n(l), self.level_nnz(l)
        rp = np.empty(n + 1, dtype=np.int64)
        ci = np.empty(nnz, dtype=np.int32)
        v = np.empty(nnz)
        lib().orc_level_csr(self.h, l, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def level_agg(self, l):
        a = np.empty(self.level_n(l), dtype=np.int32)
        lib().orc_level_agg(self.h, l, _p(a))
        return a

    def level_prolongator(self, l):
        """Smoothed P of level l as CSR (rowptr, col, val) and its damping w."""
        nnz = lib().orc_level_prolongator(self.h, l, None, None, None, None)
        n = self.level_n(l)
        rp = np.empty(n + 1, dtype=np.int64)
        ci = np.empty(nnz, dtype=np.int32)
        v = np.empty(nnz)
        w = C.c_double(0.0)
        lib().orc_level_prolongator(self.h, l, _p(rp), _p(ci), _p(v), C.byref(w))
        return (rp, ci, v), w.value

    def level_dinv(self, l):
        d = np.empty(self.level_n(l))
        lib().orc_level_dinv(self.h, l, _p(d))
        return d

    def coarse_factor(self):
        m = self.level_n(self.levels - 1)
        L = np.empty((m, m))
        lib().orc_coarse_factor(self.h, _p(L))
        return L

    def operator_complexity(self):
        return sum(self.level_nnz(l) for l in range(self.levels)) / self.level_nnz(0)

    def vcycle(self, r):
        r = _f64(r)
        z = np.empty(self.n)
        lib().orc_vcycle(self.h, _p(r), _p(z))
        return z


def block_diag(systems):
    """Concatenates CSR systems into one block-diagonal CSR; returns (A, offsets)."""
    rps, cis, vs, offs = [], [], [], [0]
    nnz = 0
    for rp, ci, v in systems:
        rp = np.asarray(rp, dtype=np.int64)
        rps.append(rp[:-1] - rp[0] + nnz)
        cis.append(np.asarray(ci, dtype=np.int64) + offs[-1])
        vs.append(np.asarray(v, dtype=np.float64))
        nnz += int(rp[-1] - rp[0])
        offs.append(offs[-1] + len(rp) - 1)
    rowptr = np.concatenate(rps + [np.array([nnz], dtype=np.int64)])
    return (rowptr, np.concatenate(cis).astype(np.int32), np.concatenate(vs)), offs


def pcg_block(hier, r0, r1, b, x0=None, tol=1e-8, maxit=500, beta_form=0):
    """PCG on diagonal block [r0, r1) of hier's level-0 matrix with its V-cycle."""
    b = _f64(b)
    x = np.zeros(r1 - r0) if x0 is None else _f64(x0).copy()
    out = np.zeros(4)
    lib().orc_pcg_block(hier.h, r0, r1, _p(b), _p(x), tol, maxit, beta_form, _p(out))
    return x, dict(iterations=int(out[0]), status=int(out[1]), relres=float(out[2]),
                   true_relres=float(out[3]))


def pcg(A, b, x0=None, tol=1e-8, maxit=500, beta_form=0, hier=None, binv=None,
        history=False, x_history=False):
    """PCG on A (CSR).  Returns (x, info) with info = dict(iterations, status,
    relres, true_relres, res_hist[, x_hist])."""
    n, rp, ci, v = csr_args(A)
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    bi = None if binv is None else _f64(binv)
    rh = np.zeros(maxit + 1) if history else None
    xh = np.zeros((maxit + 1, n)) if x_history else None
    out = np.zeros(4)
    lib().orc_pcg(hier.h if hier is not None else None, n, _p(rp), _p(ci), _p(v), _p(bi),
                  _p(b), _p(x), tol, maxit, beta_form, _p(rh), _p(xh), _p(out))
    it = int(out[0])
    info = dict(iterations=it, status=int(out[1]), relres=float(out[2]),
                true_relres=float(out[3]))
    if history:
        info["res_hist"] = rh[:it + 1]
    if x_history:
        info["x_hist"] = xh[:it + 1]
    return x, info
