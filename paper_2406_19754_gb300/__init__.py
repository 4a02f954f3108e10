"""GB300 (sm_103a) PCG preconditioned by an aggregation-based AMG V-cycle.

Python binding over the C ABI of ``include/amg.h``.  Every step of the solve
(hierarchy setup, V-cycle, PCG) runs in the library's CUDA kernels; this
module only passes device pointers of torch tensors and the current CUDA
stream.  There is no CPU path: if the compiled library is missing, importing
the binding's entry points raises.
"""

from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import (AMG_PREC_F32, AMG_PREC_F64, PCG_BETA_AUTO, PCG_BETA_FLEXIBLE,  # noqa: F401
                   PCG_BETA_FR, AmgCsr, AmgOptions, PcgOptions, PcgStats)


class AmgError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.load().amg_status_string(status).decode()
        super().__init__("%s%s (status %d)" % (what + ": " if what else "", msg, status))


def _check(rc: int, what: str = "") -> int:
    if rc < 0:
        raise AmgError(rc, what)
    return rc


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return t.contiguous()


def csr_struct(rowptr, col, val):
    rowptr = _dev(rowptr, torch.int64, "rowptr")
    col = _dev(col, torch.int32, "col")
    val = _dev(val, torch.float64, "val")
    A = AmgCsr(rowptr.numel() - 1, col.numel(), _ptr(rowptr), _ptr(col), _ptr(val))
    return A, (rowptr, col, val)


def options(**kw) -> AmgOptions:
    o = AmgOptions()
    _lib.load().amg_default_options(C.byref(o))
    prec = kw.pop("precision", None)
    if prec is not None:
        o.precision = {"f64": AMG_PREC_F64, "f32": AMG_PREC_F32}.get(prec, prec)
    agg = kw.pop("aggregation", None)
    if agg is not None:
        o.aggregation = {"matching": 0, "vbm": 1}.get(agg, agg)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    return o


class Hierarchy:
    """An AMG hierarchy built on the GPU from a CSR matrix (torch CUDA tensors:
    rowptr int64, col int32, val float64).  Keyword options are the fields of
    ``amg_options`` (``precision`` may be "f64" or "f32")."""

    def __init__(self, rowptr, col, val, stream=None, **opts):
        self._lib = _lib.load()
        A, keep = csr_struct(rowptr, col, val)
        self.n = A.n
        o = options(**opts)
        self.opts = o
        h = C.c_void_p()
        _check(self._lib.amg_setup(C.byref(A), C.byref(o), _stream(stream), C.byref(h)),
               "amg_setup")
        self.h = h
        del keep

    def update_values(self, rowptr, col, val, stream=None):
        """New values of the same sparsity: rebuilds the hierarchy on its
        existing aggregates (no matching)."""
        A, keep = csr_struct(rowptr, col, val)
        _check(self._lib.amg_update_values(self.h, C.byref(A), _stream(stream)),
               "amg_update_values")
        del keep

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.amg_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def levels(self) -> int:
        v = C.c_int()
        _check(self._lib.amg_num_levels(self.h, C.byref(v)))
        return v.value

    def level_info(self, l):
        n, nnz = C.c_int64(), C.c_int64()
        _check(self._lib.amg_level_info(self.h, l, C.byref(n), C.byref(nnz)))
        return n.value, nnz.value

    def level_layout(self, l, ap=False):
        """Kernel storage of level l's matrix (ap False/0), of A P (True/1),
        or with smoothed prolongators of P (2) or R = P^T (3): dict with
        slice_height, threads_per_row, slots, compressed."""
        o = _lib.AmgLayout()
        _check(self._lib.amg_level_layout(self.h, l, int(ap), C.byref(o)))
        return dict(slice_height=o.slice_height, threads_per_row=o.threads_per_row,
                    slots=o.slots, compressed=bool(o.compressed))

    def level_export(self, l, stream=None):
        n, nnz = self.level_info(l)
        dev = torch.device("cuda")
        out = {}
        rp = cl = vl = None
        if l > 0:
            rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
            cl = torch.empty(nnz, dtype=torch.int32, device=dev)
            vl = torch.empty(nnz, dtype=torch.float64, device=dev)
            out.update(rowptr=rp, col=cl, val=vl)
        agg = None
        if l < self.levels - 1:
            agg = torch.empty(n, dtype=torch.int32, device=dev)
            out["agg"] = agg
        ss = torch.empty(n, dtype=torch.float64, device=dev)
        out["sscale"] = ss
        _check(self._lib.amg_level_export(self.h, l, _ptr(rp), _ptr(cl), _ptr(vl), _ptr(agg),
                                          _ptr(ss), _stream(stream)), "amg_level_export")
        return out

    def level_prolongator(self, l, stream=None):
        """Smoothed prolongator of level l (option smooth_prolongator):
        ((rowptr, col, val) CUDA tensors, damping w)."""
        nnz, w = C.c_int64(), C.c_double()
        _check(self._lib.amg_level_prolongator(self.h, l, None, None, None, C.byref(nnz),
                                               C.byref(w), _stream(stream)),
               "amg_level_prolongator")
        n = self.level_info(l)[0]
        dev = torch.device("cuda")
        rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
        cl = torch.empty(nnz.value, dtype=torch.int32, device=dev)
        vl = torch.empty(nnz.value, dtype=torch.float64, device=dev)
        _check(self._lib.amg_level_prolongator(self.h, l, _ptr(rp), _ptr(cl), _ptr(vl), None,
                                               None, _stream(stream)), "amg_level_prolongator")
        return (rp, cl, vl), w.value

    def operator_complexity(self):
        nnz = [self.level_info(l)[1] for l in range(self.levels)]
        return sum(nnz) / nnz[0]

    def set_smoother_weights(self, omega=None, stream=None):
        if omega is not None:
            omega = _dev(omega, torch.float32, "omega")
        _check(self._lib.amg_set_smoother_weights(self.h, _ptr(omega), _stream(stream)))

    def vcycle(self, r, z=None, stream=None):
        r = _dev(r, torch.float64, "r")
        if z is None:
            z = torch.empty_like(r)
        _check(self._lib.amg_vcycle_apply(self.h, _ptr(r), _ptr(z), _stream(stream)),
               "amg_vcycle_apply")
        return z

    def vcycle_profile(self, r, z=None, stream=None):
        """z = B r with per-kernel event timing; returns (z, list of dicts)."""
        r = _dev(r, torch.float64, "r")
        if z is None:
            z = torch.empty_like(r)
        recs = (_lib.AmgKernelTime * 256)()
        cnt = C.c_int()
        _check(self._lib.amg_vcycle_profile(self.h, _ptr(r), _ptr(z), recs, 256, C.byref(cnt),
                                            _stream(stream)), "amg_vcycle_profile")
        kinds = ("pre", "restrict", "post", "coarse", "tail", "sweep")
        out = [dict(level=k.level, kind=kinds[k.kind], bytes=k.bytes, ms=k.ms)
               for k in recs[:min(cnt.value, 256)]]
        return z, out

    def spmv(self, x, y=None, level=0, alpha=1.0, beta=0.0, stream=None):
        x = _dev(x, torch.float64, "x")
        if y is None:
            y = torch.zeros_like(x) if beta != 0.0 else torch.empty_like(x)
        _check(self._lib.amg_spmv(self.h, level, alpha, _ptr(x), beta, _ptr(y), _stream(stream)),
               "amg_spmv")
        return y

    def pcg(self, b, x=None, tol=1e-8, maxit=500, beta_form="auto", history=False,
            x_history=False, use_graph=True, stream=None):
        """Solves A x = b; returns (x, stats dict)."""
        b = _dev(b, torch.float64, "b")
        if x is None:
            x = torch.zeros_like(b)
        o = _pcg_options(self._lib, tol, maxit, beta_form, use_graph)
        hist = None
        if history:
            hist = (C.c_double * (maxit + 1))()
            o.res_history = C.cast(hist, C.POINTER(C.c_double))
        xh = None
        if x_history:
            xh = torch.zeros((maxit + 1, b.numel()), dtype=torch.float64, device=b.device)
            o.x_history = _ptr(xh)
        st = PcgStats()
        rc = self._lib.pcg_solve(self.h, _ptr(b), _ptr(x), C.byref(o), C.byref(st),
                                 _stream(stream))
        if rc not in (_lib.AMG_ERR_BREAKDOWN, _lib.AMG_ERR_NAN):
            _check(rc, "pcg_solve")
        info = dict(iterations=st.iterations, status=st.status, relres=st.rel_residual,
                    true_relres=st.true_rel_residual, solve_ms=st.solve_ms)
        if history:
            info["res_hist"] = list(hist)[:st.iterations + 1]
        if x_history:
            info["x_hist"] = xh[:st.iterations + 1]
        return x, info

    def vcycle_multi(self, R, Z=None, stream=None):
        """Z = B R for the columns of a row-major (n, k) tensor, k <= 64."""
        R = _dev(R, torch.float64, "R")
        if Z is None:
            Z = torch.empty_like(R)
        _check(self._lib.amg_vcycle_apply_multi(self.h, R.shape[1], _ptr(R), _ptr(Z),
                                                _stream(stream)), "amg_vcycle_apply_multi")
        return Z

    def pcg_multi(self, B, X=None, tol=1e-8, maxit=500, beta_form="auto", stream=None):
        """Solves A X = B column by column (B row-major (n, k), k <= 64).
        Returns (X, list of per-column stats dicts)."""
        B = _dev(B, torch.float64, "B")
        if X is None:
            X = torch.zeros_like(B)
        o = _pcg_options(self._lib, tol, maxit, beta_form, True)
        k = B.shape[1]
        st = (PcgStats * k)()
        rc = self._lib.pcg_solve_multi(self.h, k, _ptr(B), _ptr(X), C.byref(o), st,
                                       _stream(stream))
        if rc not in (_lib.AMG_ERR_BREAKDOWN, _lib.AMG_ERR_NAN):
            _check(rc, "pcg_solve_multi")
        return X, _stats_list(st)


def _pcg_options(lib, tol, maxit, beta_form, use_graph):
    o = PcgOptions()
    lib.pcg_default_options(C.byref(o))
    o.tol = tol
    o.maxit = maxit
    o.beta_form = {"auto": PCG_BETA_AUTO, "fr": PCG_BETA_FR,
                   "flexible": PCG_BETA_FLEXIBLE}.get(beta_form, beta_form)
    # True / 1: whole loop as one graph; 2: one graph per iteration; False / 0: none
    o.use_graph = int(use_graph) if not isinstance(use_graph, bool) else (1 if use_graph else 0)
    return o


def _stats_list(st):
    return [dict(iterations=s.iterations, status=s.status, relres=s.rel_residual,
                 true_relres=s.true_rel_residual, solve_ms=s.solve_ms) for s in st]


class BatchHierarchy(Hierarchy):
    """One hierarchy for many independent systems (list of (rowptr, col, val)
    CUDA tensors); ``pcg`` solves them all with per-system scalars."""

    def __init__(self, systems, stream=None, **opts):
        self._lib = _lib.load()
        keep = []
        arr = (AmgCsr * len(systems))()
        for k, (rp, ci, v) in enumerate(systems):
            A, kp = csr_struct(rp, ci, v)
            arr[k] = A
            keep.append(kp)
        o = options(**opts)
        self.opts = o
        h = C.c_void_p()
        _check(self._lib.amg_setup_batch(len(systems), arr, C.byref(o), _stream(stream),
                                         C.byref(h)), "amg_setup_batch")
        self.h = h
        ns = C.c_int()
        offs = (C.c_int64 * (len(systems) + 1))()
        _check(self._lib.amg_batch_info(self.h, C.byref(ns), offs))
        self.nsys = ns.value
        self.offsets = list(offs)
        self.n = self.offsets[-1]
        del keep

    def pcg(self, b, x=None, tol=1e-8, maxit=500, beta_form="auto", use_graph=True,
            stream=None):
        """Solves every system; b, x concatenated.  Returns (x, list of stats dicts)."""
        b = _dev(b, torch.float64, "b")
        if x is None:
            x = torch.zeros_like(b)
        o = _pcg_options(self._lib, tol, maxit, beta_form, use_graph)
        st = (PcgStats * self.nsys)()
        rc = self._lib.pcg_solve_batch(self.h, _ptr(b), _ptr(x), C.byref(o), st,
                                       _stream(stream))
        if rc not in (_lib.AMG_ERR_BREAKDOWN, _lib.AMG_ERR_NAN):
            _check(rc, "pcg_solve_batch")
        return x, _stats_list(st)


def pairwise_match(rowptr, col, val, stream=None):
    """Locally-dominant pairwise matching; returns (mate int32 tensor, rounds)."""
    lib = _lib.load()
    A, keep = csr_struct(rowptr, col, val)
    mate = torch.empty(A.n, dtype=torch.int32, device=keep[0].device)
    rounds = C.c_int()
    _check(lib.amg_pairwise_match(C.byref(A), _ptr(mate), C.byref(rounds), _stream(stream)),
           "amg_pairwise_match")
    return mate, rounds.value


def csr_to_device(A, device="cuda"):
    """(rowptr, col, val) numpy arrays -> CUDA tensors with the ABI's dtypes."""
    rp, ci, v = A
    return (torch.as_tensor(rp, dtype=torch.int64).to(device),
            torch.as_tensor(ci, dtype=torch.int32).to(device),
            torch.as_tensor(v, dtype=torch.float64).to(device))
