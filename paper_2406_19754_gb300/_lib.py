"""ctypes declarations of the C ABI in include/amg.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamg_gb300.so")

AMG_OK = 0
AMG_NOT_CONVERGED = 1
AMG_ERR_ARG = -1
AMG_ERR_NOT_SPD = -2
AMG_ERR_BREAKDOWN = -3
AMG_ERR_NAN = -4
AMG_ERR_CUDA = -5
AMG_ERR_OOM = -6
AMG_ERR_DEVICE_CHECK = -7
AMG_ERR_UNSUPPORTED = -8
AMG_PREC_F64 = 0
AMG_PREC_F32 = 1
PCG_BETA_AUTO = -1
PCG_BETA_FR = 0
PCG_BETA_FLEXIBLE = 1

_P = C.c_void_p


class AmgCsr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", _P), ("col", _P), ("val", _P)]


class AmgOptions(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("max_levels", C.c_int), ("max_coarse", C.c_int64),
                ("stall_ratio", C.c_double), ("max_dense", C.c_int64), ("precision", C.c_int),
                ("bf16_from_level", C.c_int), ("slice_height", C.c_int),
                ("threads_per_row", C.c_int), ("autotune", C.c_int),
                ("tail_rows", C.c_int64), ("smooth_sweeps", C.c_int),
                ("variable_cycle", C.c_int), ("coarse_solver", C.c_int),
                ("coarse_maxit", C.c_int), ("coarse_tol", C.c_double),
                ("compress_columns", C.c_int),
                ("smooth_prolongator", C.c_int),
                ("aggregation", C.c_int),
                ("vbm_theta", C.c_double),
                ("prolongator_filter", C.c_double),
                ("stream_ring", C.c_int)]


class PcgOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("beta_form", C.c_int),
                ("res_history", C.POINTER(C.c_double)), ("x_history", _P),
                ("use_graph", C.c_int)]


class PcgStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("solve_ms", C.c_double)]


class AmgLayout(C.Structure):
    _fields_ = [("slice_height", C.c_int), ("threads_per_row", C.c_int), ("slots", C.c_int64),
                ("compressed", C.c_int)]


class AmgKernelTime(C.Structure):
    _fields_ = [("level", C.c_int), ("kind", C.c_int), ("bytes", C.c_double), ("ms", C.c_double)]


# name -> (restype, argtypes); every exported function of include/amg.h
SIGNATURES = {
    "amg_default_options": (C.c_int, [C.POINTER(AmgOptions)]),
    "pcg_default_options": (C.c_int, [C.POINTER(PcgOptions)]),
    "amg_status_string": (C.c_char_p, [C.c_int]),
    "amg_setup": (C.c_int, [C.POINTER(AmgCsr), C.POINTER(AmgOptions), _P, C.POINTER(_P)]),
    "amg_update_values": (C.c_int, [_P, C.POINTER(AmgCsr), _P]),
    "amg_destroy": (C.c_int, [_P]),
    "amg_set_smoother_weights": (C.c_int, [_P, _P, _P]),
    "amg_vcycle_apply": (C.c_int, [_P, _P, _P, _P]),
    "amg_vcycle_profile": (C.c_int, [_P, _P, _P, C.POINTER(AmgKernelTime), C.c_int,
                                     C.POINTER(C.c_int), _P]),
    "amg_spmv": (C.c_int, [_P, C.c_int, C.c_double, _P, C.c_double, _P, _P]),
    "pcg_solve": (C.c_int, [_P, _P, _P, C.POINTER(PcgOptions), C.POINTER(PcgStats), _P]),
    "amg_vcycle_apply_multi": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "pcg_solve_multi": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(PcgOptions),
                                  C.POINTER(PcgStats), _P]),
    "amg_setup_batch": (C.c_int, [C.c_int, C.POINTER(AmgCsr), C.POINTER(AmgOptions), _P,
                                  C.POINTER(_P)]),
    "amg_batch_info": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "pcg_solve_batch": (C.c_int, [_P, _P, _P, C.POINTER(PcgOptions), C.POINTER(PcgStats), _P]),
    "mlp_num_params": (C.c_int, []),
    "mlp_create": (C.c_int, [C.c_uint64, C.POINTER(_P)]),
    "mlp_destroy": (C.c_int, [_P]),
    "mlp_get_params": (C.c_int, [_P, _P]),
    "mlp_set_params": (C.c_int, [_P, _P]),
    "mlp_get_grad": (C.c_int, [_P, _P]),
    "mlp_set_omega_max": (C.c_int, [_P, C.c_double]),
    "mlp_set_exact_forward": (C.c_int, [_P, C.c_int]),
    "mlp_features": (C.c_int, [C.POINTER(AmgCsr), C.c_int64, C.c_int64, C.c_int64, _P, _P]),
    "mlp_forward": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "mlp_backward": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int, _P]),
    "mlp_adam_step": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_double, _P]),
    "amg_twogrid_loss": (C.c_int, [_P, C.c_int, C.c_int, _P, C.POINTER(C.c_double), _P, _P]),
    "amg_num_levels": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "amg_level_info": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "amg_level_layout": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(AmgLayout)]),
    "amg_level_export": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "amg_level_prolongator": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_double), _P]),
    "amg_pairwise_match": (C.c_int, [C.POINTER(AmgCsr), _P, C.POINTER(C.c_int), _P]),
    "amg_pairwise_match_noalloc": (C.c_int, [C.POINTER(AmgCsr), _P, C.POINTER(C.c_int), _P]),
    "amg_debug_fail_alloc_after": (C.c_int, [C.c_long]),
    "mlp_debug_gelu": (C.c_int, [_P, _P, C.c_int64, _P]),
    "amg_debug_convert": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P]),
    "amg_debug_tail_timeout": (C.c_int, [_P, C.c_int]),
}

_lib = None


def load():
    """Loads the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "GPU library %s is missing: build it with paper_2406_19754_gb300.build.build()"
                % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib
