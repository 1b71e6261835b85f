"""ctypes mirror of include/ap.h.  Argument marshalling only: every step of the
solver runs in libap.so's CUDA kernels; nothing here computes."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

AP_MAX_RHS = 32
AP_MAX_DIM = 32

AP_OK, AP_ERR_INVALID_ARG, AP_ERR_NOMEM, AP_ERR_NOT_SPD, AP_ERR_NAN = 0, 1, 2, 3, 4
AP_ERR_NOT_CONVERGED, AP_ERR_TIMEOUT, AP_ERR_CUDA, AP_ERR_UNSUPPORTED = 5, 6, 7, 8
AP_ERR_SCRATCH_LIMIT = 9
AP_ERR_CANCELLED = 10
AP_STATIC_SCRATCH_BYTES = 1 << 20
AP_RBF, AP_MATERN32, AP_MATERN52 = 0, 1, 2
AP_FP32, AP_BF16_REFINE, AP_FP16_REFINE = 0, 1, 2
AP_CACHE_TC_EXACT, AP_CACHE_FP64 = 0, 1
AP_SEL_GS, AP_SEL_CYCLIC, AP_SEL_RANDOM = 0, 1, 2
AP_STOP_MEAN_REL, AP_STOP_MAX_REL, AP_STOP_FRO, AP_STOP_Y_REL = 0, 1, 2, 3
AP_RESID_AUTO, AP_RESID_FP32, AP_RESID_COMPENSATED = 0, 1, 2

# every function include/ap.h declares
EXPORTS = ["ap_opts_default", "ap_create", "ap_set_hyper", "ap_solve", "ap_residual",
           "ap_predict_mean", "ap_grad_quadforms", "ap_mll_grad", "ap_destroy", "ap_status_str",
           "ap_sizeof_opts", "ap_sizeof_info", "ap_sizeof_hyper", "ap_launch_count", "ap_sfu_rates", "ap_phi_fp64_eval",
           "ap_grad_quadforms_static", "ap_server_create", "ap_server_submit", "ap_server_poll",
           "ap_server_wait", "ap_server_destroy", "ap_sizeof_request", "ap_sizeof_request_result",
           "ap_tracked_residual", "ap_device_bytes", "ap_last_cuda_error", "ap_server_cancel", "ap_solve_host",
           "ap_bounds_violations", "ap_bounds_selftest"]


class ap_hyper(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("d", ctypes.c_int32), ("lengthscale", ctypes.c_void_p),
                ("outputscale", ctypes.c_float), ("noise", ctypes.c_float), ("mean", ctypes.c_float)]


class ap_opts(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int64), ("select", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("tol", ctypes.c_double), ("min_epochs", ctypes.c_int32), ("max_epochs", ctypes.c_int32),
                ("max_steps", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("refine_every", ctypes.c_int32), ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("hbm_budget", ctypes.c_size_t), ("block_trace", ctypes.POINTER(ctypes.c_int32)),
                ("trace_cap", ctypes.c_int64), ("profile", ctypes.c_int32),
                ("residual_mode", ctypes.c_int32), ("cache_gemm", ctypes.c_int32),
                ("wait_limit_cycles", ctypes.c_int64), ("cancel", ctypes.c_void_p),
                ("escalate", ctypes.c_int32)]


class ap_info(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("refinements", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("bad_block", ctypes.c_int32), ("c", ctypes.c_int32),
                ("rel_res_tracked", ctypes.c_double * AP_MAX_RHS),
                ("rel_res_true", ctypes.c_double * AP_MAX_RHS),
                ("t_cache_s", ctypes.c_double), ("t_solve_s", ctypes.c_double),
                ("t_refine_s", ctypes.c_double), ("kernel_entries", ctypes.c_double),
                ("entries_per_s", ctypes.c_double), ("gpu_launches", ctypes.c_int64),
                ("data_fit", ctypes.c_double), ("t_update_s", ctypes.c_double),
                ("n_update", ctypes.c_int64), ("t_blocksolve_s", ctypes.c_double),
                ("fp32_epochs", ctypes.c_int32), ("compensated", ctypes.c_int32), ("diverged", ctypes.c_int32)]


class ap_request(ctypes.Structure):
    _fields_ = [("X_host", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("y_host", ctypes.c_void_p), ("Xtest_host", ctypes.c_void_p), ("M", ctypes.c_int64),
                ("hyper", ap_hyper), ("block", ctypes.c_int64), ("tol", ctypes.c_double),
                ("stop", ctypes.c_int32), ("min_epochs", ctypes.c_int32), ("max_epochs", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("refine_every", ctypes.c_int32), ("mean_host", ctypes.c_void_p)]


class ap_request_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int), ("epochs", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("queue_s", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("reserved_bytes", ctypes.c_size_t), ("started", ctypes.c_int32),
                ("compensated", ctypes.c_int32)]


_lib = None


def checked() -> bool:
    """True when this process uses the bounds-checked build (environment
    variable AP_CHECKED=1, read once at the first load)."""
    return os.environ.get("AP_CHECKED", "0") == "1"


def lib_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libap.so, or libap_checked.so under AP_CHECKED=1 (building it first
    if it is missing).  There is no fallback: if the CUDA library cannot be
    built or loaded this raises."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} is missing; run __graft_entry__.build()")
        _build.build(checked=checked())
    L = ctypes.CDLL(path)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    st = ctypes.c_int
    sig = {
        "ap_opts_default": (None, [ctypes.POINTER(ap_opts)]),
        "ap_create": (st, [ctypes.POINTER(P), P, i64, i32, ctypes.POINTER(ap_hyper), ctypes.POINTER(ap_opts)]),
        "ap_set_hyper": (st, [P, ctypes.POINTER(ap_hyper)]),
        "ap_solve": (st, [P, P, i32, P, P, ctypes.POINTER(ap_info)]),
        "ap_residual": (st, [P, P, i32, P, P]),
        "ap_solve_host": (st, [P, i64, i32, ctypes.POINTER(ap_hyper), ctypes.POINTER(ap_opts), P, i32, P,
                               ctypes.POINTER(ap_info)]),
        "ap_predict_mean": (st, [P, P, P, i64, P]),
        "ap_grad_quadforms": (st, [P, P, P, i32, P, P]),
        "ap_grad_quadforms_static": (st, [P, P, P, i32, P, P]),
        "ap_mll_grad": (st, [P, P, i32, P, P, ctypes.POINTER(ap_info)]),
        "ap_destroy": (None, [P]),
        "ap_launch_count": (i64, [P]),
        "ap_device_bytes": (ctypes.c_size_t, [P]),
        "ap_last_cuda_error": (i32, [P]),
        "ap_bounds_violations": (i32, [ctypes.c_char_p, i32]),
        "ap_bounds_selftest": (st, [i32]),
        "ap_tracked_residual": (st, [P, i32, P]),
        "ap_sfu_rates": (st, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "ap_phi_fp64_eval": (st, [i32, P, i64, P]),
        "ap_server_create": (st, [ctypes.POINTER(P), ctypes.c_size_t, i32, i32]),
        "ap_server_submit": (st, [P, ctypes.POINTER(ap_request), ctypes.POINTER(i64)]),
        "ap_server_poll": (st, [P, i64, ctypes.POINTER(ap_request_result)]),
        "ap_server_wait": (st, [P, i64, ctypes.c_double, ctypes.POINTER(ap_request_result)]),
        "ap_server_destroy": (None, [P]),
        "ap_server_cancel": (st, [P, i64]),
        "ap_status_str": (ctypes.c_char_p, [st]),
        "ap_sizeof_opts": (ctypes.c_size_t, []),
        "ap_sizeof_info": (ctypes.c_size_t, []),
        "ap_sizeof_hyper": (ctypes.c_size_t, []),
        "ap_sizeof_request": (ctypes.c_size_t, []),
        "ap_sizeof_request_result": (ctypes.c_size_t, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L
