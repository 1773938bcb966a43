"""ctypes binding of libfitsne_gb300.so (include/fitsne_gb300.h).

Argument marshalling only: every step of the gradient runs in the library's
CUDA kernels. torch supplies device memory and streams. If the compiled
library is missing the import fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfitsne_gb300.so")

TSNE_OK = 0
TSNE_ERR_INVALID_ARG = -1
TSNE_ERR_OOM = -2
TSNE_ERR_NONFINITE = -3
TSNE_ERR_TIMEOUT = -4
TSNE_ERR_CUDA = -5
TSNE_ERR_CAPACITY = -6

_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "NONFINITE", -4: "TIMEOUT", -5: "CUDA",
          -6: "CAPACITY"}


class TsneError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class tsne_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("nnz", ctypes.c_int64)]


class tsne_plan_opts(ctypes.Structure):
    _fields_ = [("n_min", ctypes.c_int32), ("n_int_max", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("relabel_first", ctypes.c_int32),
                ("relabel_every", ctypes.c_int32), ("force_mode", ctypes.c_int32),
                ("order_rounds", ctypes.c_int32)]


class tsne_step_params(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int32), ("early_iters", ctypes.c_int32),
                ("late_iters", ctypes.c_int32), ("mom_switch_iter", ctypes.c_int32),
                ("early_alpha", ctypes.c_float), ("late_alpha", ctypes.c_float),
                ("lr", ctypes.c_float), ("momentum_early", ctypes.c_float),
                ("momentum_late", ctypes.c_float), ("min_gain", ctypes.c_float),
                ("gain_inc", ctypes.c_float), ("gain_dec", ctypes.c_float)]


class tsne_plan_info_t(ctypes.Structure):
    _fields_ = [("y_min", ctypes.c_float), ("width", ctypes.c_float), ("b", ctypes.c_float),
                ("delta", ctypes.c_float), ("n_int", ctypes.c_int32), ("n", ctypes.c_int32),
                ("fft_len", ctypes.c_int32), ("n_chunks", ctypes.c_int32),
                ("Z", ctypes.c_double), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


TSNE_FORCE_AUTO = 0
TSNE_FORCE_GRID = 1
TSNE_FORCE_REGION = 2

TSNE_NINT_RULE = 0
TSNE_NINT_FILL = 1


class tsne_batch_opts(ctypes.Structure):
    _fields_ = [("n_min", ctypes.c_int32), ("n_int_max", ctypes.c_int32),
                ("max_jobs", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class tsne_batch_tuning(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("fft_threads", ctypes.c_int32),
                ("n_int_policy", ctypes.c_int32), ("ms_per_iter", ctypes.c_float)]


class tsne_oocpca_opts(ctypes.Structure):
    _fields_ = [("its", ctypes.c_int32), ("center", ctypes.c_int32), ("block_rows", ctypes.c_int64),
                ("stream", ctypes.c_void_p)]


# (name, restype, argtypes) for every entry point of include/fitsne_gb300.h
# and include/oocpca_gb300.h
_P = ctypes.c_void_p
_SIGNATURES = [
    ("tsne_version", ctypes.c_char_p, []),
    ("tsne_last_error_string", ctypes.c_char_p, []),
    ("tsne_step_params_default", None, [ctypes.POINTER(tsne_step_params)]),
    ("tsne_alpha_at", ctypes.c_float, [ctypes.POINTER(tsne_step_params), ctypes.c_int32]),
    ("tsne_plan_create", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(tsne_plan_opts),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("tsne_plan_destroy", ctypes.c_int, [_P]),
    ("tsne_plan_set_box", ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_int32]),
    ("tsne_gradient", ctypes.c_int, [_P, tsne_csr, _P, ctypes.c_float, _P, _P]),
    ("tsne_step", ctypes.c_int, [_P, tsne_csr, _P, _P, _P, ctypes.c_int32,
                                 ctypes.POINTER(tsne_step_params)]),
    ("tsne_run", ctypes.c_int, [_P, tsne_csr, _P, ctypes.POINTER(tsne_step_params),
                                ctypes.POINTER(ctypes.c_double)]),
    ("tsne_run_reset", ctypes.c_int, [_P]),
    ("tsne_run_iters", ctypes.c_int, [_P, tsne_csr, _P, ctypes.POINTER(tsne_step_params),
                                      ctypes.c_int32, ctypes.c_int32]),
    ("tsne_plan_order", ctypes.c_int, [_P, tsne_csr]),
    ("tsne_run_state_save", ctypes.c_int, [_P, _P, _P]),
    ("tsne_run_state_load", ctypes.c_int, [_P, _P, _P]),
    ("tsne_kl", ctypes.c_int, [_P, tsne_csr, _P, ctypes.POINTER(ctypes.c_double)]),
    ("tsne_run_host", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P,
                                     ctypes.POINTER(tsne_step_params),
                                     ctypes.POINTER(ctypes.c_double)]),
    ("tsne_validate_csr", ctypes.c_int, [_P, tsne_csr]),
    ("tsne_plan_status", ctypes.c_int, [_P]),
    ("tsne_plan_info", ctypes.c_int, [_P, ctypes.POINTER(tsne_plan_info_t)]),
    ("tsne_debug_copy", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]),
    ("tsne_plan_profile", ctypes.c_int, [_P, ctypes.c_int32]),
    ("tsne_plan_profile_read", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int64)]),
    ("tsne_plan_launch_count", ctypes.c_int64, [_P]),
    ("tsne_batch_opts_default", None, [ctypes.POINTER(tsne_batch_opts)]),
    ("tsne_batch_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(tsne_batch_opts),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("tsne_batch_destroy", ctypes.c_int, [_P]),
    ("tsne_batch_job_bytes", ctypes.c_int64, [_P, ctypes.c_int64]),
    ("tsne_batch_bytes_in_use", ctypes.c_int64, [_P]),
    ("tsne_batch_add_job", ctypes.c_int, [_P, ctypes.c_int64, tsne_csr, _P, ctypes.c_int32,
                                          ctypes.POINTER(tsne_step_params),
                                          ctypes.POINTER(ctypes.c_int32)]),
    ("tsne_batch_remove_job", ctypes.c_int, [_P, ctypes.c_int32]),
    ("tsne_batch_iterate", ctypes.c_int, [_P, ctypes.c_int32]),
    ("tsne_batch_poll", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]),
    ("tsne_batch_get_y", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("tsne_batch_kl", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    ("tsne_batch_set_tuning", ctypes.c_int, [_P, ctypes.POINTER(tsne_batch_tuning)]),
    ("tsne_batch_get_tuning", ctypes.c_int, [_P, ctypes.POINTER(tsne_batch_tuning)]),
    ("tsne_batch_autotune", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(tsne_batch_tuning)]),
    ("tsne_batch_launch_count", ctypes.c_int64, [_P]),
    ("tsne_batch_stream", ctypes.c_void_p, [_P]),
    ("tsne_kl_noalloc", ctypes.c_int, [tsne_csr, _P, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_double, _P, _P]),
    ("tsne_noalloc_last_error_string", ctypes.c_char_p, []),
    ("tsne_affinity_create", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    ("tsne_affinity_destroy", ctypes.c_int, [_P]),
    ("tsne_affinity_compute", ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.POINTER(tsne_csr)]),
    ("tsne_affinity_knn_copy", ctypes.c_int, [_P, _P, _P, _P]),
    ("tsne_affinity_phase_ms", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("tsne_affinity_launch_count", ctypes.c_int64, [_P]),
    ("tsne_affinity_knn_info", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    ("tsne_heatmap_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                           ctypes.POINTER(_P)]),
    ("tsne_heatmap_destroy", ctypes.c_int, [_P]),
    ("tsne_heatmap_bin", ctypes.c_int, [_P, _P, ctypes.c_int64, tsne_csr, _P, _P]),
    ("tsne_heatmap_nearest", ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    ("tsne_heatmap_phase_ms", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("tsne_heatmap_launch_count", ctypes.c_int64, [_P]),
    ("tsne_oocpca_create", ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(tsne_oocpca_opts), ctypes.POINTER(_P)]),
    ("tsne_oocpca_destroy", ctypes.c_int, [_P]),
    ("tsne_oocpca_run", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P]),
    ("tsne_oocpca_debug_copy", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    ("tsne_oocpca_phase_ms", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int32)]),
    ("tsne_oocpca_launch_count", ctypes.c_int64, [_P]),
]

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, res, args in _SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int) -> None:
    if rc != TSNE_OK:
        raise TsneError(rc, load().tsne_last_error_string().decode())


def exported_names():
    return [n for n, _, _ in _SIGNATURES]
