"""ctypes binding of the C ABI declared in ``include/phicomb.h`` (same names, argument marshalling only).

The shared library is built in-tree by :mod:`paper_2509_26475_gb300.build`; loading fails loudly when
it is missing.  There is no fallback: every step of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PHIC_OK, PHIC_INVALID_ARG, PHIC_NONFINITE, PHIC_TERM_CAP, PHIC_TIMEOUT, PHIC_CUDA_ERROR, PHIC_WORKSPACE_TOO_SMALL = range(7)
PHIC_F64, PHIC_F32 = 0, 1
PHIC_NO_V0 = 1
PHIC_PHASE_SERIES, PHIC_PHASE_RECOVER = 0x10, 0x20
PHIC_BATCH_SELECT, PHIC_BATCH_NO_SOLVE = 0x100, 0x200
PHIC_MAX_R, PHIC_MAX_P, PHIC_MAX_WIDTH = 16, 15, 128
PHIC_NOALLOC_MAX_BYTES = 32 << 20
PHIC_MAX_RANK = 8

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "TERM_CAP", 4: "TIMEOUT", 5: "CUDA_ERROR",
                6: "WORKSPACE_TOO_SMALL"}


class PhicError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: phicomb status {STATUS_NAMES.get(int(status), status)}")


class phic_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p), ("prec", ctypes.c_int32)]


class phic_select_opts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("max_evals", ctypes.c_int32), ("spin_limit_ms", ctypes.c_double)]


class phic_params(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("s", ctypes.c_double), ("s0", ctypes.c_double),
                ("f_star", ctypes.c_double), ("r", ctypes.c_int32), ("evals", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


class phic_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("s_int", ctypes.c_int32), ("series_terms", ctypes.c_int32),
                ("max_inner_terms", ctypes.c_int32), ("recovery_terms", ctypes.c_int64),
                ("spmm_count", ctypes.c_int64), ("xi", ctypes.c_double), ("s", ctypes.c_double),
                ("op_format", ctypes.c_int32), ("op_slots", ctypes.c_int32)]


class phic_lowrank(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("prec", ctypes.c_int32), ("U", ctypes.c_void_p),
                ("W", ctypes.c_void_p)]


class phic_batch_item(ctypes.Structure):
    _fields_ = [("A", phic_csr), ("p", ctypes.c_int32), ("r", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("max_terms", ctypes.c_int32), ("V", ctypes.c_void_p), ("W", ctypes.c_void_p),
                ("params", ctypes.c_void_p), ("stats", ctypes.c_void_p), ("v_select", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("s_hint", ctypes.c_double), ("t", ctypes.c_double * 16),
                ("alpha", ctypes.c_double * 16)]


class phic_batch_config(ctypes.Structure):
    _fields_ = [("rows_per_cta", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class phic_batch_info(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("count", ctypes.c_int32),
                ("max_team", ctypes.c_int32), ("entries", ctypes.c_int64), ("est_makespan_us", ctypes.c_double),
                ("est_busy_frac", ctypes.c_double)]


class phic_server_config(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t), ("rows_per_cta", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("max_steps", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("device", ctypes.c_int32), ("m", ctypes.c_int32), ("slice_us", ctypes.c_double)]


class phic_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("prec", ctypes.c_int32), ("p", ctypes.c_int32), ("r", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("tol", ctypes.c_double), ("max_terms", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("op", ctypes.c_int64), ("t", ctypes.c_double * 16),
                ("alpha", ctypes.c_double * 16)]


class phic_operator(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p), ("prec", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class phic_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("submit_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64), ("slices", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("params", phic_params), ("stats", phic_stats)]


class phic_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("slices", ctypes.c_int64), ("max_slice_requests", ctypes.c_int64),
                ("arena_in_use", ctypes.c_int64), ("arena_peak", ctypes.c_int64), ("gpu_busy_ms", ctypes.c_double)]

# phic_apply_fn: Y = A X on a stream (see include/phicomb.h)
APPLY_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                            ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p)


class phic_fn_op(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("prec", ctypes.c_int32), ("pad", ctypes.c_int32), ("apply", ctypes.c_void_p),
                ("ctx", ctypes.c_void_p), ("norm_bound", ctypes.c_double)]


# The public structs in the order phic_struct_sizes reports them.
STRUCTS = (phic_csr, phic_select_opts, phic_params, phic_stats, phic_lowrank, phic_batch_item, phic_batch_config,
           phic_batch_info, phic_server_config, phic_operator, phic_request, phic_request_info, phic_server_counters,
           phic_fn_op)


PHIC_REQ_QUEUED, PHIC_REQ_LOADING, PHIC_REQ_RUNNING, PHIC_REQ_COPYING, PHIC_REQ_DONE = range(5)

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) for every function declared in include/phicomb.h
_P = ctypes.c_void_p
SIGNATURES = [
    ("phic_select_opts_default", None, [ctypes.POINTER(phic_select_opts)]),
    ("phic_select_workspace_size", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_select_params", ctypes.c_int, [ctypes.POINTER(phic_csr), ctypes.POINTER(phic_select_opts), _P, _P,
                                          ctypes.c_size_t, _P, _P]),
    ("phic_params_set", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P]),
    ("phic_solve_workspace_size", ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_tile_layout", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    ("phic_solve", ctypes.c_int, [ctypes.POINTER(phic_csr), ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                  ctypes.c_double, _P, ctypes.c_uint32, ctypes.c_int32, _P, _P, ctypes.c_size_t, _P,
                                  ctypes.c_int32, _P]),
    ("phic_solve_noalloc", ctypes.c_int, [ctypes.POINTER(phic_csr), ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                          ctypes.c_double, _P, ctypes.c_uint32, ctypes.c_int32, _P, _P,
                                          ctypes.c_int32, _P]),
    ("phic_lowrank_select_workspace_size", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                          ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_lowrank_select_params", ctypes.c_int, [ctypes.POINTER(phic_lowrank), ctypes.POINTER(phic_select_opts), _P,
                                                  _P, ctypes.c_size_t, _P, _P]),
    ("phic_lowrank_solve_workspace_size", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                         ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_lowrank_solve", ctypes.c_int, [ctypes.POINTER(phic_lowrank), ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                          ctypes.c_double, _P, ctypes.c_uint32, ctypes.c_int32, _P, _P,
                                          ctypes.c_size_t, _P, ctypes.c_int32, _P]),
    ("phic_batch_workspace_size", ctypes.c_int, [ctypes.POINTER(phic_batch_item), ctypes.c_int32,
                                                 ctypes.POINTER(phic_select_opts), ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_batch_create", ctypes.c_int, [ctypes.POINTER(phic_batch_item), ctypes.c_int32,
                                         ctypes.POINTER(phic_select_opts), ctypes.POINTER(phic_batch_config), _P,
                                         ctypes.c_size_t, _P, ctypes.POINTER(ctypes.c_void_p)]),
    ("phic_batch_launch", ctypes.c_int, [_P, _P]),
    ("phic_batch_resume", ctypes.c_int, [_P, _P]),
    ("phic_batch_pending", ctypes.c_int, [_P, _P, _P]),
    ("phic_batch_info_get", ctypes.c_int, [_P, ctypes.POINTER(phic_batch_info)]),
    ("phic_batch_destroy", None, [_P]),
    ("phic_batch_plan_host", ctypes.c_int, [ctypes.POINTER(phic_batch_item), ctypes.c_int32,
                                            ctypes.POINTER(phic_select_opts), ctypes.POINTER(phic_batch_config),
                                            ctypes.c_int32, _P, _P, _P, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    ("phic_batch_autotune", ctypes.c_int, [ctypes.POINTER(phic_batch_item), ctypes.c_int32,
                                           ctypes.POINTER(phic_select_opts), _P, ctypes.c_size_t,
                                           ctypes.POINTER(phic_batch_config), ctypes.c_int32, ctypes.c_int32, _P,
                                           ctypes.POINTER(phic_batch_config), ctypes.POINTER(ctypes.c_double)]),
    ("phic_server_create", ctypes.c_int, [ctypes.POINTER(phic_server_config), ctypes.POINTER(ctypes.c_void_p)]),
    ("phic_server_submit", ctypes.c_int, [_P, ctypes.POINTER(phic_request), ctypes.POINTER(ctypes.c_int64)]),
    ("phic_server_add_operator", ctypes.c_int, [_P, ctypes.POINTER(phic_operator), ctypes.POINTER(ctypes.c_int64)]),
    ("phic_server_operator_params", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                                   ctypes.POINTER(phic_params)]),
    ("phic_server_remove_operator", ctypes.c_int, [_P, ctypes.c_int64]),
    ("phic_server_query", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(phic_request_info)]),
    ("phic_server_wait", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(phic_request_info)]),
    ("phic_server_counters_get", ctypes.c_int, [_P, ctypes.POINTER(phic_server_counters)]),
    ("phic_server_destroy", None, [_P]),
    ("phic_set_spin_limit_ms", None, [ctypes.c_double]),
    ("phic_set_blocks_per_sm", None, [ctypes.c_int32]),
    ("phic_set_test_fault", None, [ctypes.c_int32]),
    ("phic_fn_select_workspace_size", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_fn_select_params", ctypes.c_int, [ctypes.POINTER(phic_fn_op), ctypes.POINTER(phic_select_opts), _P, _P,
                                             ctypes.c_size_t, _P, _P]),
    ("phic_fn_solve_workspace_size", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.POINTER(ctypes.c_size_t)]),
    ("phic_fn_solve", ctypes.c_int, [ctypes.POINTER(phic_fn_op), ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                     ctypes.c_double, _P, ctypes.c_uint32, ctypes.c_int32, _P, _P, ctypes.c_size_t, _P,
                                     ctypes.c_int32, _P]),
    ("phic_csr_apply", ctypes.c_int32, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P]),
    ("phic_probe_fp64_fma", ctypes.c_int, [ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int64), _P]),
    ("phic_test_objective_coeffs", ctypes.c_int, [ctypes.c_int32, ctypes.c_double, _P, _P]),
    ("phic_status_string", ctypes.c_char_p, [ctypes.c_int32]),
    ("phic_launch_count", ctypes.c_uint64, []),
    ("phic_version", ctypes.c_int32, []),
    ("phic_struct_sizes", ctypes.c_int32, [ctypes.POINTER(ctypes.c_size_t), ctypes.c_int32]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libphicomb.so (optionally building it first); raises if it is not there."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"{_build.LIB} is missing: build it with __graft_entry__.build() "
                                   "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(_build.LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str):
    if int(status) != PHIC_OK:
        raise PhicError(status, where)
