"""ctypes declarations of the C ABI in include/spq.h (libspq.so, built in-tree)."""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspq.so")

SPQ_OK, SPQ_EINVAL, SPQ_ENOMEM, SPQ_ECUDA, SPQ_ETIMEOUT, SPQ_EUNSUPPORTED = range(6)
SPQ_I32, SPQ_F32 = 0, 1
SPQ_ARITH_AUTO, SPQ_ARITH_I32, SPQ_ARITH_F32 = 0, 1, 2
SPQ_ORDER_AUTO, SPQ_ORDER_ID, SPQ_ORDER_DISSECTION, SPQ_ORDER_VERTEX_DISSECTION = 0, 1, 2, 3
SPQ_BG_AUTO, SPQ_BG_FW, SPQ_BG_ELIM = 0, 1, 2
SPQ_INF_I32 = 0x20000000
SPQ_NOALLOC_MAX_PAIRS = 262144

# Every symbol include/spq.h declares, with (restype, argtypes).
P = ctypes.c_void_p
i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class SpqOpts(ctypes.Structure):
    _fields_ = [("struct_size", i32), ("arith", i32), ("order", i32), ("skip_inf_tiles", i32),
                ("profile_kernels", i32), ("query_grouped", i32), ("bg_method", i32),
                ("bg_panel_mib", i32), ("comp_method", i32), ("query_kernel", i32)]


class SpqGraph(ctypes.Structure):
    _fields_ = [("n", i32), ("row_ptr", P), ("col", P), ("w", P), ("wt", ctypes.c_int), ("part", P), ("k", i32)]


SIGNATURES = {
    "spq_opts_default": (None, [ctypes.POINTER(SpqOpts)]),
    "spq_build": (ctypes.c_int, [i32, P, P, P, ctypes.c_int, P, i32, ctypes.POINTER(SpqOpts), P,
                                 ctypes.POINTER(P)]),
    "spq_query": (ctypes.c_int, [P, P, i64, P, P]),
    "spq_query_status": (ctypes.c_int, [P, P]),
    "spq_build_many": (ctypes.c_int, [i32, ctypes.POINTER(SpqGraph), ctypes.POINTER(SpqOpts), P, ctypes.POINTER(P)]),
    "spq_query_many": (ctypes.c_int, [i32, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(i64),
                                      ctypes.POINTER(P), P]),
    "spq_query_noalloc": (ctypes.c_int, [P, P, i64, P, P]),
    "spq_query_saved": (ctypes.c_int, [P, P, i64, P, P, P]),
    "spq_query_backward": (ctypes.c_int, [P, P, i64, P, P, P, P]),
    "spq_query_paths": (ctypes.c_int, [P, P, i64, P, ctypes.c_int32, P, P, P]),
    "spq_query_matrix": (ctypes.c_int, [P, P, i64, P, i64, P, P]),
    "spq_query_tuning": (i32, [P, P, i32]),
    "spq_build_tuning": (i32, [P, P, P, i32]),
    "spq_query_plan_create": (ctypes.c_int, [i32, P, P, P, P, P, ctypes.POINTER(P)]),
    "spq_query_plan_run": (ctypes.c_int, [P, P]),
    "spq_query_plan_free": (None, [P]),
    "spq_build_plan_create": (ctypes.c_int, [i32, ctypes.POINTER(SpqGraph), ctypes.POINTER(SpqOpts), P,
                                             ctypes.POINTER(P), ctypes.POINTER(P)]),
    "spq_build_plan_run": (ctypes.c_int, [P, ctypes.POINTER(P), P]),
    "spq_build_plan_free": (None, [P]),
    "spq_server_create": (ctypes.c_int, [ctypes.c_int, i32, i64, ctypes.c_size_t, ctypes.POINTER(P)]),
    "spq_server_add_graph": (ctypes.c_int, [P, i32, P]),
    "spq_server_remove_graph": (ctypes.c_int, [P, i32]),
    "spq_server_submit": (ctypes.c_int, [P, i32, P, i64, P, ctypes.POINTER(i64)]),
    "spq_server_poll": (i32, [P, i64]),
    "spq_server_wait": (ctypes.c_int, [P, i64, ctypes.c_double]),
    "spq_server_stats": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(i64), ctypes.POINTER(i64), i32]),
    "spq_server_destroy": (None, [P]),
    "spq_free": (None, [P]),
    "spq_release_cached_memory": (None, []),
    "spq_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "spq_last_cuda_error": (ctypes.c_int, []),
    "spq_footprint_bytes": (ctypes.c_size_t, [P]),
    "spq_stats": (None, [P, ctypes.POINTER(i64), ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(i32)]),
    "spq_build_profile": (i32, [P, ctypes.POINTER(f64), i32]),
    "spq_peak_minplus": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(f64),
                                        ctypes.POINTER(f64)]),
    "spq_kernel_launches": (ctypes.c_ulonglong, []),
    "spq_test_backsub_wait": (None, [ctypes.c_ulonglong, i32]),
    "spq_query_profile": (ctypes.c_int, [P, ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(f64)]),
    "spq_pool_usage": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong),
                                      ctypes.POINTER(ctypes.c_ulonglong)]),
    "spq_component_order_host": (ctypes.c_int, [ctypes.c_int, P, P, P, ctypes.c_int, P, P]),
    "spq_boundary_order_host": (ctypes.c_int, [ctypes.c_int, P, P, P, P, P, ctypes.c_int, P]),
    "spq_boundary_layout_host": (ctypes.c_int, [ctypes.c_int, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P,
                                                ctypes.c_int]),
    "spq_get_meta": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "spq_get_apsp": (ctypes.c_int, [P, i32, P, P]),
    "spq_get_bg": (ctypes.c_int, [P, P, P]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libspq.so and declare its signatures.  Raises if the library is missing:
    there is no fallback implementation."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libspq.so not built ({path}); run paper_1503_07192_gb300.build_ext.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


class SpqError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.spq_strerror(status).decode()
        if status == SPQ_ECUDA:
            msg += f" (cudaError {lib.spq_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")
        self.status = status
