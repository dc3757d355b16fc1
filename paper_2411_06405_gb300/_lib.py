"""ctypes view of libhtruss.so (include/htruss.h).  Argument marshalling only."""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhtruss.so")

HTD_OK = 0
HTD_EINVAL = 1
HTD_ENOMEM = 2
HTD_ECUDA = 3
HTD_ETIMEOUT = 4
HTD_EOVERFLOW = 5
HTD_EUNSUPPORTED = 6
HTD_MAX_H = 8
HTD_MAX_N = 1600000
HTD_STATIC_MAX_N = 786432
HTD_OPT_TIMING = 1
HTD_OPT_NO_GRAPH = 2
HTD_OPT_REBUILD = 4
HTD_OPT_TINY_LOSS_TABLE = 8
HTD_OPT_PERSISTENT_ROUNDS = 16
HTD_OPT_COMPACT_BALLS = 32
HTD_OPT_BATCH_BLOCKS = 64
HTD_HX_PRUNE = 1

# every symbol include/htruss.h declares
EXPORTED = (
    "htd_build_csr", "htd_graph_info", "htd_edges", "htd_csr", "htd_h_support",
    "htd_truss_decompose", "htd_truss_decompose_ex", "htd_truss_decompose_host",
    "htd_graph_free", "htd_kernel_launch_count", "htd_status_string", "htd_last_error",
    "htd_h_support_static", "htd_truss_decompose_batched", "htd_batch_plan",
    "htd_hindex_decompose", "htd_hindex_decompose_ex", "htd_footprint_estimate", "htd_server_create", "htd_server_submit", "htd_server_poll",
    "htd_server_wait", "htd_server_info", "htd_server_destroy",
)


class HtdStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int64),
        ("levels", ctypes.c_int64),
        ("max_truss", ctypes.c_int32),
        ("h", ctypes.c_int32),
        ("hsup_evals", ctypes.c_int64),
        ("ball_builds", ctypes.c_int64),
        ("balls_changed", ctypes.c_int64),
        ("frontier_edges", ctypes.c_int64),
        ("pairs_tested", ctypes.c_int64),
        ("pairs_lost", ctypes.c_int64),
        ("member_tests", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("ball_pool_bytes", ctypes.c_int64),
        ("timed_slots", ctypes.c_int64),
        ("alg_bytes_ball", ctypes.c_double),
        ("alg_bytes_hsup", ctypes.c_double),
        ("alg_bytes_detect", ctypes.c_double),
        ("alg_bytes_update", ctypes.c_double),
        ("ms_initial_ball", ctypes.c_float),
        ("ms_initial_hsup", ctypes.c_float),
        ("ms_select", ctypes.c_float),
        ("ms_find", ctypes.c_float),
        ("ms_remove", ctypes.c_float),
        ("ms_ball", ctypes.c_float),
        ("ms_update", ctypes.c_float),
        ("ms_minreduce", ctypes.c_float),
        ("ms_round_kernel", ctypes.c_float),
        ("round_kernel_launches", ctypes.c_int32),
        ("incremental", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("slots", ctypes.c_int64),
        ("pairs3_tested", ctypes.c_int64),
        ("pairs2_lost", ctypes.c_int64),
        ("rounds_rebuilt", ctypes.c_int64),
        ("alg_bytes_hsup_initial", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class HtdHindexStats(ctypes.Structure):
    _fields_ = [
        ("ball_entries", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("h", ctypes.c_int32),
        ("sweeps", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("ms_total", ctypes.c_float),
        ("pruned", ctypes.c_int32),
        ("edge_evals", ctypes.c_int64),
        ("vertex_evals", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class HtdRequestInfo(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64),
        ("est_bytes", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("submit_s", ctypes.c_double),
        ("admit_s", ctypes.c_double),
        ("start_s", ctypes.c_double),
        ("done_s", ctypes.c_double),
        ("h", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("worker", ctypes.c_int32),
        ("retries", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class HtdServerStats(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_int64),
        ("reserved_bytes", ctypes.c_int64),
        ("peak_reserved_bytes", ctypes.c_int64),
        ("workers", ctypes.c_int32),
        ("running", ctypes.c_int32),
        ("peak_running", ctypes.c_int32),
        ("pending", ctypes.c_int32),
        ("admitted", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


class HtdError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load():
    """Loads the compiled library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_2411_06405_gb300.build.build() "
                "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        i32, i64, u32, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p
        pp = ctypes.POINTER(ctypes.c_void_p)
        ps = ctypes.POINTER(HtdStats)
        sig = {
            "htd_build_csr": ([i32, p, p, i64, ctypes.c_int, p, pp], ctypes.c_int),
            "htd_graph_info": ([p, ctypes.POINTER(i32), ctypes.POINTER(i64)], ctypes.c_int),
            "htd_edges": ([p, p, p, p], ctypes.c_int),
            "htd_csr": ([p, p, p, p, p], ctypes.c_int),
            "htd_h_support": ([p, i32, p, p], ctypes.c_int),
            "htd_truss_decompose": ([p, i32, p, p, ps, p], ctypes.c_int),
            "htd_truss_decompose_ex": ([p, i32, u32, p, p, ps, p], ctypes.c_int),
            "htd_truss_decompose_host": ([i32, p, p, i64, i32, p, p, p, ctypes.POINTER(i64), ps, p],
                                         ctypes.c_int),
            "htd_graph_free": ([p], None),
            "htd_kernel_launch_count": ([], i64),
            "htd_h_support_static": ([i32, p, p, i64, p, p, i32, p, p], ctypes.c_int),
            "htd_truss_decompose_batched": ([i32, p, p, p, p, p, u32, i32, p, p, p,
                                             ctypes.POINTER(i32), ps, p], ctypes.c_int),
            "htd_batch_plan": ([i32, p, p, p, i32, p, p, ctypes.POINTER(i32)], ctypes.c_int),
            "htd_hindex_decompose": ([p, i32, i32, i32, p, p, ctypes.POINTER(HtdHindexStats), p],
                                     ctypes.c_int),
            "htd_hindex_decompose_ex": ([p, i32, i32, i32, u32, p, p, ctypes.POINTER(HtdHindexStats), p],
                                        ctypes.c_int),
            "htd_footprint_estimate": ([i32, i64, i32, i64], i64),
            "htd_server_create": ([i32, i64, u32, pp], ctypes.c_int),
            "htd_server_submit": ([p, i32, p, p, i64, i32, ctypes.POINTER(i64)], ctypes.c_int),
            "htd_server_poll": ([p, i64, ctypes.POINTER(i32)], ctypes.c_int),
            "htd_server_wait": ([p, i64, p, p, p, i64, ctypes.POINTER(HtdRequestInfo)],
                                ctypes.c_int),
            "htd_server_info": ([p, ctypes.POINTER(HtdServerStats)], ctypes.c_int),
            "htd_server_destroy": ([p], None),
            "htd_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "htd_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(status: int, where: str):
    if status != HTD_OK:
        lib = load()
        msg = lib.htd_last_error().decode(errors="replace")
        base = lib.htd_status_string(status).decode(errors="replace")
        raise HtdError(status, where, f"{base}: {msg}")
