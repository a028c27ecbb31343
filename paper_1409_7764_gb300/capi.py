"""ctypes declarations of the C ABI in include/bc_gb300.h.

Loading fails loudly when the compiled library is missing: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

BC_OK = 0
BC_PENDING = 1
BC_ERR_ARG = -1
BC_ERR_GRAPH = -2
BC_ERR_OOM = -3
BC_ERR_CUDA = -4
BC_ERR_TIMEOUT = -5
BC_ERR_SIGMA_OVERFLOW = -6
BC_ERR_NOT_FOUND = -7
BC_ERR_ADMISSION = -8
BC_ERR_INTERNAL = -9

BC_SCHED_AUTO = 0
BC_SCHED_PLAIN = 1
BC_SCHED_BATCH = 2
BC_SCHED_BATCH_QUEUE = 3
BC_SCHED_BATCH_VERTEX = 4
BC_SCHED_BATCH_WARP = 5
BC_SCHED_BATCH_EDGE = 6

# every symbol include/bc_gb300.h declares
EXPORTED = [
    "bc_init", "bc_shutdown", "bc_create_graph", "bc_destroy_graph", "bc_exact", "bc_sources",
    "bc_submit", "bc_poll", "bc_wait", "bc_last_stats", "bc_debug_source", "bc_debug_sources", "bc_debug_graph", "bc_create_graphs",
    "bc_exact_many", "bc_debug_inject_barrier_skip", "bc_status_str", "bc_sources_noalloc",
    "bc_sources_estimate", "bc_sources_adaptive", "bc_last_overflow_sources",
]

BC_NOALLOC_MAX_N = 8192


class bc_opts(ctypes.Structure):
    _fields_ = [("delta_fp64", ctypes.c_int32), ("batch_k", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("normalize", ctypes.c_int32),
                ("scale_sampled", ctypes.c_int32), ("out_device", ctypes.c_int32),
                ("source_order", ctypes.c_int32), ("direction", ctypes.c_int32),
                ("count_bits", ctypes.c_int32)]


class bc_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("sources", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("max_levels", ctypes.c_int32), ("overflow_sources", ctypes.c_int32),
                ("device_ms", ctypes.c_double), ("frontier_entries", ctypes.c_int64),
                ("scanned_out_edges", ctypes.c_int64), ("scanned_in_edges", ctypes.c_int64),
                ("dag_pairs", ctypes.c_int64), ("reached_pairs", ctypes.c_int64),
                ("heavy_chunks", ctypes.c_int64), ("kernel_kind", ctypes.c_int32),
                ("levels_sum", ctypes.c_int32),
                ("chunk_edges", ctypes.c_int32), ("grab", ctypes.c_int32),
                ("batch_sources", ctypes.c_int32), ("mask_words", ctypes.c_int32),
                ("push_levels", ctypes.c_int32), ("batch_groups", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def load(path: str | None = None):
    """Loads libbc_gb300.so (building it first if it is missing or stale and
    nvcc is available).  Raises RuntimeError when it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("BC_GB300_LIB") or _build.LIB
    if path == _build.LIB and (not os.path.exists(path) or _build.stale()):
        try:
            _build.build()
        except Exception as exc:  # no silent fallback
            raise RuntimeError(f"CUDA library {path} is missing and could not be built: {exc}")
    try:
        lib = ctypes.CDLL(path)
    except OSError as exc:
        raise RuntimeError(f"cannot load CUDA library {path}: {exc}")
    vp = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "bc_init": ([ctypes.c_int, vp, ctypes.c_size_t, ctypes.POINTER(vp)], ctypes.c_int),
        "bc_shutdown": ([vp], ctypes.c_int),
        "bc_create_graph": ([vp, vp, vp, i32, i64, i64p, i64p], ctypes.c_int),
        "bc_destroy_graph": ([vp, i64], ctypes.c_int),
        "bc_exact": ([vp, i64, ctypes.POINTER(bc_opts), vp], ctypes.c_int),
        "bc_sources": ([vp, i64, vp, i32, ctypes.POINTER(bc_opts), vp], ctypes.c_int),
        "bc_submit": ([vp, i64, vp, i32, ctypes.POINTER(bc_opts), i64p], ctypes.c_int),
        "bc_poll": ([vp, i64, vp, ctypes.POINTER(bc_stats)], ctypes.c_int),
        "bc_wait": ([vp, i64, i64, vp, ctypes.POINTER(bc_stats)], ctypes.c_int),
        "bc_last_stats": ([vp, ctypes.POINTER(bc_stats)], ctypes.c_int),
        "bc_debug_source": ([vp, i64, i32, vp, vp, vp], ctypes.c_int),
        "bc_debug_graph": ([vp, i64, vp, vp, vp, vp], ctypes.c_int),
        "bc_create_graphs": ([vp, i32, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "bc_debug_sources": ([vp, i64, vp, i32, ctypes.POINTER(bc_opts), vp, vp, vp],
                             ctypes.c_int),
        "bc_exact_many": ([vp, vp, i32, ctypes.POINTER(bc_opts), vp], ctypes.c_int),
        "bc_debug_inject_barrier_skip": ([vp, i32, i32], ctypes.c_int),
        "bc_status_str": ([ctypes.c_int], ctypes.c_char_p),
        "bc_sources_noalloc": ([vp, vp, vp, vp, i32, i64, vp, i32, i32, vp, vp], ctypes.c_int),
        "bc_sources_estimate": ([vp, i64, vp, i32, ctypes.POINTER(bc_opts), vp, vp], ctypes.c_int),
        "bc_last_overflow_sources": ([vp, vp, i32, i32p], ctypes.c_int),
        "bc_sources_adaptive": ([vp, i64, vp, i32, i32, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(bc_opts), vp, vp, i32p], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib
