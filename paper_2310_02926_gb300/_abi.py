"""ctypes mirror of include/binning.h (struct layouts, constants, prototypes)."""
from __future__ import annotations

import ctypes
import os

MAX_ATTR = 16
MAX_RES = 65536
MAX_BINS = 1 << 30
HOST = -1

OK = 0
NOT_READY = 1
ERR_INVALID_ARG = -1
ERR_DEVICE_MISMATCH = -2
ERR_NO_MEMORY = -3
ERR_BUDGET = -4
ERR_TIMEOUT = -5
ERR_CUDA = -6
ERR_DEGENERATE = -7
ERR_INTERNAL = -8

F32 = 1
F64 = 2
U64 = 3

ALLOC_EXTERNAL = 0
ALLOC_TORCH = 1
ALLOC_CUDA_ASYNC = 2
ALLOC_HOST = 3
ALLOC_PINNED = 4

OP_COUNT = 1 << 0
OP_SUM = 1 << 1
OP_MIN = 1 << 2
OP_MAX = 1 << 3
OP_AVG = 1 << 4
OP_ALL = 0x1F
OP_ACCUMULATE = 1 << 5
SUM_F32C = 0 << 8
SUM_F32 = 1 << 8
SUM_F64 = 2 << 8
SUM_MASK = 3 << 8
STRATEGY_AUTO = 0 << 12
STRATEGY_PRIVATE = 1 << 12
STRATEGY_GLOBAL = 2 << 12
STRATEGY_SORT = 3 << 12
STRATEGY_HYBRID = 4 << 12
STRATEGY_MASK = 15 << 12
AGG_AUTO = 0 << 16
AGG_ON = 1 << 16
AGG_OFF = 2 << 16
AGG_MASK = 3 << 16

DELETER = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class bn_buffer(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("alloc", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("deleter", DELETER),
                ("deleter_ctx", ctypes.c_void_p)]


class bn_grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("res", ctypes.c_int32 * 2), ("auto_bounds", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class bn_result(ctypes.Structure):
    _fields_ = [("count", bn_buffer), ("sum", bn_buffer * MAX_ATTR),
                ("min", bn_buffer * MAX_ATTR), ("max", bn_buffer * MAX_ATTR),
                ("avg", bn_buffer * MAX_ATTR), ("bounds", bn_buffer)]


class bn_block(ctypes.Structure):
    _fields_ = [("x", bn_buffer), ("y", bn_buffer), ("attrs", bn_buffer * MAX_ATTR),
                ("n_attrs", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("grid", bn_grid), ("out", ctypes.POINTER(bn_result))]


class bn_grid_spec(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32), ("n_attrs", ctypes.c_int32),
                ("attrs", ctypes.c_int32 * MAX_ATTR), ("reserved", ctypes.c_int32),
                ("grid", bn_grid)]


MAX_MULTI_COLS = 64
MAX_MULTI_SPECS = 256

CTX_PROFILE = 1


class bn_options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("stream_priority", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("mempool_release_threshold", ctypes.c_size_t)]


class bn_server_options(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("stream_priority", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("staging_bytes", ctypes.c_size_t)]


class bn_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("staged", ctypes.c_uint64),
                ("staging_overflow", ctypes.c_uint64), ("overdrawn", ctypes.c_uint64)]


class bn_request_timing(ctypes.Structure):
    _fields_ = [("submit_us", ctypes.c_double), ("queue_us", ctypes.c_double),
                ("launch_us", ctypes.c_double), ("complete_us", ctypes.c_double),
                ("batch_gpu_us", ctypes.c_double), ("batch_size", ctypes.c_int32),
                ("staged", ctypes.c_int32)]


P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)
S = ctypes.c_int

# name -> (restype, argtypes); every entry point of include/binning.h
PROTOTYPES = {
    "bn_context_create": (S, [ctypes.c_int, ctypes.POINTER(bn_options), PP]),
    "bn_context_destroy": (S, [P]),
    "bn_context_stream": (S, [P, PP]),
    "bn_context_launch_count": (S, [P, ctypes.POINTER(ctypes.c_uint64)]),
    "bn_context_autotune_report": (S, [P, ctypes.c_char_p, ctypes.c_size_t]),
    "bn_context_profile": (S, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(ctypes.c_int32)]),
    "bn_bin_particles": (S, [P, ctypes.POINTER(bn_buffer), ctypes.POINTER(bn_buffer),
                             ctypes.POINTER(bn_buffer), ctypes.c_int, ctypes.POINTER(bn_grid),
                             ctypes.c_uint32, ctypes.POINTER(bn_result), ctypes.c_int, PP]),
    "bn_bin_particles_static": (S, [ctypes.POINTER(bn_buffer), ctypes.POINTER(bn_buffer),
                                    ctypes.POINTER(bn_buffer), ctypes.c_int,
                                    ctypes.POINTER(bn_grid), ctypes.c_uint32,
                                    ctypes.POINTER(bn_result), P, ctypes.c_int]),
    "bn_bin_batch": (S, [P, ctypes.POINTER(bn_block), ctypes.c_int, ctypes.c_uint32,
                         ctypes.c_int, PP]),
    "bn_bin_multi": (S, [P, ctypes.POINTER(bn_buffer), ctypes.c_int, ctypes.POINTER(bn_grid_spec),
                         ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(bn_result), ctypes.c_int, PP]),
    "bn_merge_results": (S, [P, ctypes.POINTER(bn_result), ctypes.c_int, ctypes.c_int32,
                             ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.POINTER(bn_result), ctypes.c_int, PP]),
    "bn_query": (S, [P]),
    "bn_wait": (S, [P, ctypes.c_int64]),
    "bn_request_release": (S, [P]),
    "bn_buffer_release": (S, [ctypes.POINTER(bn_buffer)]),
    "bn_server_create": (S, [P, ctypes.POINTER(bn_server_options), PP]),
    "bn_server_submit": (S, [P, ctypes.POINTER(bn_block), ctypes.c_uint32, PP]),
    "bn_server_stats_get": (S, [P, ctypes.POINTER(bn_server_stats)]),
    "bn_server_request_timing": (S, [P, ctypes.POINTER(bn_request_timing)]),
    "bn_exchange_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int]),
    "bn_exchange_pack": (S, [P, ctypes.POINTER(bn_result), ctypes.c_int32, ctypes.c_int, ctypes.c_int64,
                             P, ctypes.c_int, PP]),
    "bn_exchange_unpack": (S, [P, P, ctypes.c_int32, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                               ctypes.POINTER(bn_result), ctypes.c_int, PP]),
    "bn_select_device": (S, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)]),
    "bn_server_destroy": (S, [P]),
    "bn_nbody_step": (S, [P, P, P, ctypes.POINTER(ctypes.c_int), ctypes.c_int64, ctypes.c_float,
                          ctypes.c_float, P]),
    "bn_last_error": (ctypes.c_char_p, []),
    "bn_version": (ctypes.c_char_p, []),
}


def header_entry_points(path: str) -> list:
    """Names of the entry points declared in a header (or every header of a
    directory) under include/."""
    import glob
    import re
    paths = sorted(glob.glob(os.path.join(path, "*.h"))) if os.path.isdir(path) else [path]
    names = set()
    for p in paths:
        with open(p) as f:
            src = f.read()
        names.update(re.findall(r"^BN_API\s+[\w\s\*]+?\b(bn_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADER = os.path.join(INCLUDE, "binning.h")
