"""Python access to the CPU oracle for particle data binning (Sec. 4.2).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package; the CUDA library and
its Python binding never do. The arithmetic lives in ``binning_oracle.c``
(plain C, FP64 Neumaier sums, compiled with ``-ffp-contract=off``); this file
only builds it with gcc and marshals numpy arrays through ctypes.

Readings of the paper that the oracle fixes (R1-R7) are listed at the top of
``binning_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "binning_oracle.c")
_SRC_THREADED = os.path.join(_HERE, "binning_threaded.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_NO_MEMORY = -3
ERR_DEGENERATE = -7
MAX_ATTR = 16
MAX_RES = 65536

_lock = threading.Lock()
_lib = None


class Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("res", ctypes.c_int32 * 2), ("auto_bounds", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC_THREADED),
                                                   os.path.getmtime(_SRC[:-1] + "h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-pthread", "-shared", "-o", tmp, _SRC, _SRC_THREADED, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.bno_bin_f64.restype = ctypes.c_int
            L.bno_bin_f64.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, P, ctypes.POINTER(Grid),
                                      P, P, P, P, P, P]
            L.bno_bin_f32.restype = ctypes.c_int
            L.bno_bin_f32.argtypes = L.bno_bin_f64.argtypes
            for nm in ("bno_setup_axes_f64", "bno_setup_axes_f32"):
                f = getattr(L, nm)
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.POINTER(Grid), P, P, ctypes.c_int64, P, P, P]
            for nm in ("bno_state_init_f64", "bno_state_init_f32"):
                f = getattr(L, nm)
                f.restype = None
                f.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, P]
            for nm in ("bno_accumulate_f64", "bno_accumulate_f32"):
                f = getattr(L, nm)
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, P, ctypes.POINTER(Grid),
                              P, P, P, P, P, P, P, P]
            for nm in ("bno_state_merge_f64", "bno_state_merge_f32"):
                f = getattr(L, nm)
                f.restype = None
                f.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 10
            for nm in ("bno_bin_threaded_f64", "bno_bin_threaded_f32"):
                f = getattr(L, nm)
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, P, ctypes.POINTER(Grid),
                              ctypes.c_int, P, P, P, P, P]
            L.bno_finalize.restype = None
            L.bno_finalize.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, P]
            for nm in ("bno_particle_bin_f64", "bno_particle_bin_f32"):
                f = getattr(L, nm)
                f.restype = ctypes.c_int
                ft = ctypes.c_double if nm.endswith("64") else ctypes.c_float
                f.argtypes = [ft, ft, P, P, P, P, ctypes.c_int, P]
            _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}")
        self.code = code


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def make_grid(lo=(0.0, 0.0), hi=(1.0, 1.0), res=(64, 64), auto_bounds=False) -> Grid:
    g = Grid()
    g.lo[0], g.lo[1] = float(lo[0]), float(lo[1])
    g.hi[0], g.hi[1] = float(hi[0]), float(hi[1])
    g.res[0], g.res[1] = int(res[0]), int(res[1])
    g.auto_bounds = 1 if auto_bounds else 0
    return g


def _columns(x, y, attrs):
    x = np.ascontiguousarray(x)
    dt = x.dtype
    if dt not in (np.float32, np.float64):
        raise TypeError("coordinates must be float32 or float64")
    y = np.ascontiguousarray(y, dtype=dt)
    attrs = [np.ascontiguousarray(a, dtype=dt) for a in attrs]
    n = x.shape[0]
    if y.shape[0] != n or any(a.shape[0] != n for a in attrs):
        raise ValueError("column lengths differ")
    return x, y, attrs, dt


def bin_particles(x, y, attrs: Sequence[np.ndarray], lo=(0.0, 0.0), hi=(1.0, 1.0),
                  res=(64, 64), auto_bounds=False) -> Dict[str, np.ndarray]:
    """Bin (x, y) onto a res[0] x res[1] mesh; reduce every attribute.

    Returns count[B] u64, sum/avg[A, B] f64, min/max[A, B] in T, and
    bounds = (lo_x, hi_x, lo_y, hi_y) as used (in T, widened to f64).
    Bins are row-major: b = iy * res[0] + ix.
    """
    x, y, attrs, dt = _columns(x, y, attrs)
    n, A = x.shape[0], len(attrs)
    if A > MAX_ATTR:
        raise ValueError("too many attributes")
    g = make_grid(lo, hi, res, auto_bounds)
    B = int(res[0]) * int(res[1])
    count = np.zeros(B, np.uint64)
    s = np.zeros((A, B), np.float64)
    avg = np.zeros((A, B), np.float64)
    mn = np.zeros((A, B), dt)
    mx = np.zeros((A, B), dt)
    bounds = np.zeros(4, np.float64)
    ptrs = (ctypes.c_void_p * max(A, 1))(*[_ptr(a) for a in attrs])
    fn = lib().bno_bin_f64 if dt == np.float64 else lib().bno_bin_f32
    st = fn(n, _ptr(x), _ptr(y), A, ctypes.cast(ptrs, ctypes.c_void_p), ctypes.byref(g),
            _ptr(count), _ptr(s), _ptr(mn), _ptr(mx), _ptr(avg), _ptr(bounds))
    if st != OK:
        raise OracleError(st)
    return {"count": count, "sum": s, "min": mn, "max": mx, "avg": avg, "bounds": bounds}


def bin_particles_threaded(x, y, attrs: Sequence[np.ndarray], lo=(0.0, 0.0), hi=(1.0, 1.0),
                           res=(64, 64), auto_bounds=False, threads: int = 0) -> Dict[str, np.ndarray]:
    """bin_particles on `threads` host threads (0: every core this process
    may run on): one private mesh per thread, then a merge
    (binning_threaded.c). The all-core CPU baseline; same outputs."""
    x, y, attrs, dt = _columns(x, y, attrs)
    n, A = x.shape[0], len(attrs)
    if A > MAX_ATTR:
        raise ValueError("too many attributes")
    if threads <= 0:
        threads = len(os.sched_getaffinity(0))
    g = make_grid(lo, hi, res, auto_bounds)
    B = int(res[0]) * int(res[1])
    count = np.zeros(B, np.uint64)
    s = np.zeros((A, B), np.float64)
    avg = np.zeros((A, B), np.float64)
    mn = np.zeros((A, B), dt)
    mx = np.zeros((A, B), dt)
    ptrs = (ctypes.c_void_p * max(A, 1))(*[_ptr(a) for a in attrs])
    fn = lib().bno_bin_threaded_f64 if dt == np.float64 else lib().bno_bin_threaded_f32
    st = fn(n, _ptr(x), _ptr(y), A, ctypes.cast(ptrs, ctypes.c_void_p), ctypes.byref(g), int(threads),
            _ptr(count), _ptr(s), _ptr(mn), _ptr(mx), _ptr(avg))
    if st != OK:
        raise OracleError(st)
    return {"count": count, "sum": s, "min": mn, "max": mx, "avg": avg}


def bin_workload(w, auto_bounds=False) -> Dict[str, np.ndarray]:
    """bin_particles on a ``workloads.Workload``."""
    return bin_particles(w.x, w.y, w.attrs, w.lo, w.hi, w.res, auto_bounds)


def particle_bin(x, y, lo, hi, s, res, closed=False, dtype=np.float64):
    """(ix, iy) of one particle, or None when it is outside (R1-R3)."""
    lo_a = np.asarray(lo, np.float64)
    hi_a = np.asarray(hi, np.float64)
    s_a = np.asarray(s, np.float64)
    r_a = np.asarray(res, np.int32)
    out = np.zeros(2, np.int32)
    fn = lib().bno_particle_bin_f64 if dtype == np.float64 else lib().bno_particle_bin_f32
    ok = fn(x, y, _ptr(lo_a), _ptr(hi_a), _ptr(s_a), _ptr(r_a), 1 if closed else 0, _ptr(out))
    return (int(out[0]), int(out[1])) if ok else None


def setup_axes(x, y, lo=(0.0, 0.0), hi=(1.0, 1.0), res=(64, 64), auto_bounds=False):
    """lo_T, hi_T and s_T per axis as the oracle uses them (widened to f64)."""
    x = np.ascontiguousarray(x)
    dt = x.dtype
    y = np.ascontiguousarray(y, dtype=dt)
    g = make_grid(lo, hi, res, auto_bounds)
    lo_o, hi_o, s_o = (np.zeros(2, np.float64) for _ in range(3))
    fn = lib().bno_setup_axes_f64 if dt == np.float64 else lib().bno_setup_axes_f32
    st = fn(ctypes.byref(g), _ptr(x), _ptr(y), x.shape[0], _ptr(lo_o), _ptr(hi_o), _ptr(s_o))
    if st != OK:
        raise OracleError(st)
    return lo_o, hi_o, s_o


class State:
    """Partial per-bin state (count, Neumaier pair, min, max) of one shard,
    for shard-and-merge checks (the per-rank partial meshes of Sec. 4.2)."""

    def __init__(self, res, n_attrs, dtype):
        self.res = (int(res[0]), int(res[1]))
        self.B = self.res[0] * self.res[1]
        self.A = n_attrs
        self.dtype = np.dtype(dtype)
        self.count = np.zeros(self.B, np.uint64)
        self.s = np.zeros((n_attrs, self.B), np.float64)
        self.c = np.zeros((n_attrs, self.B), np.float64)
        self.mn = np.zeros((n_attrs, self.B), self.dtype)
        self.mx = np.zeros((n_attrs, self.B), self.dtype)
        init = lib().bno_state_init_f64 if self.dtype == np.float64 else lib().bno_state_init_f32
        init(self.B, self.A, _ptr(self.count), _ptr(self.s), _ptr(self.c), _ptr(self.mn),
             _ptr(self.mx))

    def accumulate(self, x, y, attrs, axes, auto_bounds=False):
        x, y, attrs, dt = _columns(x, y, attrs)
        assert dt == self.dtype and len(attrs) == self.A
        lo, hi, s = (np.ascontiguousarray(v, np.float64) for v in axes)
        g = make_grid(lo, hi, self.res, auto_bounds)
        ptrs = (ctypes.c_void_p * max(self.A, 1))(*[_ptr(a) for a in attrs])
        fn = lib().bno_accumulate_f64 if dt == np.float64 else lib().bno_accumulate_f32
        st = fn(x.shape[0], _ptr(x), _ptr(y), self.A, ctypes.cast(ptrs, ctypes.c_void_p),
                ctypes.byref(g), _ptr(lo), _ptr(hi), _ptr(s), _ptr(self.count), _ptr(self.s),
                _ptr(self.c), _ptr(self.mn), _ptr(self.mx))
        if st != OK:
            raise OracleError(st)
        return self

    def merge(self, other: "State"):
        fn = lib().bno_state_merge_f64 if self.dtype == np.float64 else lib().bno_state_merge_f32
        fn(self.B, self.A, _ptr(self.count), _ptr(self.s), _ptr(self.c), _ptr(self.mn),
           _ptr(self.mx), _ptr(other.count), _ptr(other.s), _ptr(other.c), _ptr(other.mn),
           _ptr(other.mx))
        return self

    def finalize(self) -> Dict[str, np.ndarray]:
        s = np.zeros((self.A, self.B), np.float64)
        avg = np.zeros((self.A, self.B), np.float64)
        lib().bno_finalize(self.B, self.A, _ptr(self.count), _ptr(self.s), _ptr(self.c),
                           _ptr(s), _ptr(avg))
        return {"count": self.count.copy(), "sum": s, "min": self.mn.copy(),
                "max": self.mx.copy(), "avg": avg}
