"""GB300-native particle data binning (Sec. 4.2 of the SENSEI extensions paper).

A thin Python binding over ``libbinning.so`` (C ABI in ``include/binning.h``).
Functions named ``bn_*`` mirror the C entry points and only marshal
arguments: torch tensors become ``bn_buffer`` handles (pointer, length,
stride, dtype, device, owning stream), and every step of the binning runs in
the library's CUDA kernels. There is no CPU fallback: if the library is not
built, every call raises.

PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

from . import _abi
from ._abi import (CTX_PROFILE, ALLOC_CUDA_ASYNC, ALLOC_EXTERNAL, ALLOC_HOST, ALLOC_PINNED, ALLOC_TORCH,
                   ERR_BUDGET, ERR_CUDA, ERR_DEGENERATE, ERR_DEVICE_MISMATCH, ERR_INTERNAL,
                   ERR_INVALID_ARG, ERR_NO_MEMORY, ERR_TIMEOUT, F32, F64, HOST, MAX_ATTR,
                   MAX_BINS, MAX_RES, NOT_READY, OK, OP_ACCUMULATE, OP_ALL, OP_AVG, OP_COUNT,
                   OP_MAX, OP_MIN, OP_SUM, STRATEGY_AUTO, STRATEGY_GLOBAL, STRATEGY_MASK,
                   STRATEGY_PRIVATE, STRATEGY_SORT, STRATEGY_HYBRID, SUM_F32, SUM_F32C, SUM_F64, SUM_MASK, U64,
                   AGG_AUTO, AGG_ON, AGG_OFF, AGG_MASK,
                   MAX_MULTI_COLS, MAX_MULTI_SPECS,
                   bn_block, bn_buffer, bn_grid, bn_grid_spec, bn_options, bn_result,
                   bn_server_options, bn_server_stats, bn_request_timing)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbinning.so")
_lib = None


class BinningError(RuntimeError):
    """A bn_* call returned an error status."""

    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded libbinning.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libbinning.so is not built (expected at %s); run "
                "paper_2310_02926_gb300.build.build() first -- there is no CPU fallback" % LIB_PATH)
        _lib = _abi.bind(ctypes.CDLL(LIB_PATH))
    return _lib


def build(force: bool = False) -> str:
    from .build import build as _build
    return _build(force=force)


def check(st: int) -> int:
    if st < 0:
        raise BinningError(st, lib().bn_last_error().decode(errors="replace"))
    return st


# --------------------------------------------------------------- marshalling
def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    if t.dtype in (torch.int64, getattr(torch, "uint64", torch.int64)):
        return U64
    raise TypeError(f"unsupported dtype {t.dtype}")


def buffer(t, stream: Optional[int] = None) -> bn_buffer:
    """A borrowed bn_buffer view of a 1-D torch tensor (CUDA or CPU)."""
    torch = _torch()
    if t.dim() != 1:
        raise ValueError("columns must be 1-D tensors")
    b = bn_buffer()
    b.ptr = t.data_ptr() if t.numel() else None
    b.n = t.numel()
    b.stride = t.stride(0) if t.numel() else 1
    b.dtype = dtype_code(t)
    if t.is_cuda:
        b.device = t.device.index if t.device.index is not None else torch.cuda.current_device()
        b.stream = stream if stream is not None else torch.cuda.current_stream(t.device).cuda_stream
        b.alloc = ALLOC_TORCH
    else:
        b.device = HOST
        b.stream = None
        b.alloc = ALLOC_PINNED if t.is_pinned() else ALLOC_HOST
    return b


def grid(lo=(0.0, 0.0), hi=(1.0, 1.0), res=(64, 64), auto_bounds=False) -> bn_grid:
    g = bn_grid()
    g.lo[0], g.lo[1] = float(lo[0]), float(lo[1])
    g.hi[0], g.hi[1] = float(hi[0]), float(hi[1])
    g.res[0], g.res[1] = int(res[0]), int(res[1])
    g.auto_bounds = 1 if auto_bounds else 0
    return g


def alloc_outputs(n_attrs: int, bins: int, dtype, device, ops: int = OP_ALL,
                  bounds: bool = False) -> Dict[str, object]:
    """torch tensors for every requested output of one mesh.

    count is int64 storage (the library writes u64; counts stay below 2^63)."""
    torch = _torch()
    out: Dict[str, object] = {}
    if ops & OP_COUNT:
        out["count"] = torch.empty(bins, dtype=torch.int64, device=device)
    for key, flag, dt in (("sum", OP_SUM, torch.float64), ("min", OP_MIN, dtype),
                          ("max", OP_MAX, dtype), ("avg", OP_AVG, torch.float64)):
        if ops & flag:
            out[key] = [torch.empty(bins, dtype=dt, device=device) for _ in range(n_attrs)]
    if bounds:
        out["bounds"] = torch.empty(4, dtype=torch.float64, device=device)
    return out


def result_struct(out: Dict[str, object], stream=None) -> bn_result:
    r = bn_result()
    if "count" in out:
        b = buffer(out["count"], stream)
        b.dtype = U64
        r.count = b
    for key in ("sum", "min", "max", "avg"):
        for a, t in enumerate(out.get(key, [])):
            getattr(r, key)[a] = buffer(t, stream)
    if "bounds" in out:
        r.bounds = buffer(out["bounds"], stream)
    return r


# --------------------------------------------------------------- C mirrors
def bn_context_create(device: int = 0, stream: Optional[int] = None, priority: int = 0,
                      flags: int = 0) -> int:
    opt = bn_options()
    opt.stream = stream
    opt.stream_priority = priority
    opt.flags = flags
    h = ctypes.c_void_p()
    check(lib().bn_context_create(device, ctypes.byref(opt), ctypes.byref(h)))
    return h.value


def bn_context_destroy(ctx: int) -> None:
    check(lib().bn_context_destroy(ctx))


def bn_context_stream(ctx: int) -> int:
    s = ctypes.c_void_p()
    check(lib().bn_context_stream(ctx, ctypes.byref(s)))
    return s.value or 0


STRATEGY_NAMES = {STRATEGY_PRIVATE: "private", STRATEGY_GLOBAL: "global", STRATEGY_SORT: "sort",
                  STRATEGY_HYBRID: "hybrid"}


def bn_context_profile(ctx: int):
    """(total device ms, launches, last strategy name) of the particle-pass
    kernels since the last call."""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    st = ctypes.c_int32()
    check(lib().bn_context_profile(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(st)))
    return ms.value, n.value, STRATEGY_NAMES.get(st.value, "none")


def bn_context_autotune_report(ctx: int) -> str:
    buf = ctypes.create_string_buffer(16384)
    check(lib().bn_context_autotune_report(ctx, buf, len(buf)))
    return buf.value.decode()


def bn_context_launch_count(ctx: int) -> int:
    n = ctypes.c_uint64()
    check(lib().bn_context_launch_count(ctx, ctypes.byref(n)))
    return n.value


def bn_bin_particles(ctx: int, x, y, attrs: Sequence, g: bn_grid, ops: int,
                     out: bn_result, sync: bool = True) -> Optional[int]:
    """Bin x, y (torch tensors) with attribute columns into `out` (a
    bn_result, e.g. from result_struct). Returns a request handle when
    sync is False."""
    n_attrs = len(attrs)
    arr = (bn_buffer * max(n_attrs, 1))(*[buffer(a) for a in attrs])
    bx, by = buffer(x), buffer(y)
    req = ctypes.c_void_p()
    check(lib().bn_bin_particles(ctx, ctypes.byref(bx), ctypes.byref(by), arr, n_attrs,
                                 ctypes.byref(g), ops, ctypes.byref(out), 1 if sync else 0,
                                 None if sync else ctypes.byref(req)))
    return None if sync else req.value


def bn_merge_results(ctx: int, parts: Sequence[bn_result], dtype: int, n_attrs: int,
                     bins: int, ops: int, out: bn_result, sync: bool = True) -> Optional[int]:
    arr = (bn_result * len(parts))(*parts)
    req = ctypes.c_void_p()
    check(lib().bn_merge_results(ctx, arr, len(parts), dtype, n_attrs, bins, ops,
                                 ctypes.byref(out), 1 if sync else 0,
                                 None if sync else ctypes.byref(req)))
    return None if sync else req.value


def bn_bin_batch(ctx: int, blocks: Sequence[bn_block], ops: int, sync: bool = True) -> Optional[int]:
    arr = (bn_block * max(len(blocks), 1))(*blocks)
    req = ctypes.c_void_p()
    check(lib().bn_bin_batch(ctx, arr, len(blocks), ops, 1 if sync else 0,
                             None if sync else ctypes.byref(req)))
    return None if sync else req.value


def grid_spec(x: int, y: int, attrs: Sequence[int], g: bn_grid) -> bn_grid_spec:
    """One binning of bn_bin_multi: column indices of its coordinates and
    attributes, and its mesh."""
    sp = bn_grid_spec()
    sp.x, sp.y = int(x), int(y)
    sp.n_attrs = len(attrs)
    for k, a in enumerate(attrs):
        sp.attrs[k] = int(a)
    sp.grid = g
    return sp


def bn_bin_multi(ctx: int, cols: Sequence, specs: Sequence[bn_grid_spec], ops: int,
                 outs: Sequence[bn_result], sync: bool = True,
                 stream: Optional[int] = None) -> Optional[int]:
    """Fused multi-grid pass over torch columns; outs[k] receives spec k."""
    carr = (bn_buffer * len(cols))(*[buffer(t, stream) for t in cols])
    sarr = (bn_grid_spec * len(specs))(*specs)
    oarr = (bn_result * len(outs))(*outs)
    req = ctypes.c_void_p()
    check(lib().bn_bin_multi(ctx, carr, len(cols), sarr, len(specs), ops, oarr, 1 if sync else 0,
                             None if sync else ctypes.byref(req)))
    return None if sync else req.value


def bn_exchange_bytes(bins: int, n_attrs: int) -> int:
    return int(lib().bn_exchange_bytes(bins, n_attrs))


def bn_exchange_pack(ctx: int, partial: bn_result, dtype: int, n_attrs: int, bins: int, exchange,
                     sync: bool = True) -> Optional[int]:
    """Pack a rank's result into the exchange buffer (a CUDA uint8 tensor of
    bn_exchange_bytes bytes)."""
    req = ctypes.c_void_p()
    check(lib().bn_exchange_pack(ctx, ctypes.byref(partial), dtype, n_attrs, bins, exchange.data_ptr(),
                                 1 if sync else 0, None if sync else ctypes.byref(req)))
    return None if sync else req.value


def bn_exchange_unpack(ctx: int, exchange, dtype: int, n_attrs: int, bins: int, ops: int, out: bn_result,
                       sync: bool = True) -> Optional[int]:
    req = ctypes.c_void_p()
    check(lib().bn_exchange_unpack(ctx, exchange.data_ptr(), dtype, n_attrs, bins, ops, ctypes.byref(out),
                                   1 if sync else 0, None if sync else ctypes.byref(req)))
    return None if sync else req.value


def bn_select_device(rank: int, n_avail: int, n_use: int = 0, stride: int = 0, offset: int = 0) -> int:
    """The paper's automatic placement rule (Eq. 1) for this rank."""
    d = ctypes.c_int(-1)
    check(lib().bn_select_device(rank, n_use, stride, offset, n_avail, ctypes.byref(d)))
    return d.value


def exchange_sections(exchange, bins: int, n_attrs: int):
    """Views of the exchange buffer's four sections (count, sum, minkey,
    maxkey) as int64 / float64 tensors; counts stay below 2^63."""
    torch = _torch()
    B, A = int(bins), int(n_attrs)
    e = exchange.view(torch.uint8)
    cut = [0, 8 * B, 8 * B * (1 + A), 8 * B * (1 + 2 * A), 8 * B * (1 + 3 * A)]
    types = (torch.int64, torch.float64, torch.int64, torch.int64)
    return [e[cut[k]:cut[k + 1]].view(types[k]) for k in range(4)]


def allreduce_exchange(exchange, bins: int, n_attrs: int, group=None) -> None:
    """Combine the exchange buffers of every rank of `group` in place: counts
    and sums with SUM, min keys with MIN, max keys with MAX (one collective
    per section). A gloo group reduces CPU copies of CUDA sections."""
    import torch.distributed as dist
    ops = (dist.ReduceOp.SUM, dist.ReduceOp.SUM, dist.ReduceOp.MIN, dist.ReduceOp.MAX)
    host_only = dist.get_backend(group) == "gloo"
    for sec, op in zip(exchange_sections(exchange, bins, n_attrs), ops):
        if sec.numel() == 0:
            continue
        if host_only and sec.is_cuda:
            tmp = sec.cpu()
            dist.all_reduce(tmp, op=op, group=group)
            sec.copy_(tmp)
        else:
            dist.all_reduce(sec, op=op, group=group)


def reduce_across_ranks(ctx: "Context", partial: Dict[str, object], dtype: int, n_attrs: int, bins: int,
                        ops: int = OP_ALL, group=None,
                        out: Optional[Dict[str, object]] = None) -> Dict[str, object]:
    """The whole mesh from every rank's partial result (count, sum, min, max):
    pack, one collective per section, unpack (avg recomputed)."""
    torch = _torch()
    dev = torch.device("cuda", ctx.device)
    ex = torch.empty(bn_exchange_bytes(bins, n_attrs), dtype=torch.uint8, device=dev)
    bn_exchange_pack(ctx.handle, result_struct(partial), dtype, n_attrs, bins, ex)
    allreduce_exchange(ex, bins, n_attrs, group)
    if out is None:
        tdt = torch.float64 if dtype == F64 else torch.float32
        out = alloc_outputs(n_attrs, bins, tdt, dev, ops | OP_COUNT)
    bn_exchange_unpack(ctx.handle, ex, dtype, n_attrs, bins, ops, result_struct(out))
    return out


def bn_query(req: int) -> int:
    return check(lib().bn_query(req))


def bn_wait(req: int, timeout_us: int = -1) -> int:
    return check(lib().bn_wait(req, timeout_us))


def bn_request_release(req: int) -> None:
    check(lib().bn_request_release(req))


def bn_server_create(ctx: int, budget_bytes: int, max_inflight: int = 4, max_batch: int = 64,
                     priority: int = 0, staging_bytes: int = 0) -> int:
    o = bn_server_options()
    o.budget_bytes = budget_bytes
    o.staging_bytes = staging_bytes
    o.max_inflight = max_inflight
    o.max_batch = max_batch
    o.stream_priority = priority
    h = ctypes.c_void_p()
    check(lib().bn_server_create(ctx, ctypes.byref(o), ctypes.byref(h)))
    return h.value


def bn_server_submit(srv: int, block: bn_block, ops: int) -> int:
    req = ctypes.c_void_p()
    check(lib().bn_server_submit(srv, ctypes.byref(block), ops, ctypes.byref(req)))
    return req.value


def bn_server_request_timing(req: int) -> Optional[Dict[str, float]]:
    """Timing record of a completed server request (None while it runs)."""
    t = bn_request_timing()
    st = lib().bn_server_request_timing(req, ctypes.byref(t))
    if st == NOT_READY:
        return None
    check(st)
    return {k: getattr(t, k) for k, _ in bn_request_timing._fields_}


def bn_server_stats_get(srv: int) -> Dict[str, int]:
    s = bn_server_stats()
    check(lib().bn_server_stats_get(srv, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in bn_server_stats._fields_}


def bn_server_destroy(srv: int) -> None:
    check(lib().bn_server_destroy(srv))


def bn_nbody_step(pos, vel, acc, state: ctypes.c_int, dt: float, eps: float,
                  stream: Optional[int] = None) -> None:
    """One leapfrog step of the direct-sum gravity producer (harness, not
    binning). pos/vel/acc: CUDA float32 tensors of shape (n, 4)."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream(pos.device).cuda_stream
    check(lib().bn_nbody_step(pos.data_ptr(), vel.data_ptr(), acc.data_ptr(), ctypes.byref(state),
                              pos.shape[0], dt, eps, s))


def bn_version() -> str:
    return lib().bn_version().decode()


def block(x, y, attrs: Sequence, g: bn_grid, out: bn_result, stream: Optional[int] = None) -> bn_block:
    """A bn_block over torch tensors; keep `out` alive while it is in use.
    stream: owning stream of the columns (default: torch's current stream)."""
    b = bn_block()
    b.x = buffer(x, stream)
    b.y = buffer(y, stream)
    for a, t in enumerate(attrs):
        b.attrs[a] = buffer(t, stream)
    b.n_attrs = len(attrs)
    b.grid = g
    b.out = ctypes.pointer(out)
    return b


# --------------------------------------------------------------- convenience
class Context:
    """A binning context on one CUDA device (owns a bn_context)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None, priority: int = 0,
                 profile: bool = False):
        self.device = device
        self.handle = bn_context_create(device, stream, priority,
                                        _abi.CTX_PROFILE if profile else 0)

    def close(self):
        if self.handle:
            bn_context_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self) -> int:
        return bn_context_stream(self.handle)

    @property
    def launches(self) -> int:
        return bn_context_launch_count(self.handle)

    def bin_particles(self, x, y, attrs: Sequence = (), lo=(0.0, 0.0), hi=(1.0, 1.0),
                      res=(64, 64), auto_bounds: bool = False, ops: int = OP_ALL,
                      out: Optional[Dict[str, object]] = None, bounds: bool = False,
                      sync: bool = True):
        """Bin torch columns; returns a dict of output tensors (allocated on
        the context's device unless `out` is given). With sync=False returns
        (outputs, request handle)."""
        torch = _torch()
        bins = int(res[0]) * int(res[1])
        if out is None:
            dev = torch.device("cuda", self.device)
            out = alloc_outputs(len(attrs), bins, x.dtype, dev, ops, bounds)
        r = result_struct(out)
        g = grid(lo, hi, res, auto_bounds)
        req = bn_bin_particles(self.handle, x, y, attrs, g, ops, r, sync)
        return out if sync else (out, req)


def loaded_library_path() -> Optional[str]:
    return LIB_PATH if _lib is not None else None
