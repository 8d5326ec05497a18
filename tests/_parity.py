"""Helpers for the GPU-vs-oracle parity tests (no binning arithmetic here).

Counts, min and max must match the oracle bit for bit. Sums and averages
must satisfy |gpu - oracle| <= tol * S per bin, where S is the per-bin sum
of |a| (as the oracle bins it) and, for averages, S / count. Empty bins
must carry the exact fill values (sum +0.0, min +inf, max -inf, avg
0x7ff8000000000000).
"""
from __future__ import annotations

import numpy as np

import oracle

TOL_F64 = 1e-12   # FP64 accumulation (f64 data; f32 data in BN_SUM_F64)
TOL_F32C = 1e-6   # FP32 compensated partials merged in FP64
QNAN_BITS = 0x7FF8000000000000


def to_np(t):
    return t.detach().cpu().numpy()


def run_gpu(ctx, w, ops=None, flags=0, auto_bounds=False, bounds=False, device=0,
            host_inputs=False):
    """Bin a workloads.Workload on the GPU through the C ABI; numpy results."""
    import torch
    import paper_2310_02926_gb300 as bn
    ops = bn.OP_ALL if ops is None else ops
    dev = torch.device("cuda", device)
    if host_inputs:
        cols = [torch.from_numpy(np.ascontiguousarray(c)) for c in (w.x, w.y, *w.attrs)]
    else:
        cols = [torch.from_numpy(np.ascontiguousarray(c)).to(dev) for c in (w.x, w.y, *w.attrs)]
    out = ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res, auto_bounds,
                            ops | flags, bounds=bounds)
    torch.cuda.synchronize(dev)
    return to_numpy_result(out)


def to_numpy_result(out):
    res = {}
    for k, v in out.items():
        if isinstance(v, list):
            res[k] = np.stack([to_np(t) for t in v]) if v else np.zeros((0, 0))
        else:
            res[k] = to_np(v)
    if "count" in res:
        res["count"] = res["count"].astype(np.uint64)
    return res


def abs_sums(w, auto_bounds=False):
    """Per-bin sum of |a| for each attribute, binned by the oracle."""
    r = oracle.bin_particles(w.x, w.y, [np.abs(a) for a in w.attrs], w.lo, w.hi, w.res,
                             auto_bounds)
    return r["sum"]


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.int64 if a.dtype.itemsize == 8 else np.int32)


def assert_parity(gpu, ref, sabs, tol, check=("count", "sum", "min", "max", "avg"), label=""):
    """Raise AssertionError with a short report on the first mismatch."""
    if "count" in check and "count" in gpu:
        bad = np.nonzero(gpu["count"] != ref["count"])[0]
        assert bad.size == 0, f"{label} count differs in {bad.size} bins, first {bad[:5]}: " \
                              f"gpu {gpu['count'][bad[:5]]} oracle {ref['count'][bad[:5]]}"
    for key in ("min", "max"):
        if key in check and key in gpu:
            g, r = bits(gpu[key]), bits(ref[key])
            bad = np.argwhere(g != r)
            assert bad.size == 0, f"{label} {key} differs at {bad[:5].tolist()}: " \
                                  f"gpu {gpu[key][tuple(bad[0])]} oracle {ref[key][tuple(bad[0])]}"
    worst = {}
    if "sum" in check and "sum" in gpu:
        with np.errstate(invalid="ignore"):
            err = np.abs(gpu["sum"] - ref["sum"])
        lim = tol * sabs
        same = gpu["sum"] == ref["sum"]                   # includes +/-inf
        ok = same | (err <= lim) | (np.isnan(gpu["sum"]) & np.isnan(ref["sum"]))
        ok &= ~(np.isnan(gpu["sum"]) ^ np.isnan(ref["sum"]))
        bad = np.argwhere(~ok)
        assert bad.size == 0, f"{label} sum outside tol {tol} at {bad[:5].tolist()}: " \
                              f"gpu {gpu['sum'][tuple(bad[0])]!r} oracle {ref['sum'][tuple(bad[0])]!r} " \
                              f"sum|a| {sabs[tuple(bad[0])]!r}"
        empty = ref["count"] == 0
        assert (bits(gpu["sum"][:, empty]) == 0).all(), f"{label} empty-bin sums must be +0.0"
        with np.errstate(invalid="ignore", divide="ignore"):
            rel = np.where((sabs > 0) & np.isfinite(sabs), err / sabs, 0.0)
        worst["sum"] = float(np.nanmax(rel)) if rel.size else 0.0
    if "avg" in check and "avg" in gpu:
        cnt = ref["count"].astype(np.float64)
        empty = ref["count"] == 0
        assert (bits(gpu["avg"][:, empty]) == QNAN_BITS).all(), f"{label} empty-bin avg must be qNaN"
        ne = ~empty
        with np.errstate(invalid="ignore"):
            err = np.abs(gpu["avg"][:, ne] - ref["avg"][:, ne])
            lim = tol * sabs[:, ne] / cnt[ne]
        nan_both = np.isnan(gpu["avg"][:, ne]) & np.isnan(ref["avg"][:, ne])
        ok = (gpu["avg"][:, ne] == ref["avg"][:, ne]) | (err <= lim) | nan_both
        bad = np.argwhere(~ok)
        assert bad.size == 0, f"{label} avg outside tol {tol} at {bad[:5].tolist()}"
    return worst
