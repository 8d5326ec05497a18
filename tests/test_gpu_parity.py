"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Counts, bin indices, min and max bit-exact; FP64 sums within 1e-12 and
FP32-compensated sums within 1e-6 of the per-bin sum of |a|. Sizes are
chosen so the oracle finishes in seconds while the kernels still run many
tiles with ragged tails; the slow tests run the full benchmark sizes.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
import workloads
from _parity import TOL_F32C, TOL_F64, abs_sums, assert_parity, run_gpu, to_numpy_result

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bn():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def ctx(bn):
    c = bn.Context(0)
    yield c
    c.close()


def check(w, gpu, tol, auto_bounds=False, label=""):
    ref = oracle.bin_workload(w, auto_bounds)
    sabs = abs_sums(w, auto_bounds) if w.attrs else None
    return assert_parity(gpu, ref, sabs, tol, label=label), ref


# ------------------------------------------------------------------ configs
@pytest.mark.parametrize("strategy", ["auto", "private", "global"])
def test_uniform64_f64_config(bn, ctx, strategy):
    """100,000 uniform particles, f64, 64x64 over [0,1)^2, all ops."""
    w = workloads.uniform(100_000, seed=0, dtype=np.float64, res=64)
    flags = {"auto": 0, "private": bn.STRATEGY_PRIVATE, "global": bn.STRATEGY_GLOBAL}[strategy]
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64, label=strategy)


STRAT = {"auto": 0, "private": "STRATEGY_PRIVATE", "global": "STRATEGY_GLOBAL", "sort": "STRATEGY_SORT",
         "hybrid": "STRATEGY_HYBRID"}


def sflag(bn, name):
    v = STRAT[name]
    return v if isinstance(v, int) else getattr(bn, v)


@pytest.mark.parametrize("strategy", ["auto", "global", "sort", "hybrid"])
def test_plummer_f64_reduced(bn, ctx, strategy):
    """Plummer sphere projected on x-y, 3 f64 attributes, 1024x1024 over [-10,10]^2."""
    w = workloads.plummer(2_000_003, seed=1, dtype=np.float64, res=1024)
    flags = sflag(bn, strategy)
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64, label=strategy)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sort_splits_dense_bucket_across_items(bn, ctx, dtype):
    """300,000 particles in one bin and 100,000 spread out: the dense bucket
    holds more records than one work item, so its items merge atomically."""
    rng = np.random.default_rng(31)
    n1, n2 = 300_000, 100_000
    x = np.concatenate([np.full(n1, 0.3141), rng.random(n2)]).astype(dtype)
    y = np.concatenate([np.full(n1, 0.2718), rng.random(n2)]).astype(dtype)
    p = rng.permutation(n1 + n2)
    a = [rng.normal(0, 1, n1 + n2).astype(dtype)[p], rng.uniform(-5, 5, n1 + n2).astype(dtype)[p]]
    w = workloads.Workload("dense", x[p], y[p], a, (0.0, 0.0), (1.0, 1.0), (600, 500))
    check(w, run_gpu(ctx, w, flags=bn.STRATEGY_SORT), TOL_F64 if dtype == np.float64 else TOL_F32C)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_autotuned_calls_repeat_exactly(bn, dtype):
    """A fresh context tunes on the first call of a shape (global may get a
    shared-memory window over the densest bins); later calls reuse the
    choice. Every call must match the oracle."""
    c = bn.Context(0)
    try:
        for seed in (51, 52, 53):
            w = workloads.plummer(3_000_000, seed=seed, dtype=dtype, res=1024)
            check(w, run_gpu(c, w), TOL_F64 if dtype == np.float64 else TOL_F32C, label=f"seed {seed}")
    finally:
        c.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n_attrs", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("aggregate", [False, True])
def test_global_key_records_any_attribute_count(bn, ctx, dtype, n_attrs, aggregate):
    """Global strategy: each bin's min/max keys form one record of all
    attributes, padded to 32-byte pieces (read with 256-bit loads); every
    attribute count, odd or past one piece, and both commit paths."""
    rng = np.random.default_rng(60 + n_attrs)
    n = 300_001
    x = rng.normal(0.5, 0.15, n).astype(dtype)
    y = rng.normal(0.5, 0.15, n).astype(dtype)
    attrs = [rng.standard_normal(n).astype(dtype) * (k + 1) for k in range(n_attrs)]
    attrs[0][::97] = np.nan
    w = workloads.Workload("records", x, y, attrs, (0.0, 0.0), (1.0, 1.0), (300, 200))
    flags = bn.STRATEGY_GLOBAL | (bn.AGG_ON if aggregate else bn.AGG_OFF)
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64 if dtype == np.float64 else TOL_F32C)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n_attrs", [0, 1, 2, 3, 4])
def test_hybrid_window_any_attribute_count(bn, ctx, dtype, n_attrs):
    """Hybrid strategy: a centred shared-memory window (fixed-point sums)
    plus global atomics around it; particles both inside and outside it,
    every attribute count the window kernel is compiled for."""
    w = workloads.plummer(400_001, seed=80 + n_attrs, dtype=dtype, res=1024)
    rng = np.random.default_rng(90 + n_attrs)
    w.attrs = [rng.standard_normal(w.n).astype(dtype) * 10.0 ** k for k in range(n_attrs)]
    if n_attrs == 0:
        got = run_gpu(ctx, w, ops=bn.OP_COUNT, flags=bn.STRATEGY_HYBRID)
        np.testing.assert_array_equal(got["count"], oracle.bin_workload(w)["count"])
        return
    check(w, run_gpu(ctx, w, flags=bn.STRATEGY_HYBRID), TOL_F64 if dtype == np.float64 else TOL_F32C)


def test_hybrid_rejects_more_than_four_attributes(bn, ctx):
    w = workloads.plummer(10_000, seed=3, dtype=np.float64, res=64)
    w.attrs = [w.x.copy() for _ in range(5)]
    with pytest.raises(bn.BinningError) as e:
        run_gpu(ctx, w, flags=bn.STRATEGY_HYBRID)
    assert e.value.code == bn.ERR_INVALID_ARG


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_hybrid_fixed_point_ranges(bn, ctx, dtype):
    """Window sums are fixed-point integers with a scale chosen from the
    first values each CTA reads. Values outside that scale's range (tiny,
    huge, subnormal, +-inf, NaN), signed zeros, long runs of carries and
    borrows, and a second half of the input a million times larger than the
    sampled first half all go through it; counts, min and max stay exact,
    sums within tolerance, integer-valued sums exact."""
    rng = np.random.default_rng(123)
    n = 600_001
    half = n // 2
    x = np.clip(rng.normal(0.5, 0.02, n), 0.0, 0.999).astype(dtype)
    y = np.clip(rng.normal(0.5, 0.02, n), 0.0, 0.999).astype(dtype)
    big = np.float64(2.0 ** 100 if dtype == np.float64 else 2.0 ** 60)
    wide = (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-30, 30, n)).astype(dtype)
    carry = np.where(np.arange(n) % 2 == 0, 1.0, -1.0) * (1.75 + rng.random(n) * 1e-3)
    carry = carry.astype(dtype)
    special = rng.uniform(-1, 1, n).astype(dtype)
    special[::101] = np.nan
    special[1::103] = np.inf
    special[2::107] = -np.inf
    special[3::109] = -0.0
    special[4::113] = 0.0
    special[5::127] = np.finfo(dtype).smallest_subnormal
    special[6::131] = -np.finfo(dtype).smallest_subnormal
    special[7::137] = big
    step = np.where(np.arange(n) < half, 1e-3, 1e3).astype(dtype) * rng.uniform(1, 2, n).astype(dtype)
    ones = np.ones(n, dtype=dtype)
    w = workloads.Workload("ranges", x, y, [wide, carry, special, step], (0.0, 0.0), (1.0, 1.0),
                           (512, 512))
    gpu = run_gpu(ctx, w, flags=bn.STRATEGY_HYBRID)
    check(w, gpu, TOL_F64 if dtype == np.float64 else TOL_F32C)
    w1 = workloads.Workload("ones", x, y, [ones], (0.0, 0.0), (1.0, 1.0), (512, 512))
    g1 = run_gpu(ctx, w1, flags=bn.STRATEGY_HYBRID)
    ref = oracle.bin_workload(w1)
    np.testing.assert_array_equal(g1["sum"][0], ref["sum"][0])


@pytest.mark.parametrize("strategy", ["private", "global", "hybrid"])
def test_min_max_with_tied_extremes(bn, ctx, strategy):
    """Attributes whose values tie at a bin's extreme (a constant column, a
    two-valued column, signed zeros): every tied particle reaches the exact
    keys; results stay exact."""
    rng = np.random.default_rng(71)
    n = 500_000
    x = rng.random(n)
    y = rng.random(n)
    const = np.full(n, 1.25)
    two = np.where(rng.random(n) < 0.5, -3.0, 7.0)
    zeros = np.where(rng.random(n) < 0.5, -0.0, 0.0)
    w = workloads.Workload("ties", x, y, [const, two, zeros], (0.0, 0.0), (1.0, 1.0), (48, 40))
    check(w, run_gpu(ctx, w, flags=sflag(bn, strategy)), TOL_F64)


def test_tuned_private_class_with_a_larger_mesh(bn):
    """A shape class spans a factor of two in bins: after the class tunes to
    the private strategy on a 64x64 mesh, a 90x90 mesh of the same class
    (too large for one CTA's shared memory) still bins, on another strategy."""
    c = bn.Context(0)
    try:
        for side in (64, 90):
            w = workloads.uniform(1 << 23, seed=80 + side, res=side)
            check(w, run_gpu(c, w), TOL_F64, label=f"{side}^2")
            if side == 64:
                assert "-> private" in bn.bn_context_autotune_report(c.handle)
    finally:
        c.close()


def test_private_rejects_mesh_too_large_for_shared_memory(bn, ctx):
    w = workloads.plummer(10_000, seed=2, dtype=np.float64, res=1024)
    with pytest.raises(bn.BinningError) as e:
        run_gpu(ctx, w, flags=bn.STRATEGY_PRIVATE)
    assert e.value.code == bn.ERR_INVALID_ARG


@pytest.mark.parametrize("res,strategy", [(1024, "global"), (64, "private"), (128, "global"),
                                          (1024, "sort"), (128, "sort")])
@pytest.mark.parametrize("mode", ["f32c", "f32", "f64"])
def test_gaussians_f32_sum_modes(bn, ctx, res, strategy, mode):
    """16-Gaussian mixture, f32 columns; the three sum modes against the FP64 oracle."""
    w = workloads.gaussians(2 ** 21 + 13, seed=3, res=res)
    flags = {"f32c": bn.SUM_F32C, "f32": bn.SUM_F32, "f64": bn.SUM_F64}[mode]
    flags |= sflag(bn, strategy)
    gpu = run_gpu(ctx, w, flags=flags)
    ref = oracle.bin_workload(w)
    sabs = abs_sums(w)
    if mode == "f32" and strategy in ("private", "sort"):
        # plain FP32 partials: exact counts/min/max; sums bounded by the
        # number of terms a CTA adds into one bin times 2^-24
        assert_parity(gpu, ref, sabs, 1.0, label=mode)
        rel = np.abs(gpu["sum"] - ref["sum"]) / np.where(sabs > 0, sabs, 1)
        assert rel.max() < 1e-3
    else:
        tol = TOL_F64 if mode == "f64" or strategy == "global" else TOL_F32C
        assert_parity(gpu, ref, sabs, tol, label=f"{mode}/{strategy}")


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["private", "global", "sort", "hybrid"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 31, 33, 1023, 1025, 4095, 4097, 70_001])
def test_ragged_lengths(bn, ctx, dtype, strategy, n):
    w = workloads.uniform(n, seed=4 + n, dtype=dtype, res=16)
    flags = sflag(bn, strategy)
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64 if dtype == np.float64 else TOL_F32C,
          label=f"n={n}")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["private", "global", "sort", "hybrid"])
@pytest.mark.parametrize("offsets", [(1, 1, 1, 1), (1, 2, 3, 0), (3, 3, 3, 3)])
def test_misaligned_columns(bn, ctx, dtype, strategy, offsets):
    """Sub-range views whose starts are not 16-byte aligned (same or mixed phase)."""
    w = workloads.uniform(50_000, seed=5, dtype=dtype, res=32)
    dev = torch.device("cuda", 0)
    n = w.n - 4
    full = [torch.from_numpy(c).to(dev) for c in (w.x, w.y, *w.attrs)]
    cols = [t[o:o + n] for t, o in zip(full, offsets)]
    host = [np.ascontiguousarray(c[o:o + n]) for c, o in zip((w.x, w.y, *w.attrs), offsets)]
    wv = workloads.Workload("view", host[0], host[1], host[2:], w.lo, w.hi, w.res)
    flags = sflag(bn, strategy)
    out = ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res, ops=bn.OP_ALL | flags)
    torch.cuda.synchronize()
    check(wv, to_numpy_result(out), TOL_F64 if dtype == np.float64 else TOL_F32C)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["auto", "private", "global", "hybrid", "sort"])
@pytest.mark.parametrize("auto_bounds", [False, True])
def test_strided_columns(bn, ctx, dtype, strategy, auto_bounds):
    """Array-of-structs columns (a record of 7 values, the columns at
    different offsets in it) read in place by the particle pass (private,
    global, hybrid), or gathered first (sort); with explicit and automatic
    bounds, and a length that leaves ragged tails."""
    w = workloads.plummer(150_001, seed=6, dtype=dtype, res=40 if strategy == "private" else 300)
    rng = np.random.default_rng(7)
    aos = np.stack([rng.random(w.n).astype(dtype), w.y, w.attrs[2], w.x, w.attrs[0],
                    rng.random(w.n).astype(dtype), w.attrs[1]], axis=1)
    t = torch.from_numpy(aos).to("cuda")
    flags = sflag(bn, strategy)
    out = ctx.bin_particles(t[:, 3], t[:, 1], [t[:, 4], t[:, 6], t[:, 2]], w.lo, w.hi, w.res,
                            auto_bounds, bn.OP_ALL | flags)
    torch.cuda.synchronize()
    check(w, to_numpy_result(out), TOL_F64 if dtype == np.float64 else TOL_F32C, auto_bounds=auto_bounds,
          label=strategy)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["private", "global", "sort", "hybrid"])
def test_special_values(bn, ctx, dtype, strategy):
    rng = np.random.default_rng(7)
    n = 20_000
    x = rng.uniform(-0.2, 1.2, n).astype(dtype)
    y = rng.uniform(-0.2, 1.2, n).astype(dtype)
    a = rng.normal(0, 1, n).astype(dtype)
    b = rng.uniform(-1, 1, n).astype(dtype)
    x[::97] = np.nan
    y[5::101] = np.inf
    x[7::103] = -np.inf
    x[11::89] = 0.0
    x[13::89] = -0.0
    y[17::83] = 1.0           # == hi: outside (half-open)
    x[19::79] = np.nextafter(dtype(1.0), dtype(0.0))
    a[::53] = np.nan
    a[3::59] = -0.0
    a[4::61] = 0.0
    b[::67] = np.inf
    b[1::71] = -np.inf
    w = workloads.Workload("special", x, y, [a, b], (0.0, 0.0), (1.0, 1.0), (8, 8))
    flags = sflag(bn, strategy)
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64 if dtype == np.float64 else TOL_F32C)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("agg", ["AGG_ON", "AGG_OFF"])
def test_global_record_sums_edge_values(bn, ctx, dtype, agg):
    """Global strategy, whose count and sums reach L2 as one bulk reduction of
    each bin's record: bins holding only subnormal values, normal values that
    cancel through the subnormal range, infinities, NaN and signed zeros,
    several warps of particles per bin. Each of these sums is exact in any
    order of addition, so it must equal the oracle's bit for bit."""
    rng = np.random.default_rng(41)
    per, nb = 700, 8
    tiny = float(np.finfo(np.float64).smallest_subnormal)  # 2^-1074
    half_min = 2.0 ** -1023
    f = np.finfo(dtype)

    def case(k):
        if k == 0:  # subnormal (f64) / smallest f32 subnormal multiples
            unit = tiny if dtype == np.float64 else float(f.smallest_subnormal)
            return rng.integers(-50, 51, per) * unit
        if k == 1:
            # normal values 3u, -2u, 4u (u = 2^-1023 for f64, 2^-127 for f32)
            # in random order: the partial sums cross zero and the subnormal
            # range, and the total is u, itself subnormal
            unit = half_min if dtype == np.float64 else 2.0 ** -127
            return rng.permutation(np.array([3.0] * 279 + [-2.0] * 420 + [4.0])) * unit
        if k == 2:
            v = rng.normal(0, 1, per)
            v[rng.integers(per)] = np.inf
            return v
        if k == 3:
            v = rng.normal(0, 1, per)
            v[:2] = [np.inf, -np.inf]
            return v
        if k == 4:
            v = rng.normal(0, 1, per)
            v[rng.integers(per)] = np.nan
            return v
        if k == 5:
            return np.full(per, -0.0)
        return rng.normal(0, 1, per)

    xs, ys, cols = [], [], [[], [], []]
    for b in range(nb - 1):  # the last bin stays empty
        xs.append(np.full(per, (b % 4 + 0.5) / 4))
        ys.append(np.full(per, (b // 4 + 0.5) / 2))
        for a in range(3):
            cols[a].append(case((b + 2 * a) % (nb - 1)))
    p = rng.permutation(per * (nb - 1))
    x = np.concatenate(xs)[p].astype(dtype)
    y = np.concatenate(ys)[p].astype(dtype)
    attrs = [np.concatenate(c)[p].astype(dtype) for c in cols]
    w = workloads.Workload("record-edges", x, y, attrs, (0.0, 0.0), (1.0, 1.0), (4, 2))
    flags = bn.STRATEGY_GLOBAL | getattr(bn, agg)
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64 if dtype == np.float64 else TOL_F32C, label=agg)


F64_GRIDS = [
    ((-10.0, -10.0), (10.0, 10.0), (1024, 1024)),
    ((-1.3, 0.1), (2.7, 0.35), (37, 5)),
    ((0.0, 0.0), (1.0, 1.0), (3, 7)),
    ((1e6, -3.0), (1e6 + 1.0, 3.0), (1000, 3)),    # too fine for the FP32 estimate
    ((-1e-3, 5.0), (2e-3, 5.0 + 1e-9), (999, 17)),
    ((1e300, -1e300), (2e300, 1e300), (16, 9)),     # FP32 estimate overflows: search only
    ((1e-300, 0.0), (2e-300, 1.0), (5, 5)),         # bin width below FP32 range
]


@pytest.mark.parametrize("grid", F64_GRIDS)
@pytest.mark.parametrize("strategy", ["private", "global", "sort", "hybrid"])
def test_f64_bin_edges_exact(bn, ctx, grid, strategy):
    """Particles on and within a few ulp of every bin edge: indices must
    follow the round-to-nearest sequence exactly (via the edge-key method)."""
    lo, hi, res = grid
    if strategy == "private" and res[0] * res[1] * 4 * 8 > 200_000:
        pytest.skip("mesh does not fit shared memory")
    pts = []
    for a in range(2):
        s = res[a] / (hi[a] - lo[a])
        for i in range(0, res[a] + 1, max(1, res[a] // 64)):
            e = lo[a] + i / s
            for k in range(-3, 4):
                v = e
                step = np.inf if k > 0 else -np.inf
                for _ in range(abs(k)):
                    v = np.nextafter(v, step)
                pts.append((a, v))
    rng = np.random.default_rng(8)
    n = len(pts)
    x = rng.uniform(lo[0], hi[0], n)
    y = rng.uniform(lo[1], hi[1], n)
    for k, (a, v) in enumerate(pts):
        (x if a == 0 else y)[k] = v
    m = rng.uniform(1, 2, n)
    w = workloads.Workload("edges", x, y, [m], lo, hi, res)
    flags = sflag(bn, strategy)
    check(w, run_gpu(ctx, w, flags=flags), TOL_F64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["private", "global", "sort", "hybrid"])
def test_auto_bounds(bn, ctx, dtype, strategy):
    w = workloads.plummer(300_001, seed=9, dtype=dtype, res=40)
    w.x[::1000] = np.nan
    flags = sflag(bn, strategy)
    gpu = run_gpu(ctx, w, flags=flags, auto_bounds=True, bounds=True)
    (_, ref) = check(w, gpu, TOL_F64 if dtype == np.float64 else TOL_F32C, auto_bounds=True)
    assert gpu["bounds"].tolist() == ref["bounds"].tolist()


def test_auto_bounds_degenerate_reports_error(bn, ctx):
    x = torch.full((1000,), 3.0, dtype=torch.float64, device="cuda")
    y = torch.linspace(0, 1, 1000, dtype=torch.float64, device="cuda")
    with pytest.raises(bn.BinningError) as e:
        ctx.bin_particles(x, y, [], res=(4, 4), auto_bounds=True)
    assert e.value.code == bn.ERR_DEGENERATE
    out, req = ctx.bin_particles(x, y, [], res=(4, 4), auto_bounds=True, sync=False)
    with pytest.raises(bn.BinningError) as e:
        bn.bn_wait(req, 5_000_000)
    assert e.value.code == bn.ERR_DEGENERATE
    bn.bn_request_release(req)
    # the context stays usable
    w = workloads.uniform(1000, seed=10, res=4)
    check(w, run_gpu(ctx, w), TOL_F64)


# ------------------------------------------------------------------ data model
def test_host_inputs_and_outputs(bn, ctx):
    """Location-agnostic access: host columns are staged to the device, host
    outputs are copied back."""
    w = workloads.uniform(123_457, seed=11, dtype=np.float64, res=32)
    cols = [torch.from_numpy(c) for c in (w.x, w.y, *w.attrs)]
    out = bn.alloc_outputs(2, 32 * 32, torch.float64, torch.device("cpu"))
    ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res, out=out)
    check(w, to_numpy_result(out), TOL_F64)
    pinned = [c.pin_memory() for c in cols]
    out2 = bn.alloc_outputs(2, 32 * 32, torch.float64, torch.device("cpu"))
    ctx.bin_particles(pinned[0], pinned[1], pinned[2:], w.lo, w.hi, w.res, out=out2)
    check(w, to_numpy_result(out2), TOL_F64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["auto", "private", "global", "sort", "hybrid"])
@pytest.mark.parametrize("auto_bounds", [False, True])
def test_pinned_host_columns_read_in_place(bn, ctx, dtype, strategy, auto_bounds):
    """Page-locked host columns are read by the kernels over the host link;
    slices start inside the pinned block at odd element offsets."""
    w = workloads.plummer(400_003, seed=19, dtype=dtype, res=40)
    off = 3
    pinned = [torch.from_numpy(np.concatenate([np.zeros(off, c.dtype), c])).pin_memory()
              for c in (w.x, w.y, *w.attrs)]
    cols = [t[off:] for t in pinned]
    out = bn.alloc_outputs(3, 40 * 40, cols[0].dtype, torch.device("cuda"))
    ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res, auto_bounds,
                      bn.OP_ALL | sflag(bn, strategy), out=out)
    torch.cuda.synchronize()
    check(w, to_numpy_result(out), TOL_F64 if dtype == np.float64 else TOL_F32C,
          auto_bounds=auto_bounds)


def test_library_allocated_outputs(bn, ctx):
    w = workloads.uniform(50_000, seed=12, dtype=np.float32, res=20)
    cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
    r = bn.bn_result()  # every handle zeroed: the library allocates
    bn.bn_bin_particles(ctx.handle, cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res),
                        bn.OP_ALL, r, True)
    B = 400
    assert r.count.ptr and r.count.alloc == bn.ALLOC_CUDA_ASYNC and r.count.n == B

    cudart = ctypes.CDLL("libcudart.so.13")

    def fetch(buf, dt):
        tdt = {np.uint64: torch.int64, np.float64: torch.float64, np.float32: torch.float32}[dt]
        t = torch.empty(B, dtype=tdt, device="cuda")
        torch.cuda.synchronize()
        rc = cudart.cudaMemcpy(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(buf.ptr),
                               ctypes.c_size_t(B * t.element_size()), 3)  # device to device
        assert rc == 0
        return t.cpu().numpy().view(dt)

    gpu = {"count": fetch(r.count, np.uint64),
           "sum": np.stack([fetch(r.sum[a], np.float64) for a in range(2)]),
           "min": np.stack([fetch(r.min[a], np.float32) for a in range(2)]),
           "max": np.stack([fetch(r.max[a], np.float32) for a in range(2)]),
           "avg": np.stack([fetch(r.avg[a], np.float64) for a in range(2)])}
    check(w, gpu, TOL_F32C)
    bn.lib().bn_buffer_release(ctypes.byref(r.count))
    assert not r.count.ptr
    for a in range(2):
        for key in ("sum", "min", "max", "avg"):
            bn.lib().bn_buffer_release(ctypes.byref(getattr(r, key)[a]))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("strategy", ["auto", "private", "global", "sort", "hybrid"])
def test_accumulate_shards_into_one_state(bn, ctx, dtype, strategy):
    """Shards binned one after another into the same outputs (BN_OP_ACCUMULATE)
    equal the whole set binned at once, whatever strategy each shard takes."""
    res = 32 if strategy == "private" else 128  # the private mesh must fit shared memory
    w = workloads.plummer(400_000, seed=13, dtype=dtype, res=res)
    cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
    out = bn.alloc_outputs(3, res * res, cols[0].dtype, torch.device("cuda"))
    cuts = [0, 1, 150_000, 150_003, w.n]
    for k, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
        ops = bn.OP_ALL | (bn.OP_ACCUMULATE if k else 0) | sflag(bn, strategy)
        ctx.bin_particles(cols[0][a:b], cols[1][a:b], [c[a:b] for c in cols[2:]], w.lo, w.hi,
                          w.res, ops=ops, out=out)
    torch.cuda.synchronize()
    check(w, to_numpy_result(out), TOL_F64 if dtype == np.float64 else TOL_F32C)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_merge_partial_results(bn, ctx, dtype):
    """Shard, bin each shard, merge the partial meshes (the per-rank merge)."""
    w = workloads.plummer(300_000, seed=14, dtype=dtype, res=64)
    cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
    B = 64 * 64
    parts, structs = [], []
    for a, b in ((0, 100_000), (100_000, 100_001), (100_001, w.n)):
        o = ctx.bin_particles(cols[0][a:b], cols[1][a:b], [c[a:b] for c in cols[2:]], w.lo,
                              w.hi, w.res)
        parts.append(o)
        structs.append(bn.result_struct(o))
    merged = bn.alloc_outputs(3, B, cols[0].dtype, torch.device("cuda"))
    bn.bn_merge_results(ctx.handle, structs, bn.F64 if dtype == np.float64 else bn.F32, 3, B,
                        bn.OP_ALL, bn.result_struct(merged), True)
    check(w, to_numpy_result(merged), TOL_F64 if dtype == np.float64 else TOL_F32C)


def test_batch_of_uneven_blocks(bn, ctx):
    plan = workloads.batch(n_blocks=12, seed=15, size_range=(1e3, 2e5), side_range=(8, 600))
    blocks, outs, keep = [], [], []
    for k in range(plan.n_blocks):
        w = plan.block(k)
        cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
        o = bn.alloc_outputs(2, w.res[0] * w.res[1], torch.float32, torch.device("cuda"))
        r = bn.result_struct(o)
        keep += [cols, r]
        outs.append((w, o))
        blocks.append(bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r))
    bn.bn_bin_batch(ctx.handle, blocks, bn.OP_ALL)
    torch.cuda.synchronize()
    for w, o in outs:
        check(w, to_numpy_result(o), TOL_F32C, label=w.name)


def _batch_blocks(bn, plan, dtype, host=False, scale=None):
    import torch as T
    blocks, outs, keep = [], [], []
    for k in range(plan.n_blocks):
        w = plan.block(k)
        if scale is not None:
            w.attrs = [a * scale for a in w.attrs]
        w.x, w.y = w.x.astype(dtype), w.y.astype(dtype)
        w.attrs = [a.astype(dtype) for a in w.attrs]
        dev = T.device("cpu") if host else T.device("cuda")
        cols = [T.from_numpy(np.ascontiguousarray(c)).to(dev) for c in (w.x, w.y, *w.attrs)]
        o = bn.alloc_outputs(2, w.res[0] * w.res[1], cols[0].dtype, T.device("cuda"))
        r = bn.result_struct(o)
        keep += [cols, r]
        outs.append((w, o))
        blocks.append(bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r))
    return blocks, outs, keep


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("strategy", ["auto", "private", "global", "sort"])
def test_batch_persistent_path(bn, ctx, dtype, strategy):
    """All-device batch: one persistent launch (graph-captured), every block
    checked against the oracle; then the same shapes with new values replay
    the cached graph."""
    plan = workloads.batch(n_blocks=20, seed=41, size_range=(1e3, 3e5),
                           side_range=(8, 40 if strategy == "private" else 700))
    tol = TOL_F64 if dtype == np.float64 else TOL_F32C
    flags = {"auto": 0, "private": bn.STRATEGY_PRIVATE, "global": bn.STRATEGY_GLOBAL,
             "sort": bn.STRATEGY_SORT}[strategy]
    per_replay = []
    for rep, scale in enumerate((None, -3.0, 0.5)):
        blocks, outs, keep = _batch_blocks(bn, plan, dtype, scale=scale)
        launches0 = ctx.launches
        bn.bn_bin_batch(ctx.handle, blocks, bn.OP_ALL | flags)
        torch.cuda.synchronize()
        if rep >= 1:
            per_replay.append(ctx.launches - launches0)
        if rep >= 1 and strategy in ("private", "global"):
            # a replay of the captured graph: init/edges, persistent pass, finalize
            assert ctx.launches - launches0 <= 4
        for w, o in outs:
            check(w, to_numpy_result(o), tol, label=f"{w.name} rep{rep}")
    # replays of one cached plan launch the same kernels (auto may put some
    # blocks on the sort path, whose chains add four launches each)
    assert per_replay[0] == per_replay[1] <= 3 + 4 * plan.n_blocks


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batch_private_in_mesh_bands(bn, ctx, dtype):
    """Private strategy forced on meshes larger than shared memory: each mesh
    is cut into bands of rows and every band of every tile is a work item of
    its own; every block against the oracle, then the same shapes again with
    new values (a replay of the cached graph)."""
    plan = workloads.batch(n_blocks=10, seed=43, size_range=(1e4, 4e5), side_range=(80, 220))
    tol = TOL_F64 if dtype == np.float64 else TOL_F32C
    for rep, scale in enumerate((None, 7.0)):
        blocks, outs, keep = _batch_blocks(bn, plan, dtype, scale=scale)
        bn.bn_bin_batch(ctx.handle, blocks, bn.OP_ALL | bn.STRATEGY_PRIVATE)
        torch.cuda.synchronize()
        for w, o in outs:
            check(w, to_numpy_result(o), tol, label=f"{w.name} rep{rep}")


def test_batch_general_path_with_host_columns(bn, ctx):
    plan = workloads.batch(n_blocks=5, seed=42, size_range=(1e3, 5e4), side_range=(8, 200))
    blocks, outs, keep = _batch_blocks(bn, plan, np.float32, host=True)
    bn.bn_bin_batch(ctx.handle, blocks, bn.OP_ALL)
    torch.cuda.synchronize()
    for w, o in outs:
        check(w, to_numpy_result(o), TOL_F32C, label=w.name)


def test_async_query_and_wait(bn, ctx):
    w = workloads.uniform(2_000_000, seed=16, dtype=np.float64, res=64)
    cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
    out, req = ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res, sync=False)
    st = bn.bn_query(req)
    assert st in (bn.OK, bn.NOT_READY)
    assert bn.bn_wait(req, 10_000_000) == bn.OK
    assert bn.bn_query(req) == bn.OK
    bn.bn_request_release(req)
    check(w, to_numpy_result(out), TOL_F64)


@pytest.mark.parametrize("ops_name", ["count", "count_avg", "min", "sum_max"])
def test_op_subsets(bn, ctx, ops_name):
    ops = {"count": bn.OP_COUNT, "count_avg": bn.OP_COUNT | bn.OP_AVG, "min": bn.OP_MIN,
           "sum_max": bn.OP_SUM | bn.OP_MAX}[ops_name]
    w = workloads.plummer(100_000, seed=17, dtype=np.float64, res=50)
    gpu = run_gpu(ctx, w, ops=ops)
    ref = oracle.bin_workload(w)
    if "count" not in gpu:
        gpu["count"] = ref["count"]
    assert_parity(gpu, ref, abs_sums(w), TOL_F64, check=tuple(k for k in gpu))


def test_invalid_arguments_are_reported(bn, ctx):
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    y = torch.zeros(11, dtype=torch.float64, device="cuda")
    with pytest.raises(bn.BinningError) as e:
        ctx.bin_particles(x, y, [])
    assert e.value.code == bn.ERR_INVALID_ARG
    y = torch.zeros(10, dtype=torch.float32, device="cuda")
    with pytest.raises(bn.BinningError):
        ctx.bin_particles(x, y, [])
    y = torch.zeros(10, dtype=torch.float64, device="cuda")
    for lo, hi, res in [((0, 0), (1, 1), (0, 4)), ((1, 0), (1, 1), (4, 4)),
                        ((0, 0), (1, 1), (70_000, 1)), ((0, 0), (math.inf, 1), (4, 4))]:
        with pytest.raises(bn.BinningError) as e:
            ctx.bin_particles(x, y, [], lo, hi, res)
        assert e.value.code == bn.ERR_INVALID_ARG
    many = (bn.bn_buffer * 17)(*[bn.buffer(x) for _ in range(17)])
    r = bn.bn_result()
    st = bn.lib().bn_bin_particles(ctx.handle, ctypes.byref(bn.buffer(x)), ctypes.byref(bn.buffer(y)),
                                   many, 17, ctypes.byref(bn.grid()), bn.OP_COUNT, ctypes.byref(r),
                                   1, None)
    assert st == bn.ERR_INVALID_ARG
    bx = bn.buffer(x)
    bx.device = torch.cuda.device_count()  # a device this process does not have
    by = bn.buffer(y)
    r = bn.bn_result()
    st = bn.lib().bn_bin_particles(ctx.handle, ctypes.byref(bx), ctypes.byref(by), None, 0,
                                   ctypes.byref(bn.grid()), bn.OP_COUNT, ctypes.byref(r), 1, None)
    assert st == bn.ERR_DEVICE_MISMATCH
    assert b"device" in bn.lib().bn_last_error()


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two GPUs (one per box here)")
@pytest.mark.parametrize("where", ["inputs", "outputs", "both"])
def test_columns_and_outputs_on_another_device(bn, where):
    """Location-agnostic access across devices: a context on device 0 bins
    columns that live on device 1 (copied peer to peer, strided ones
    included) and/or writes outputs that live on device 1."""
    w = workloads.plummer(200_001, seed=12, dtype=np.float64, res=128)
    d_in = torch.device("cuda", 1 if where in ("inputs", "both") else 0)
    d_out = torch.device("cuda", 1 if where in ("outputs", "both") else 0)
    aos = torch.from_numpy(np.stack([w.x, w.y, *w.attrs], axis=1)).to(d_in)
    cols = [aos[:, 0].contiguous(), aos[:, 1], aos[:, 2].contiguous(), aos[:, 3], aos[:, 4]]
    out = bn.alloc_outputs(3, 128 * 128, torch.float64, d_out)
    with bn.Context(0) as c:
        c.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res, out=out)
        torch.cuda.synchronize(0)
        torch.cuda.synchronize(1)
    check(w, to_numpy_result(out), TOL_F64, label=where)


# ------------------------------------------------------------------ serving
def test_server_results_equal_alone(bn, ctx):
    """Requests binned in the server's batches give the same result as alone."""
    plan = workloads.serving(n_requests=24, seed=18, size_range=(1e3, 3e5), side_range=(16, 300),
                             pool_n=400_000)
    pool = [torch.from_numpy(c).cuda() for c in (plan.pool.x, plan.pool.y, *plan.pool.attrs)]
    srv = bn.bn_server_create(ctx.handle, 1 << 28, max_inflight=3, max_batch=5)
    reqs = []
    for i in range(plan.n_requests):
        o0, n = int(plan.offsets[i]), int(plan.sizes[i])
        side = int(plan.sides[i])
        cols = [c[o0:o0 + n] for c in pool]
        o = bn.alloc_outputs(3, side * side, torch.float32, torch.device("cuda"))
        r = bn.result_struct(o)
        blk = bn.block(cols[0], cols[1], cols[2:], bn.grid((-10, -10), (10, 10), (side, side)), r)
        reqs.append((bn.bn_server_submit(srv, blk, bn.OP_ALL), o, r, blk, (o0, n, side)))
    for req, o, r, blk, (o0, n, side) in reqs:
        assert bn.bn_wait(req, 60_000_000) == bn.OK
        bn.bn_request_release(req)
    stats = bn.bn_server_stats_get(srv)
    bn.bn_server_destroy(srv)
    assert stats["completed"] == plan.n_requests and stats["failed"] == 0
    for req, o, r, blk, (o0, n, side) in reqs:
        alone = ctx.bin_particles(*[c[o0:o0 + n] for c in pool[:2]],
                                  [c[o0:o0 + n] for c in pool[2:]], (-10, -10), (10, 10), (side, side))
        torch.cuda.synchronize()
        g, a = to_numpy_result(o), to_numpy_result(alone)
        np.testing.assert_array_equal(g["count"], a["count"])
        np.testing.assert_array_equal(g["min"], a["min"])
        np.testing.assert_array_equal(g["max"], a["max"])
        w = workloads.Workload("req", plan.pool.x[o0:o0 + n], plan.pool.y[o0:o0 + n],
                               [c[o0:o0 + n] for c in plan.pool.attrs], (-10, -10), (10, 10),
                               (side, side))
        check(w, g, TOL_F32C)


def test_server_does_not_run_autotuner_trials(bn):
    """Server batches take tuned or heuristic strategies, never timed trials."""
    import paper_2310_02926_gb300 as pkg
    fresh = pkg.Context(0)
    w = workloads.uniform(n=1 << 17, seed=21, res=48)
    cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
    srv = bn.bn_server_create(fresh.handle, 1 << 28, max_inflight=2, max_batch=4)
    o = bn.alloc_outputs(len(w.attrs), 48 * 48, torch.float64, torch.device("cuda"))
    r = bn.result_struct(o)
    blk = bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r)
    req = bn.bn_server_submit(srv, blk, bn.OP_ALL)
    assert bn.bn_wait(req, 60_000_000) == bn.OK
    bn.bn_request_release(req)
    bn.bn_server_destroy(srv)
    assert bn.bn_context_autotune_report(fresh.handle) == ""
    check(w, to_numpy_result(o), TOL_F64)
    # a direct call of the same shape class does tune
    fresh.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res)
    torch.cuda.synchronize()
    assert "attrs=2" in bn.bn_context_autotune_report(fresh.handle)
    fresh.close()


@pytest.mark.parametrize("inputs", ["host", "device_tight_budget", "strided", "arena_overflow"])
def test_server_staging_paths(bn, ctx, inputs):
    """Requests whose columns are on the host (deep copy into the staging
    arena), or that arrive while the budget is used up (staged, admitted
    later), or whose columns are strided, or that find the staging arena
    full (a page-locked allocation of their own): every result equals
    binning the block alone, and the admission charge covers every
    request's temporaries."""
    rng = np.random.default_rng(61)
    n_req = 12
    sizes = rng.integers(20_000, 120_000, n_req)
    side = 48
    budget = 6 << 20 if inputs == "device_tight_budget" else 1 << 30
    staging = 1 << 20 if inputs == "arena_overflow" else 0
    srv = bn.bn_server_create(ctx.handle, budget, max_inflight=2, max_batch=3, staging_bytes=staging)
    reqs = []
    for i in range(n_req):
        w = workloads.plummer(int(sizes[i]), seed=100 + i, dtype=np.float32, res=side)
        w.attrs[2] = np.abs(w.attrs[2])
        if inputs in ("host", "arena_overflow"):
            cols = [torch.from_numpy(c) for c in (w.x, w.y, *w.attrs)]
        elif inputs == "strided":
            aos = torch.from_numpy(np.stack([w.x, w.y, *w.attrs], axis=1)).cuda()
            cols = [aos[:, k] for k in range(aos.shape[1])]
        else:
            cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
        o = bn.alloc_outputs(3, side * side, torch.float32, torch.device("cuda"))
        r = bn.result_struct(o)
        blk = bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r)
        reqs.append((bn.bn_server_submit(srv, blk, bn.OP_ALL), o, r, blk, cols, w))
    for req, *_ in reqs:
        assert bn.bn_wait(req, 60_000_000) == bn.OK
        t = bn.bn_server_request_timing(req)
        assert t is not None and t["batch_size"] >= 1 and t["submit_us"] >= 0 and t["batch_gpu_us"] > 0
        bn.bn_request_release(req)
    stats = bn.bn_server_stats_get(srv)
    bn.bn_server_destroy(srv)
    assert stats["completed"] == n_req and stats["failed"] == 0
    assert stats["overdrawn"] == 0
    if inputs == "device_tight_budget":
        assert stats["peak_bytes"] <= budget
    if inputs == "host":
        assert stats["staged"] == n_req and stats["staging_overflow"] == 0
    if inputs == "arena_overflow":
        assert stats["staging_overflow"] > 0
    for req, o, r, blk, cols, w in reqs:
        check(w, to_numpy_result(o), TOL_F32C, label=f"{inputs} {w.n}")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_server_charges_cover_temporaries(bn, dtype):
    """Requests of every strategy and shape class (min/max key records and
    their f64 filter, sort scratch, host outputs, avg without sum) through
    one server: what each request's plan allocates never exceeds what
    admission charged it, and every result matches the oracle."""
    c = bn.Context(0)
    srv = bn.bn_server_create(c.handle, 8 << 30, max_inflight=3, max_batch=4)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    cases = [  # (n, side, n_attrs, flags, ops, host outputs)
        (300_000, 1024, 3, bn.STRATEGY_GLOBAL, bn.OP_ALL, False),
        (400_000, 2048, 2, bn.STRATEGY_SORT, bn.OP_ALL, False),
        (200_000, 512, 3, bn.STRATEGY_HYBRID, bn.OP_ALL, False),
        (200_000, 40, 3, bn.STRATEGY_PRIVATE, bn.OP_ALL, False),
        (150_000, 700, 3, 0, bn.OP_COUNT | bn.OP_AVG | bn.OP_MIN, False),
        (150_000, 300, 2, 0, bn.OP_ALL, True),
    ]
    reqs = []
    try:
        for k, (n, side, A, flags, ops, host) in enumerate(cases):
            w = workloads.plummer(n, seed=500 + k, dtype=dtype, res=side, n_attrs=A)
            cols = [torch.from_numpy(x).cuda() for x in (w.x, w.y, *w.attrs)]
            dev = torch.device("cpu") if host else torch.device("cuda")
            o = bn.alloc_outputs(A, side * side, tdt, dev, ops=ops)
            if host:
                o = {kk: ([t.pin_memory() for t in v] if isinstance(v, list) else v.pin_memory())
                     for kk, v in o.items()}
            r = bn.result_struct(o)
            blk = bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r)
            reqs.append((bn.bn_server_submit(srv, blk, ops | flags), o, r, blk, cols, w, ops))
        for req, *_ in reqs:
            assert bn.bn_wait(req, 120_000_000) == bn.OK
            bn.bn_request_release(req)
        stats = bn.bn_server_stats_get(srv)
    finally:
        bn.bn_server_destroy(srv)
        c.close()
    assert stats["failed"] == 0 and stats["overdrawn"] == 0
    assert stats["peak_bytes"] <= 8 << 30
    tol = TOL_F64 if dtype == np.float64 else TOL_F32C
    for req, o, r, blk, cols, w, ops in reqs:
        got = to_numpy_result(o)
        ref = oracle.bin_workload(w)
        keys = [k for k in ("count", "sum", "min", "max", "avg") if k in got]
        assert_parity(got, ref, abs_sums(w), tol, check=keys, label=f"{w.n} {w.res}")


def test_nbody_producer_forces_match_float64_reference(bn):
    """The serving benchmark's producer (harness, not binning): after one
    step, the accelerations it keeps equal the direct sum over all pairs
    evaluated in float64 by plain torch, for a body count that spans two
    force chunks and a ragged tail."""
    import ctypes
    g = torch.Generator().manual_seed(3)
    n, eps = 5_003, 1e-2
    pos = torch.zeros(n, 4)
    pos[:, :3] = torch.randn(n, 3, generator=g)
    pos[:, 3] = torch.rand(n, generator=g) / n
    vel = torch.zeros(n, 4)
    dp, dv, da = pos.cuda(), vel.cuda(), torch.zeros(n, 4, device="cuda")
    ok = ctypes.c_int(0)
    bn.bn_nbody_step(dp, dv, da, ok, 0.0, eps)  # dt = 0: positions stay, forces of pos
    torch.cuda.synchronize()
    p = pos.double()
    got = da[:, :3].double().cpu()
    for i0 in range(0, n, 500):  # rows in blocks: the pair arrays stay small
        d = p[None, :, :3] - p[i0:i0 + 500, None, :3]
        r2 = (d ** 2).sum(-1) + eps * eps
        ref = (d * (p[None, :, 3] / r2 ** 1.5)[..., None]).sum(1)
        scale = (p[None, :, 3] / r2).sum(1)[:, None]  # sum of |term| bounds
        assert ((got[i0:i0 + 500] - ref).abs() <= 1e-4 * scale).all(), i0


def test_server_rejects_over_budget(bn, ctx):
    x = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    o = bn.alloc_outputs(0, 16, torch.float32, torch.device("cuda"), ops=bn.OP_COUNT)
    r = bn.result_struct(o)
    srv = bn.bn_server_create(ctx.handle, 1 << 20)
    blk = bn.block(x, x, [], bn.grid(res=(4, 4)), r)
    with pytest.raises(bn.BinningError) as e:
        bn.bn_server_submit(srv, blk, bn.OP_COUNT)
    assert e.value.code == bn.ERR_BUDGET
    bn.bn_server_destroy(srv)


# ------------------------------------------------------------------ full size
@pytest.mark.slow
def test_plummer_f64_full_size(bn, ctx):
    """50,000,000 Plummer particles, f64, 3 attributes, 1024x1024: the
    benchmark workload, in the launch configuration the benchmark times."""
    w = workloads.plummer(50_000_000, seed=0, dtype=np.float64, res=1024)
    check(w, run_gpu(ctx, w), TOL_F64, label="plummer full")


@pytest.mark.slow
def test_gaussians_f32_full_size(bn, ctx):
    """2^27 f32 particles from 16 Gaussians on a 4096x4096 mesh (compensated sums)."""
    w = workloads.gaussians(2 ** 27, seed=0, res=4096)
    check(w, run_gpu(ctx, w), TOL_F32C, label="gaussians full")


@pytest.mark.slow
def test_batch256_full_plan(bn, ctx):
    """The batching workload at full size: 256 blocks of log-uniform 1e3..1e7
    f32 particles, each with its own mesh (32^2..2048^2), in one
    bn_bin_batch call with the autotuned strategy per block (sort blocks
    included); every block against the oracle."""
    plan = workloads.batch(n_blocks=256, seed=0)
    blocks, outs, keep = [], [], []
    for k in range(plan.n_blocks):
        w = plan.block(k)
        cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
        o = bn.alloc_outputs(2, w.res[0] * w.res[1], torch.float32, torch.device("cuda"))
        r = bn.result_struct(o)
        keep += [cols, r]
        outs.append(o)
        blocks.append(bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r))
    for rep in range(2):  # the second call replays the cached graph
        for o in outs:
            for t in [o["count"], *o["sum"]]:
                t.fill_(3)
        bn.bn_bin_batch(ctx.handle, blocks, bn.OP_ALL)
        torch.cuda.synchronize()
    del keep
    for k in range(plan.n_blocks):
        w = plan.block(k)
        check(w, to_numpy_result(outs[k]), TOL_F32C, label=f"block {k} n={w.n} res={w.res}")
        outs[k] = None


@pytest.mark.slow
def test_multi_grid_phase_space_full(bn, ctx):
    """The fused multi-grid workload at full size: 2^22 f64 particles of a
    Plummer snapshot, 10 variables binned in 9 coordinate systems on 256^2
    meshes (the paper's 90 binnings per step), every spec against the oracle."""
    n, res = 2 ** 22, (256, 256)
    cols = workloads.phase_space(n, seed=0)
    names = list(cols)
    tcols = [torch.from_numpy(cols[k]).cuda() for k in names]
    variables = [names.index(v) for v in workloads.PHASE_SPACE_VARIABLES]
    specs, keep = [], []
    for (a, b) in workloads.PHASE_SPACE_SYSTEMS:
        ha, hb = workloads.PHASE_SPACE_BOUNDS[a], workloads.PHASE_SPACE_BOUNDS[b]
        specs.append(bn.grid_spec(names.index(a), names.index(b), variables, bn.grid((-ha, -hb), (ha, hb), res)))
        keep.append(bn.alloc_outputs(len(variables), res[0] * res[1], torch.float64, torch.device("cuda")))
    bn.bn_bin_multi(ctx.handle, tcols, specs, bn.OP_ALL, [bn.result_struct(o) for o in keep])
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(workloads.PHASE_SPACE_SYSTEMS):
        ha, hb = workloads.PHASE_SPACE_BOUNDS[a], workloads.PHASE_SPACE_BOUNDS[b]
        w = workloads.Workload(f"{a}-{b}", cols[a], cols[b], [cols[v] for v in workloads.PHASE_SPACE_VARIABLES],
                               (-ha, -hb), (ha, hb), res)
        check(w, to_numpy_result(keep[k]), TOL_F64, label=f"system {a}-{b}")


# ------------------------------------------------------------------ fused multi-grid pass
def _multi_columns(n, seed, dtype):
    """Positions and velocities of a Plummer-like cloud plus two scalars."""
    rng = np.random.default_rng(seed)
    pos = rng.standard_normal((3, n)) * 2.0
    vel = rng.standard_normal((3, n))
    mass = rng.uniform(1.0, 2.0, n)
    energy = 0.5 * mass * (vel ** 2).sum(0)
    return [c.astype(dtype) for c in (*pos, *vel, mass, energy)]


MULTI_SPECS = [  # (x, y, attrs, lo, hi, res): columns 0-2 x,y,z, 3-5 vx,vy,vz, 6 mass, 7 energy
    (0, 1, [6, 7], (-6.0, -6.0), (6.0, 6.0), (64, 64)),
    (0, 2, [6], (-6.0, -6.0), (6.0, 6.0), (50, 33)),
    (1, 2, [7, 3, 4], (-4.0, -5.0), (4.0, 5.0), (128, 96)),
    (3, 4, [6, 7], (-3.0, -3.0), (3.0, 3.0), (40, 40)),
    (0, 1, [0, 1, 6], (-1.0, -1.0), (1.0, 1.0), (300, 300)),   # coordinates as attributes
    (5, 6, [], (-2.0, 1.0), (2.0, 2.0), (7, 5)),               # count only, mass on an axis
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("where", ["device", "host"])
def test_multi_grid_matches_each_binning(bn, ctx, dtype, where):
    """bn_bin_multi: each spec's result equals binning its columns alone."""
    n = 70_001  # not a multiple of the tile
    cols = _multi_columns(n, 90, dtype)
    tcols = [torch.from_numpy(c) for c in cols]
    if where == "device":
        tcols = [t.cuda() for t in tcols]
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    specs, outs, keep = [], [], []
    for (x, y, attrs, lo, hi, res) in MULTI_SPECS:
        specs.append(bn.grid_spec(x, y, attrs, bn.grid(lo, hi, res)))
        o = bn.alloc_outputs(len(attrs), res[0] * res[1], tdt, torch.device("cuda"))
        keep.append(o)
        outs.append(bn.result_struct(o))
    bn.bn_bin_multi(ctx.handle, tcols, specs, bn.OP_ALL, outs)
    torch.cuda.synchronize()
    for k, (x, y, attrs, lo, hi, res) in enumerate(MULTI_SPECS):
        w = workloads.Workload(f"spec{k}", cols[x], cols[y], [cols[a] for a in attrs], lo, hi, res)
        got = to_numpy_result(keep[k])
        if attrs:
            check(w, got, TOL_F64, label=f"spec {k}")
        else:
            ref = oracle.bin_workload(w, False)
            np.testing.assert_array_equal(got["count"], ref["count"], err_msg=f"spec {k}")


def test_multi_grid_rejects_bad_arguments(bn, ctx):
    cols = [torch.zeros(10, dtype=torch.float64, device="cuda") for _ in range(3)]
    g = bn.grid((0, 0), (1, 1), (4, 4))
    o = bn.alloc_outputs(1, 16, torch.float64, torch.device("cuda"))
    r = bn.result_struct(o)
    bad = [
        ([bn.grid_spec(0, 3, [1], g)], bn.OP_ALL),                      # column out of range
        ([bn.grid_spec(0, 1, [7], g)], bn.OP_ALL),                      # attribute out of range
        ([bn.grid_spec(0, 1, [2], bn.grid((0, 0), (1, 1), (4, 4), auto_bounds=True))], bn.OP_ALL),
        ([bn.grid_spec(0, 1, [2], g)], bn.OP_ALL | bn.OP_ACCUMULATE),
        ([bn.grid_spec(0, 1, [2], g)], bn.OP_ALL | bn.STRATEGY_PRIVATE),
    ]
    for specs, ops in bad:
        with pytest.raises(bn.BinningError) as e:
            bn.bn_bin_multi(ctx.handle, cols, specs, ops, [r])
        assert e.value.code == bn.ERR_INVALID_ARG
    odd = [cols[0], cols[1], torch.zeros(9, dtype=torch.float64, device="cuda")]
    with pytest.raises(bn.BinningError):
        bn.bn_bin_multi(ctx.handle, odd, [bn.grid_spec(0, 1, [2], g)], bn.OP_ALL, [r])
