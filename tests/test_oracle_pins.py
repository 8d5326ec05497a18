"""Pins for the CPU oracle, checked against things other than itself.

Each test fixes a part of the oracle with something the paper or
mathematics decides: a hand-worked example of the Sec. 4.2 definition,
exact rational arithmetic (fractions.Fraction), correctly rounded sums
(math.fsum), closed forms, invariants, and numpy's histogram routines on
grids where the scaling is exact. None of these need a GPU.
"""
import json
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F64_EPS = 2.0 ** -53


# ---------------------------------------------------------------- helpers
def exact_bin(x, lo, hi, res, closed=False):
    """(bin, distance of the exact real t to the nearest integer) or None.

    lo and hi are the already-rounded bounds in T; the real t is
    (x - lo) * res / (hi - lo) evaluated exactly."""
    if math.isnan(x):
        return None
    inside = (lo <= x <= hi) if closed else (lo <= x < hi)
    if not inside:
        return None
    t = (Fraction(x) - Fraction(lo)) * res / (Fraction(hi) - Fraction(lo))
    k = math.floor(t)
    dist = min(t - k, k + 1 - t)
    return min(k, res - 1), dist


def group_by_exact_bins(x, y, lo, hi, res):
    """Map bin -> particle indices, using exact bins (tiny inputs only).
    Returns None for a particle within 1e-9 of an edge (ambiguous)."""
    groups = {}
    for k in range(len(x)):
        bx = exact_bin(float(x[k]), lo[0], hi[0], res[0])
        by = exact_bin(float(y[k]), lo[1], hi[1], res[1])
        if bx is None or by is None:
            continue
        if bx[1] < Fraction(1, 10 ** 9) or by[1] < Fraction(1, 10 ** 9):
            return None
        groups.setdefault(by[0] * res[0] + bx[0], []).append(k)
    return groups


def bits64(v):
    return struct.unpack("<Q", struct.pack("<d", float(v)))[0]


# ---------------------------------------------------------------- golden
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_handworked_fixture(dtype):
    with open(os.path.join(GOLDEN, "handworked_2x2.json")) as f:
        fx = json.load(f)
    g, p, e = fx["grid"], fx["particles"], fx["expected"]
    r = oracle.bin_particles(np.array(p["x"], dtype), np.array(p["y"], dtype),
                             [np.array(p["mass"], dtype)], g["lo"], g["hi"], g["res"])
    assert r["count"].tolist() == e["count"]
    conv = lambda v: float(v)  # "inf", "-inf", "nan" parse too
    np.testing.assert_array_equal(r["sum"][0], [conv(v) for v in e["sum"]])
    np.testing.assert_array_equal(r["min"][0], np.array([conv(v) for v in e["min"]], dtype))
    np.testing.assert_array_equal(r["max"][0], np.array([conv(v) for v in e["max"]], dtype))
    np.testing.assert_array_equal(r["avg"][0], [conv(v) for v in e["avg"]])


# ---------------------------------------------------------------- bin index
GRIDS = [
    ((0.0, 0.0), (1.0, 1.0), (64, 64)),
    ((-10.0, -10.0), (10.0, 10.0), (1024, 1024)),
    ((-1.3, 0.1), (2.7, 0.35), (7, 5)),
    ((1e6, -3.0), (1e6 + 1.0, 3.0), (1000, 3)),
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("grid", GRIDS)
def test_bin_index_equals_exact_real_bin_away_from_edges(dtype, grid):
    lo, hi, res = grid
    rng = np.random.default_rng(1)
    n = 3000
    span = [hi[a] - lo[a] for a in range(2)]
    x = (lo[0] - 0.05 * span[0] + 1.1 * span[0] * rng.random(n)).astype(dtype)
    y = (lo[1] - 0.05 * span[1] + 1.1 * span[1] * rng.random(n)).astype(dtype)
    lo_t, hi_t, s_t = oracle.setup_axes(x[:1], y[:1], lo, hi, res)
    checked = 0
    for k in range(n):
        got = oracle.particle_bin(dtype(x[k]), dtype(y[k]), lo_t, hi_t, s_t, res, dtype=dtype)
        ex = exact_bin(float(x[k]), lo_t[0], hi_t[0], res[0])
        ey = exact_bin(float(y[k]), lo_t[1], hi_t[1], res[1])
        if ex is None or ey is None:
            assert got is None
            continue
        # t = RN(RN(x - lo) * s) with s = RN(res / RN(hi - lo)): four roundings,
        # each a relative error of at most u, so |t - t_exact| <= ~4 u res.
        # Farther than that from an integer the bin is the exact real one.
        u = Fraction(2.0 ** -24 if dtype == np.float32 else 2.0 ** -53)
        if ex[1] > 5 * u * res[0] and ey[1] > 5 * u * res[1]:
            assert got == (ex[0], ey[0]), (x[k], y[k])
            checked += 1
    assert checked > n // 4


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_bin_index_monotone_and_surjective(dtype):
    lo, hi, res = (-1.3, 0.0), (2.7, 1.0), (37, 1)
    rng = np.random.default_rng(2)
    x = np.sort(rng.uniform(lo[0], hi[0], 20000).astype(dtype))
    lo_t, hi_t, s_t = oracle.setup_axes(x[:1], x[:1], lo, hi, res)
    prev = -1
    seen = set()
    for v in x:
        got = oracle.particle_bin(dtype(v), dtype(0.5), lo_t, hi_t, s_t, res, dtype=dtype)
        if got is None:
            continue
        assert got[0] >= prev
        prev = got[0]
        seen.add(got[0])
    assert seen == set(range(res[0]))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_bin_index_special_points(dtype):
    lo, hi, res = (-10.0, 0.0), (10.0, 1.0), (1024, 64)
    lo_t, hi_t, s_t = oracle.setup_axes(np.zeros(1, dtype), np.zeros(1, dtype), lo, hi, res)
    pb = lambda x, y: oracle.particle_bin(dtype(x), dtype(y), lo_t, hi_t, s_t, res, dtype=dtype)
    assert pb(-10.0, 0.0) == (0, 0)                       # x == lo -> first bin
    below_hi = np.nextafter(dtype(10.0), dtype(-np.inf))
    assert pb(below_hi, 0.5) == (1023, 32)                # just below hi -> last bin
    assert pb(10.0, 0.5) is None                          # hi excluded (half-open)
    assert pb(np.nextafter(dtype(-10.0), dtype(-np.inf)), 0.5) is None
    assert pb(float("nan"), 0.5) is None
    assert pb(0.5, float("nan")) is None
    assert pb(float("inf"), 0.5) is None
    assert pb(float("-inf"), 0.5) is None
    # -0.0 compares equal to lo = 0 on the y axis, so it is inside bin 0
    assert pb(0.0, -0.0) == (512, 0)
    # bin centres land in their own bin
    w = 20.0 / 1024
    for i in (0, 1, 100, 511, 512, 1000, 1023):
        assert pb(-10.0 + (i + 0.5) * w, (i % 64 + 0.5) / 64) == (i, i % 64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_bin_index_near_edges_follows_round_to_nearest_sequence(dtype):
    """At a bin edge only the rounding sequence decides. There, compare with
    numpy scalar arithmetic in T (IEEE round-to-nearest, never fused)."""
    lo, hi, res = (-1.3, 0.0), (2.7, 1.0), (37, 1)
    T = dtype
    lo_t, hi_t, s_t = oracle.setup_axes(np.zeros(1, T), np.zeros(1, T), lo, hi, res)
    assert T(s_t[0]) == T(T(res[0]) / (T(hi_t[0]) - T(lo_t[0])))
    for i in range(1, res[0]):
        e = T(lo_t[0]) + T(i) / T(s_t[0])
        v = e
        for _ in range(3):
            v = np.nextafter(v, T(-np.inf))
        for _ in range(7):
            t = (T(v) - T(lo_t[0])) * T(s_t[0])
            want = min(int(t), res[0] - 1)
            got = oracle.particle_bin(T(v), T(0.5), lo_t, hi_t, s_t, res, dtype=T)
            assert got[0] == want
            v = np.nextafter(v, T(np.inf))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_counts_match_numpy_histogram2d_on_dyadic_grid(dtype):
    w = workloads.uniform(200_000, seed=3, dtype=dtype, res=64)
    r = oracle.bin_workload(w)
    H, _, _ = np.histogram2d(w.x.astype(np.float64), w.y.astype(np.float64), bins=64,
                             range=[[0.0, 1.0], [0.0, 1.0]])
    np.testing.assert_array_equal(r["count"].reshape(64, 64), H.T.astype(np.uint64))


def test_scatter_reductions_match_numpy_ufunc_at_on_dyadic_grid():
    w = workloads.uniform(100_000, seed=4, dtype=np.float64, res=128)
    r = oracle.bin_workload(w)
    b = (np.floor(w.y * 128).astype(np.int64) * 128 + np.floor(w.x * 128).astype(np.int64))
    for a, col in enumerate(w.attrs):
        mn = np.full(128 * 128, np.inf)
        mx = np.full(128 * 128, -np.inf)
        s = np.zeros(128 * 128)
        np.minimum.at(mn, b, col)
        np.maximum.at(mx, b, col)
        np.add.at(s, b, col)
        np.testing.assert_array_equal(r["min"][a], mn)
        np.testing.assert_array_equal(r["max"][a], mx)
        np.testing.assert_allclose(r["sum"][a], s, rtol=1e-13, atol=0)


# ---------------------------------------------------------------- reductions
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_reductions_equal_brute_force(dtype):
    rng = np.random.default_rng(5)
    n = 4000
    lo, hi, res = (-1.3, 0.1), (2.7, 0.35), (7, 5)
    x = rng.uniform(-1.5, 2.9, n).astype(dtype)
    y = rng.uniform(0.05, 0.4, n).astype(dtype)
    attrs = [rng.normal(0, 1, n).astype(dtype), rng.uniform(-1e3, 1e5, n).astype(dtype)]
    r = oracle.bin_particles(x, y, attrs, lo, hi, res)
    lo_t, hi_t, _ = oracle.setup_axes(x, y, lo, hi, res)
    groups = group_by_exact_bins(x, y, lo_t, hi_t, res)
    assert groups is not None
    B = res[0] * res[1]
    for b in range(B):
        idx = groups.get(b, [])
        assert r["count"][b] == len(idx)
        for a, col in enumerate(attrs):
            vals = [float(col[k]) for k in idx]
            if not vals:
                assert r["sum"][a][b] == 0.0 and not math.copysign(1, r["sum"][a][b]) < 0
                assert r["min"][a][b] == np.inf and r["max"][a][b] == -np.inf
                assert bits64(r["avg"][a][b]) == 0x7FF8000000000000
                continue
            exact = math.fsum(vals)
            sabs = math.fsum(abs(v) for v in vals)
            assert abs(r["sum"][a][b] - exact) <= 2 * F64_EPS * abs(exact) + 4 * len(vals) ** 2 * F64_EPS ** 2 * sabs
            assert r["min"][a][b] == dtype(min(vals))
            assert r["max"][a][b] == dtype(max(vals))
            assert abs(r["avg"][a][b] - exact / len(vals)) <= 4 * F64_EPS * sabs / len(vals)


def test_sum_is_compensated():
    # plain left-to-right FP64 summation returns 0 here; the exact sum is 2
    x = np.full(4, 0.5)
    y = np.full(4, 0.5)
    a = np.array([1e16, 1.0, -1e16, 1.0])
    r = oracle.bin_particles(x, y, [a], (0, 0), (1, 1), (1, 1))
    assert r["sum"][0][0] == 2.0
    assert r["avg"][0][0] == 0.5


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_integer_valued_sums_are_exact(dtype):
    rng = np.random.default_rng(6)
    n = 50_000
    x = rng.random(n).astype(dtype)
    y = rng.random(n).astype(dtype)
    ints = rng.integers(-1000, 1000, n)
    r = oracle.bin_particles(x, y, [ints.astype(dtype)], (0, 0), (1, 1), (16, 16))
    b = np.floor(y.astype(np.float64) * 16).astype(np.int64) * 16 + np.floor(x.astype(np.float64) * 16).astype(np.int64)
    want = [0] * 256
    for k in range(n):
        want[b[k]] += int(ints[k])
    assert r["sum"][0].tolist() == [float(v) for v in want]


def test_one_particle_at_each_bin_centre():
    res = (13, 9)
    lo, hi = (-2.0, 3.0), (5.0, 4.0)
    ix, iy = np.meshgrid(np.arange(res[0]), np.arange(res[1]))
    ix, iy = ix.ravel(), iy.ravel()
    x = lo[0] + (ix + 0.5) * (hi[0] - lo[0]) / res[0]
    y = lo[1] + (iy + 0.5) * (hi[1] - lo[1]) / res[1]
    mass = (iy * res[0] + ix).astype(np.float64) * 1.5
    r = oracle.bin_particles(x, y, [mass], lo, hi, res)
    assert (r["count"] == 1).all()
    np.testing.assert_array_equal(r["sum"][0], np.arange(res[0] * res[1]) * 1.5)
    np.testing.assert_array_equal(r["min"][0], r["sum"][0])
    np.testing.assert_array_equal(r["max"][0], r["sum"][0])
    np.testing.assert_array_equal(r["avg"][0], r["sum"][0])


def test_all_particles_in_one_bin():
    n = 10_001
    rng = np.random.default_rng(7)
    x = np.full(n, 0.3)
    y = np.full(n, 0.7)
    a = rng.uniform(1, 2, n)
    r = oracle.bin_particles(x, y, [a], (0, 0), (1, 1), (10, 10))
    b = 7 * 10 + 3
    assert r["count"][b] == n and r["count"].sum() == n
    assert r["sum"][0][b] == math.fsum(a)
    assert r["min"][0][b] == a.min() and r["max"][0][b] == a.max()


def test_nan_attribute_skipped_by_min_max_and_propagates_to_sum():
    x = np.array([0.1, 0.2, 0.3])
    y = np.array([0.1, 0.1, 0.1])
    a = np.array([2.0, np.nan, -1.0])
    r = oracle.bin_particles(x, y, [a], (0, 0), (1, 1), (1, 1))
    assert r["count"][0] == 3
    assert math.isnan(r["sum"][0][0]) and math.isnan(r["avg"][0][0])
    assert r["min"][0][0] == -1.0 and r["max"][0][0] == 2.0


def test_sums_exact_at_the_bottom_of_the_range():
    """Sums of subnormal values, and of normal values whose partial sums cross
    zero and the subnormal range, are exact in FP64 (every partial sum is a
    small multiple of 2^-1074): the oracle must return the exact rational
    sum. Signed zeros add to +0.0; an infinity dominates; +inf and -inf give
    NaN (IEEE 754 addition)."""
    rng = np.random.default_rng(43)
    tiny = 2.0 ** -1074
    cases = {
        "subnormal": rng.integers(-50, 51, 700) * tiny,
        "cancel": rng.permutation(np.array([3.0] * 279 + [-2.0] * 420 + [4.0])) * 2.0 ** -1023,
        "zeros": np.where(rng.random(300) < 0.5, -0.0, 0.0),
        "neg_zeros": np.full(300, -0.0),
        "inf": np.concatenate([rng.normal(0, 1, 50), [np.inf]]),
        "inf_minus_inf": np.concatenate([rng.normal(0, 1, 50), [np.inf, -np.inf]]),
    }
    for name, a in cases.items():
        x = np.full(a.size, 0.5)
        y = np.full(a.size, 0.5)
        r = oracle.bin_particles(x, y, [a], (0, 0), (1, 1), (1, 1))
        got = r["sum"][0][0]
        if name == "inf":
            assert got == np.inf, name
        elif name == "inf_minus_inf":
            assert math.isnan(got), name
        else:
            exact = sum((Fraction(float(v)) for v in a), Fraction(0))
            assert Fraction(float(got)) == exact, name
            if exact == 0:
                assert math.copysign(1.0, got) == 1.0, f"{name}: a zero sum is +0.0"
    # the cancellation case ends on 2^-1023, itself subnormal
    r = oracle.bin_particles(np.full(700, 0.5), np.full(700, 0.5), [cases["cancel"]], (0, 0), (1, 1), (1, 1))
    assert r["sum"][0][0] == 2.0 ** -1023


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_min_max_in_total_order_for_signed_zero(dtype):
    x = np.array([0.1, 0.2], dtype)
    y = np.array([0.1, 0.1], dtype)
    for a in ([0.0, -0.0], [-0.0, 0.0]):
        r = oracle.bin_particles(x, y, [np.array(a, dtype)], (0, 0), (1, 1), (1, 1))
        assert np.signbit(r["min"][0][0]) and r["min"][0][0] == 0
        assert not np.signbit(r["max"][0][0])


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_invariants_on_plummer(dtype):
    w = workloads.plummer(200_000, seed=8, dtype=dtype, res=256)
    r = oracle.bin_workload(w)
    inb = ((w.x >= dtype(-10)) & (w.x < dtype(10)) & (w.y >= dtype(-10)) & (w.y < dtype(10)))
    assert int(r["count"].sum()) == int(inb.sum())
    for a, col in enumerate(w.attrs):
        tot = math.fsum(col[inb].astype(np.float64))
        sabs = math.fsum(np.abs(col[inb].astype(np.float64)))
        assert abs(math.fsum(r["sum"][a]) - tot) <= 1e-13 * sabs
        ne = r["count"] > 0
        assert (r["min"][a][ne] <= r["avg"][a][ne]).all()
        assert (r["avg"][a][ne] <= r["max"][a][ne]).all()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_permutation_invariance(dtype):
    w = workloads.plummer(100_000, seed=9, dtype=dtype, res=128)
    r1 = oracle.bin_workload(w)
    p = np.random.default_rng(10).permutation(w.n)
    r2 = oracle.bin_particles(w.x[p], w.y[p], [a[p] for a in w.attrs], w.lo, w.hi, w.res)
    for k in ("count", "min", "max"):
        np.testing.assert_array_equal(r1[k], r2[k])
    np.testing.assert_allclose(r1["sum"], r2["sum"], rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_shard_and_merge_equals_whole(dtype):
    w = workloads.plummer(60_000, seed=11, dtype=dtype, res=64)
    whole = oracle.bin_workload(w)
    axes = oracle.setup_axes(w.x, w.y, w.lo, w.hi, w.res)
    cuts = [0, 7, 20_000, 20_001, 45_000, w.n]
    states = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        st = oracle.State(w.res, len(w.attrs), dtype)
        st.accumulate(w.x[a:b], w.y[a:b], [c[a:b] for c in w.attrs], axes)
        states.append(st)
    acc = states[0]
    for st in states[1:]:
        acc.merge(st)
    merged = acc.finalize()
    for k in ("count", "min", "max"):
        np.testing.assert_array_equal(whole[k], merged[k])
    np.testing.assert_allclose(whole["sum"], merged["sum"], rtol=1e-14, atol=1e-12)


# ---------------------------------------------------------------- bounds
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_auto_bounds_are_finite_min_max_and_closed(dtype):
    rng = np.random.default_rng(12)
    x = rng.normal(0, 3, 5000).astype(dtype)
    y = rng.normal(1, 2, 5000).astype(dtype)
    x[10] = np.nan
    x[11] = np.inf
    y[12] = -np.inf
    a = rng.random(5000).astype(dtype)
    r = oracle.bin_particles(x, y, [a], res=(50, 40), auto_bounds=True)
    fin = np.isfinite(x) & np.isfinite(y)
    fx, fy = x[np.isfinite(x)], y[np.isfinite(y)]
    assert r["bounds"].tolist() == [float(fx.min()), float(fx.max()), float(fy.min()), float(fy.max())]
    assert int(r["count"].sum()) == int(fin.sum())
    # the particle at the maximum x is in the last column of bins
    k = int(np.argmax(np.where(fin, x, -np.inf)))
    lo_t, hi_t, s_t = oracle.setup_axes(x, y, res=(50, 40), auto_bounds=True)
    assert oracle.particle_bin(x[k], y[k], lo_t, hi_t, s_t, (50, 40), closed=True, dtype=dtype)[0] == 49


def test_auto_bounds_degenerate_and_invalid_grids():
    x = np.full(10, 3.0)
    y = np.linspace(0, 1, 10)
    with pytest.raises(oracle.OracleError) as e:
        oracle.bin_particles(x, y, [], res=(4, 4), auto_bounds=True)
    assert e.value.code == oracle.ERR_DEGENERATE
    with pytest.raises(oracle.OracleError) as e:
        oracle.bin_particles(np.array([np.nan]), np.array([0.5]), [], res=(4, 4), auto_bounds=True)
    assert e.value.code == oracle.ERR_DEGENERATE
    for lo, hi, res in [((0, 0), (1, 1), (0, 4)), ((1, 0), (1, 1), (4, 4)), ((2, 0), (1, 1), (4, 4)),
                        ((0, 0), (np.inf, 1), (4, 4)), ((0, 0), (1, 1), (70000, 1))]:
        with pytest.raises(oracle.OracleError) as e:
            oracle.bin_particles(y, y, [], lo, hi, res)
        assert e.value.code == oracle.ERR_INVALID_ARG
    # f32: bounds that collapse when rounded to float are rejected too
    with pytest.raises(oracle.OracleError):
        oracle.bin_particles(y.astype(np.float32), y.astype(np.float32), [], (1.0, 0.0),
                             (1.0 + 1e-12, 1.0), (4, 4))


def test_empty_input():
    r = oracle.bin_particles(np.zeros(0), np.zeros(0), [np.zeros(0)], (0, 0), (1, 1), (3, 2))
    assert (r["count"] == 0).all()
    assert all(bits64(v) == 0x7FF8000000000000 for v in r["avg"][0])


def test_f32_sums_widen_exactly():
    rng = np.random.default_rng(13)
    n = 3000
    x = np.full(n, 0.5, np.float32)
    y = np.full(n, 0.5, np.float32)
    a = rng.uniform(0, 1e4, n).astype(np.float32)
    r = oracle.bin_particles(x, y, [a], (0, 0), (1, 1), (1, 1))
    exact = math.fsum(float(v) for v in a)
    assert abs(r["sum"][0][0] - exact) <= 2 * F64_EPS * exact
    assert r["min"].dtype == np.float32 and r["min"][0][0] == a.min()


def test_shard_merge_keeps_both_compensation_terms():
    # each shard's plain sum loses its +1.0; the merged sum must still be exact (2.0)
    x = np.full(2, 0.5)
    y = np.full(2, 0.5)
    axes = oracle.setup_axes(x, y, (0, 0), (1, 1), (1, 1))
    a = oracle.State((1, 1), 1, np.float64).accumulate(x, y, [np.array([1e16, 1.0])], axes)
    b = oracle.State((1, 1), 1, np.float64).accumulate(x, y, [np.array([-1e16, 1.0])], axes)
    r = a.merge(b).finalize()
    assert r["sum"][0][0] == math.fsum([1e16, 1.0, -1e16, 1.0]) == 2.0
    assert r["count"][0] == 4



@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("threads", [1, 3, 16])
def test_threaded_baseline_equals_oracle(dtype, threads):
    """The all-core CPU baseline (per-thread meshes, then a merge) gives the
    single-threaded oracle's counts, min and max exactly and its sums to
    within the reordering of Neumaier partial sums; automatic bounds and
    NaN attributes included."""
    w = workloads.plummer(200_003, seed=5, dtype=dtype, res=96)
    w.attrs[1][::37] = np.nan
    for auto in (False, True):
        ref = oracle.bin_workload(w, auto)
        got = oracle.bin_particles_threaded(w.x, w.y, w.attrs, w.lo, w.hi, w.res, auto, threads=threads)
        np.testing.assert_array_equal(got["count"], ref["count"])
        for k in ("min", "max"):
            np.testing.assert_array_equal(got[k].view(np.int64 if dtype == np.float64 else np.int32),
                                          ref[k].view(np.int64 if dtype == np.float64 else np.int32))
        sabs = oracle.bin_particles(w.x, w.y, [np.abs(a) for a in w.attrs], w.lo, w.hi, w.res, auto)["sum"]
        both_nan = np.isnan(got["sum"]) & np.isnan(ref["sum"])
        assert (both_nan | (np.abs(got["sum"] - ref["sum"]) <= 1e-15 * sabs)).all()
        assert (np.isnan(got["avg"]) == np.isnan(ref["avg"])).all()


def test_threaded_baseline_more_threads_than_particles_and_empty():
    x = np.array([0.1, 0.9, 0.5]); y = np.array([0.2, 0.8, 0.5]); a = np.array([1.0, 2.0, 3.0])
    got = oracle.bin_particles_threaded(x, y, [a], res=(2, 2), threads=64)
    ref = oracle.bin_particles(x, y, [a], res=(2, 2))
    np.testing.assert_array_equal(got["count"], ref["count"])
    np.testing.assert_array_equal(got["sum"], ref["sum"])
    e = np.zeros(0)
    got = oracle.bin_particles_threaded(e, e, [e], res=(2, 2), threads=4)
    assert got["count"].sum() == 0 and (got["sum"] == 0).all()
