"""Exact integer-limb sums of f32 data in shared-memory meshes.

The private, sort and batched-private paths add f32 values into three
32-bit integer limbs of 16-bit digits (native 32-bit shared-memory atomics
only). Each mesh sets a 24-binade window from a sample of its own values;
values outside it (far below or above the sample's largest, subnormal,
inf, NaN) go to the FP64 sums directly, and a mesh takes at most 65,536
values per bin between its clear and its merge. Inside the window the sum
is exact until one rounding to FP64, so these sums meet the FP64 tolerance
in both modes that use limbs (BN_SUM_F32C, BN_SUM_F64); counts, min and
max stay bit-exact (Sec. 4.2's per-bin reductions).
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import TOL_F64, abs_sums, assert_parity, run_gpu, to_numpy_result

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


def _flags(bn, strategy, mode):
    s = {"private": bn.STRATEGY_PRIVATE, "sort": bn.STRATEGY_SORT}[strategy]
    return s | {"f32c": bn.SUM_F32C, "f64": bn.SUM_F64}[mode]


def _check(w, gpu, label):
    ref = oracle.bin_workload(w)
    assert_parity(gpu, ref, abs_sums(w), TOL_F64, label=label)
    return ref


def wide_range_workload(n, seed):
    """Attribute 0 spans 60 decades with both signs, zeros, subnormals, inf
    and NaN; attribute 1 starts with 5,000 values near 1e-3 (the sample a
    mesh takes) and continues near 1e5..1e6, far above the sampled window."""
    rng = np.random.default_rng(seed)
    x = rng.random(n).astype(np.float32)
    y = rng.random(n).astype(np.float32)
    a0 = (np.sign(rng.random(n) - 0.5) * 10.0 ** rng.uniform(-30, 30, n)).astype(np.float32)
    a0[::97] = 0.0
    a0[1::101] = -0.0
    a0[2::103] = np.float32(1e-41)      # subnormal
    a0[3::5003] = np.inf
    a0[4::7001] = np.nan
    a1 = rng.uniform(1e5, 1e6, n).astype(np.float32)
    a1[:5000] = rng.uniform(0.0, 1e-3, 5000).astype(np.float32)
    return workloads.Workload("wide range", x, y, [a0, a1], (0.0, 0.0), (1.0, 1.0), (48, 48))


@pytest.mark.parametrize("n", [60_000, 300_001])
@pytest.mark.parametrize("mode", ["f32c", "f64"])
@pytest.mark.parametrize("strategy", ["private", "sort"])
def test_limb_window_and_fallback(bn, ctx, strategy, mode, n):
    """60,000 records make one sort item per bucket (its bins are stored, the
    fallback sums added to them); 300,001 split the bucket into items merged
    with atomics."""
    w = wide_range_workload(n, seed=71)
    _check(w, run_gpu(ctx, w, flags=_flags(bn, strategy, mode)), f"{strategy} {mode} n={n}")


@pytest.mark.parametrize("mode", ["f32c", "f64"])
@pytest.mark.parametrize("strategy", ["private", "sort"])
def test_limb_hot_bin_past_digit_headroom(bn, ctx, strategy, mode):
    """400,000 particles, 390,000 of them in one bin: more than one mesh's
    65,536 adds per bin, so the work must be split across meshes (private:
    enough CTAs; sort: items of at most 65,536 records)."""
    rng = np.random.default_rng(72)
    n = 400_000
    x = rng.random(n).astype(np.float32)
    y = rng.random(n).astype(np.float32)
    x[:390_000] = 0.51
    y[:390_000] = 0.52
    a0 = rng.uniform(0.0, 1e4, n).astype(np.float32)
    a1 = rng.normal(0.0, 1.0, n).astype(np.float32)
    w = workloads.Workload("hot bin", x, y, [a0, a1], (0.0, 0.0), (1.0, 1.0), (16, 16))
    ref = _check(w, run_gpu(ctx, w, flags=_flags(bn, strategy, mode)), f"{strategy} {mode}")
    assert ref["count"].max() >= 390_000


@pytest.mark.parametrize("mode", ["f32c", "f64"])
def test_limb_batch_private_items(bn, ctx, mode):
    """Batched private items (tiles of at most 65,536 particles) with a hot
    bin and a wide value range, against the oracle per block."""
    rng = np.random.default_rng(73)
    flags = bn.STRATEGY_PRIVATE | {"f32c": bn.SUM_F32C, "f64": bn.SUM_F64}[mode]
    ws = [wide_range_workload(150_001, seed=74)]
    n = 250_000
    x = rng.random(n).astype(np.float32)
    y = rng.random(n).astype(np.float32)
    x[: n - 1000] = 0.25
    y[: n - 1000] = 0.75
    ws.append(workloads.Workload("hot", x, y, [rng.uniform(0, 1e4, n).astype(np.float32),
                                               rng.normal(0, 1, n).astype(np.float32)],
                                 (0.0, 0.0), (1.0, 1.0), (20, 20)))
    blocks, outs, keep = [], [], []
    for w in ws:
        cols = [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in (w.x, w.y, *w.attrs)]
        o = bn.alloc_outputs(2, w.res[0] * w.res[1], torch.float32, torch.device("cuda"))
        r = bn.result_struct(o)
        keep += [cols, r]
        outs.append((w, o))
        blocks.append(bn.block(cols[0], cols[1], cols[2:], bn.grid(w.lo, w.hi, w.res), r))
    bn.bn_bin_batch(ctx.handle, blocks, bn.OP_ALL | flags)
    torch.cuda.synchronize()
    for w, o in outs:
        _check(w, to_numpy_result(o), f"batch {w.name} {mode}")
