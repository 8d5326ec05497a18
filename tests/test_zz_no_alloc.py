"""bn_bin_particles_static: binning for callers that cannot allocate.

Checks the no-allocation entry point through the C ABI against the CPU
oracle (counts, min and max bit for bit, sums within the stated tolerance)
and against the regular bn_bin_particles on the same inputs (within the same
tolerance), on two calls in a row: the shared fixed scratch keeps the
previous call's contents, so the second call shows that each call starts
clean. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from _parity import TOL_F32C, TOL_F64, assert_parity, to_numpy_result

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bn():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as m
    assert torch.cuda.is_available()
    return m


def static_call(bn, cols, g, ops, out, sync=1):
    n_attrs = len(cols) - 2
    arr = (bn.bn_buffer * max(n_attrs, 1))(*[bn.buffer(c) for c in cols[2:]])
    r = bn.result_struct(out)
    stream = torch.cuda.current_stream().cuda_stream
    return bn.lib().bn_bin_particles_static(ctypes.byref(bn.buffer(cols[0])),
                                            ctypes.byref(bn.buffer(cols[1])), arr, n_attrs,
                                            ctypes.byref(g), ops, ctypes.byref(r), stream, sync)


def close(a, b, tol, sabs):
    for k in ("count", "min", "max"):
        np.testing.assert_array_equal(a[k], b[k])
    assert (np.abs(a["sum"] - b["sum"]) <= tol * sabs).all()
    ne = a["count"] > 0
    assert (np.abs(a["avg"][:, ne] - b["avg"][:, ne]) <= tol * sabs[:, ne] / a["count"][ne]).all()
    assert (a["avg"][:, ~ne].view(np.int64) == b["avg"][:, ~ne].view(np.int64)).all()


@pytest.mark.parametrize("case", ["plummer_f64_1024", "gaussians_f32_256", "uniform_f64_64_auto"])
def test_static_matches_regular_entry_point_twice(bn, case):
    if case == "plummer_f64_1024":
        w, tol, auto = workloads.plummer(400_003, seed=21, dtype=np.float64, res=1024), TOL_F64, False
    elif case == "gaussians_f32_256":
        w, tol, auto = workloads.gaussians(300_001, seed=22, res=256), TOL_F32C, False
    else:
        w, tol, auto = workloads.uniform(200_001, seed=23, dtype=np.float64, res=64), TOL_F64, True
    dev = torch.device("cuda", 0)
    cols = [torch.from_numpy(c).to(dev) for c in (w.x, w.y, *w.attrs)]
    B = w.res[0] * w.res[1]
    A = len(w.attrs)
    g = bn.grid(w.lo, w.hi, w.res, auto)
    with bn.Context(0) as ctx:
        ref = to_numpy_result(ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res,
                                                auto_bounds=auto))
        torch.cuda.synchronize()
    sabs = oracle.bin_particles(w.x, w.y, [np.abs(a) for a in w.attrs], w.lo, w.hi, w.res, auto)["sum"]
    want = oracle.bin_workload(w, auto)
    for call in range(2):
        out = bn.alloc_outputs(A, B, cols[0].dtype, dev)
        for t in [out["count"], *out["sum"], *out["avg"]]:
            t.fill_(7)  # stale contents must not leak into the result
        st = static_call(bn, cols, g, bn.OP_ALL, out)
        assert st == bn.OK, bn.lib().bn_last_error()
        got = to_numpy_result(out)
        assert_parity(got, want, sabs, tol, label=f"{case} call {call}")
        close(got, ref, tol, sabs)


def test_static_rejects_oversized_f64_mesh_and_reports_degenerate_bounds(bn):
    dev = torch.device("cuda", 0)
    x = torch.rand(1000, dtype=torch.float64, device=dev)
    out = bn.alloc_outputs(0, 5000 * 4000, torch.float64, dev, ops=bn.OP_COUNT)
    st = static_call(bn, [x, x], bn.grid(res=(5000, 4000)), bn.OP_COUNT, out)
    assert st == bn.ERR_INVALID_ARG
    assert b"edge keys" in bn.lib().bn_last_error()
    same = torch.full((1000,), 2.0, dtype=torch.float64, device=dev)
    out = bn.alloc_outputs(0, 16, torch.float64, dev, ops=bn.OP_COUNT)
    st = static_call(bn, [same, x], bn.grid(res=(4, 4), auto_bounds=True), bn.OP_COUNT, out)
    assert st == bn.ERR_DEGENERATE
    # the status word is cleared by the next call
    st = static_call(bn, [x, x], bn.grid(res=(4, 4), auto_bounds=True), bn.OP_COUNT, out)
    assert st == bn.OK
    assert int(out["count"].sum()) == 1000
    # asynchronous: no status comes back, the bounds output marks the failure
    out = bn.alloc_outputs(0, 16, torch.float64, dev, ops=bn.OP_COUNT, bounds=True)
    st = static_call(bn, [same, x], bn.grid(res=(4, 4), auto_bounds=True), bn.OP_COUNT, out, sync=0)
    assert st == bn.OK
    torch.cuda.synchronize()
    assert torch.isnan(out["bounds"]).all()
    assert int(out["count"].sum()) == 0
    st = static_call(bn, [x, x], bn.grid(res=(4, 4), auto_bounds=True), bn.OP_COUNT, out, sync=0)
    assert st == bn.OK
    torch.cuda.synchronize()
    assert not torch.isnan(out["bounds"]).any() and int(out["count"].sum()) == 1000
