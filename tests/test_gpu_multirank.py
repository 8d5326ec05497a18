"""Partial meshes across ranks on the GPU: the exchange buffer (Sec. 4.2's
MPI-parallel binning combines per-rank meshes).

- bn_exchange_pack writes exactly the documented exchange format (counts,
  sums, totalOrder keys of min and max as int64) for f32 and f64 results;
- with one NCCL rank the pack / all-reduce / unpack round trip returns the
  partial result unchanged (avg recomputed);
- two gloo ranks, each a process binning its own shard through
  bn_bin_particles on the one GPU, combine their partial meshes with
  reduce_across_ranks; the result equals the oracle on the whole set,
  including bins where one rank's minimum is -0.0 and the other's +0.0.
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import workloads
from _exchange import encode_keys, shard_workload
from _parity import TOL_F32C, TOL_F64, abs_sums, assert_parity, to_numpy_result

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bn():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as m
    assert torch.cuda.is_available()
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_exchange_pack_writes_the_documented_format(bn, dtype):
    w = workloads.plummer(200_001, seed=40, dtype=dtype, res=96)
    w.attrs[1][::7] = -0.0
    with bn.Context(0) as ctx:
        cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
        out = ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res)
        B, A = w.res[0] * w.res[1], len(w.attrs)
        ex = torch.empty(bn.bn_exchange_bytes(B, A), dtype=torch.uint8, device="cuda")
        assert ex.numel() == 8 * B * (1 + 3 * A)
        code = bn.F64 if dtype == np.float64 else bn.F32
        bn.bn_exchange_pack(ctx.handle, bn.result_struct(out), code, A, B, ex)
        torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in bn.exchange_sections(ex, B, A)]
    res = to_numpy_result(out)
    assert np.array_equal(got[0], res["count"].astype(np.int64))
    assert np.array_equal(got[1].view(np.int64), res["sum"].reshape(-1).view(np.int64))
    assert np.array_equal(got[2], encode_keys(res["min"]).reshape(-1))
    assert np.array_equal(got[3], encode_keys(res["max"]).reshape(-1))


def test_single_nccl_rank_round_trip(bn):
    """World size 1 over NCCL: reduce_across_ranks returns the rank's own
    result bit for bit (avg recomputed the same way)."""
    port = _free_port()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        w = workloads.plummer(150_001, seed=41, dtype=np.float64, res=200)
        with bn.Context(0) as ctx:
            cols = [torch.from_numpy(c).cuda() for c in (w.x, w.y, *w.attrs)]
            part = ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res)
            B, A = w.res[0] * w.res[1], len(w.attrs)
            whole = bn.reduce_across_ranks(ctx, part, bn.F64, A, B)
            torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    a, b = to_numpy_result(part), to_numpy_result(whole)
    for k in ("count", "sum", "min", "max", "avg"):
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def _gpu_rank(rank, world, port, dtype, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import paper_2310_02926_gb300 as bn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = shard_workload(dtype, world)
        cuts = np.linspace(0, w.n, world + 1).astype(int)
        a, b = cuts[rank], cuts[rank + 1]
        with bn.Context(0) as ctx:
            cols = [torch.from_numpy(np.ascontiguousarray(c[a:b])).cuda() for c in (w.x, w.y, *w.attrs)]
            part = ctx.bin_particles(cols[0], cols[1], cols[2:], w.lo, w.hi, w.res)
            B, A = w.res[0] * w.res[1], len(w.attrs)
            code = bn.F64 if dtype == np.float64 else bn.F32
            whole = bn.reduce_across_ranks(ctx, part, code, A, B)
            torch.cuda.synchronize()
            res = {k: (v.cpu().numpy() if not isinstance(v, list) else np.stack([t.cpu().numpy() for t in v]))
                   for k, v in whole.items()}
        q.put((rank, res))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_two_gloo_ranks_bin_on_the_gpu_and_combine(bn, dtype):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, dtype, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    w = shard_workload(dtype, 2)
    ref = oracle.bin_workload(w)
    tol = TOL_F64 if dtype == np.float64 else TOL_F32C
    for r in (0, 1):
        res = dict(got[r])
        res["count"] = res["count"].astype(np.uint64)
        assert_parity(res, ref, abs_sums(w), tol, label=f"rank {r}")
    mixed = np.signbit(got[0]["min"][2]) & ~np.signbit(got[0]["max"][2]) & (ref["count"] > 0)
    assert mixed.sum() > 100
