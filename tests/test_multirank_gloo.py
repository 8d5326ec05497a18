"""Cross-rank combination of partial meshes on the CPU (gloo), and Eq. 1.

Sec. 4.2 bins with MPI: every rank bins its own particles and the partial
meshes combine. The library packs a rank's result into an exchange buffer
of four sections (count, sum, min keys, max keys; include/binning.h) that
combine with SUM, SUM, MIN and MAX; the collective is the library binding's
own host code (allreduce_exchange). These tests run it on two gloo ranks
with no GPU: each rank's partial mesh comes from the oracle, is encoded in
the documented exchange format by the test, combined by
allreduce_exchange, decoded, and must equal binning all particles at once,
including a bin where one rank's minimum is -0.0 and the other's +0.0 (a
float MIN would not order them). The packing kernels themselves are checked
against the same encoding on the GPU (test_gpu_multirank.py).

Eq. 1 (Sec. 3) is checked against a table worked out by hand.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
from _exchange import decode_keys, encode_keys, shard_workload  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, dtype, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    import paper_2310_02926_gb300 as bn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = shard_workload(dtype)
    cuts = np.linspace(0, w.n, world + 1).astype(int)
    a, b = cuts[rank], cuts[rank + 1]
    part = oracle.bin_particles(w.x[a:b], w.y[a:b], [c[a:b] for c in w.attrs], w.lo, w.hi, w.res)
    B, A = w.res[0] * w.res[1], len(w.attrs)
    ex = torch.zeros(8 * B * (1 + 3 * A), dtype=torch.uint8)
    cnt, s, mnk, mxk = bn.exchange_sections(ex, B, A)
    cnt.copy_(torch.from_numpy(part["count"].astype(np.int64)))
    s.copy_(torch.from_numpy(part["sum"].reshape(-1)))
    mnk.copy_(torch.from_numpy(encode_keys(part["min"]).reshape(-1)))
    mxk.copy_(torch.from_numpy(encode_keys(part["max"]).reshape(-1)))
    bn.allreduce_exchange(ex, B, A)
    if rank == 0:
        whole = oracle.bin_workload(w)
        cnt, s, mnk, mxk = bn.exchange_sections(ex, B, A)
        ok = bool(np.array_equal(cnt.numpy().astype(np.uint64), whole["count"]))
        mn = decode_keys(mnk.numpy(), dtype).reshape(A, B)
        mx = decode_keys(mxk.numpy(), dtype).reshape(A, B)
        bits = np.int64 if dtype == np.float64 else np.int32
        ok &= bool(np.array_equal(mn.view(bits), whole["min"].view(bits)))
        ok &= bool(np.array_equal(mx.view(bits), whole["max"].view(bits)))
        mixed = np.signbit(mn[2]) & ~np.signbit(mx[2]) & (whole["count"] > 0)
        ok &= bool(mixed.sum() > 100)
        sabs = oracle.bin_particles(w.x, w.y, [np.abs(c) for c in w.attrs], w.lo, w.hi, w.res)["sum"]
        ok &= bool((np.abs(s.numpy().reshape(A, B) - whole["sum"]) <= 1e-12 * sabs).all())
        q.put(ok)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_two_gloo_ranks_combine_exchange_buffers(dtype):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, dtype, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True


def test_exchange_keys_order_like_total_order():
    """Integer order of the keys is IEEE totalOrder (-0 < +0) for both types."""
    for dt in (np.float64, np.float32):
        v = np.array([-np.inf, -3.0, -1e-30, -0.0, 0.0, 1e-30, 2.0, np.inf], dtype=dt)
        k = encode_keys(v)
        assert (np.diff(k) > 0).all()
        back = decode_keys(k, dt)
        assert np.array_equal(back.view(np.int64 if dt == np.float64 else np.int32),
                              v.view(np.int64 if dt == np.float64 else np.int32))


# Eq. 1: d = ((r mod n_u) * s + d_0) mod n_a, worked by hand.
# (n_avail, n_use, stride, offset) -> devices of ranks 0..7
EQ1_TABLE = [
    ((4, 0, 0, 0), [0, 1, 2, 3, 0, 1, 2, 3]),    # the paper's defaults
    ((4, 2, 2, 0), [0, 2, 0, 2, 0, 2, 0, 2]),    # two devices per node, every other one
    ((4, 2, 1, 2), [2, 3, 2, 3, 2, 3, 2, 3]),    # the upper two devices
    ((4, 3, 2, 1), [1, 3, 1, 1, 3, 1, 1, 3]),    # (r mod 3) * 2 + 1 mod 4
    ((4, 4, 1, -1), [3, 0, 1, 2, 3, 0, 1, 2]),   # a negative offset wraps
    ((1, 0, 0, 0), [0, 0, 0, 0, 0, 0, 0, 0]),    # one device
]


@pytest.mark.parametrize("args,want", EQ1_TABLE)
def test_select_device_follows_eq1(args, want):
    import paper_2310_02926_gb300 as bn
    if not os.path.exists(bn.LIB_PATH):
        pytest.skip("libbinning.so not built")
    n_avail, n_use, stride, offset = args
    got = [bn.bn_select_device(r, n_avail, n_use, stride, offset) for r in range(8)]
    assert got == want


def test_select_device_rejects_bad_arguments():
    import paper_2310_02926_gb300 as bn
    if not os.path.exists(bn.LIB_PATH):
        pytest.skip("libbinning.so not built")
    for rank, n_avail in ((-1, 4), (0, 0)):
        with pytest.raises(bn.BinningError) as e:
            bn.bn_select_device(rank, n_avail)
        assert e.value.code == bn.ERR_INVALID_ARG
