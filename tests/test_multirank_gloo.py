"""Cross-rank merge of partial meshes with torch.distributed (gloo, CPU).

Sec. 4.2 bins with MPI: every rank bins its own particles and the partial
meshes combine (count and sum add, min and max reduce). This runs two gloo
ranks on the CPU: each bins its shard with the oracle, the ranks all-reduce
(SUM for count/sum, MIN/MAX for min/max), and the finalised result must equal
binning all particles at once. No GPU is used.
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


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import oracle
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workloads.plummer(90_001, seed=5, dtype=np.float64, res=48)
    cuts = np.linspace(0, w.n, world + 1).astype(int)
    a, b = cuts[rank], cuts[rank + 1]
    part = oracle.bin_particles(w.x[a:b], w.y[a:b], [c[a:b] for c in w.attrs], w.lo, w.hi, w.res)
    cnt = torch.from_numpy(part["count"].astype(np.int64))
    s = torch.from_numpy(part["sum"].copy())
    mn = torch.from_numpy(part["min"].copy())
    mx = torch.from_numpy(part["max"].copy())
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(mn, op=dist.ReduceOp.MIN)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    if rank == 0:
        whole = oracle.bin_workload(w)
        ok = bool(np.array_equal(cnt.numpy().astype(np.uint64), whole["count"]))
        ok &= bool(np.array_equal(mn.numpy(), whole["min"]) and np.array_equal(mx.numpy(), whole["max"]))
        sabs = oracle.bin_particles(w.x, w.y, [np.abs(c) for c in w.attrs], w.lo, w.hi, w.res)["sum"]
        ok &= bool((np.abs(s.numpy() - whole["sum"]) <= 1e-12 * sabs).all())
        q.put(ok)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_partial_meshes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
