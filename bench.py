#!/usr/bin/env python
"""Benchmark: particle data binning on GB300 (one JSON line on stdout).

Workload (one step = one full binning call): 50,000,000 particles drawn
from a Plummer sphere (scale radius 1, truncated at r = 10) projected on
x-y, three f64 attributes (mass ~ U[1,2], vx, vy ~ N(0,1)), binned onto a
1024 x 1024 mesh over [-10,10]^2 with count/sum/min/max/avg. Inputs
(2.0 GB) are larger than L2 (129 MB), so no flush is needed between steps.

value     particles/s over all ranks, inputs resident in HBM, CUDA events on
          the library's stream, max over ranks
e2e       the same metric through the public API with pinned host buffers:
          every step copies the inputs host->device and the outputs back
roofline  the particle-pass kernel: algorithmic bytes per launch over its
          event-timed average duration, against the measured HBM copy peak
cpu_baseline  the CPU oracle (single thread) on the same workload

--impl reference times the CPU oracle itself (the reference arm).
Multi-GPU (torchrun): every rank bins its own replica of the workload
(replicas only: there is no data-path collective), barrier + max time.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("binned particles/s and % of HBM peak, batched FP32 vs plain FP64; p99 latency")
UNIT = "particles/s"
N_PART = 50_000_000
RES = 1024
N_ATTR = 3

# name -> (generator, default particles, mesh side, attributes, dtype label, description)
WORKLOADS = {
    "plummer1024": ("plummer", 50_000_000, 1024, 3, "f64",
                    "plummer a=1 r<10 x-y, {n:,} particles, 3 f64 attributes, 1024x1024 mesh over "
                    "[-10,10]^2, count/sum/min/max/avg"),
    "uniform64": ("uniform", 100_000, 64, 2, "f64",
                  "uniform [0,1)^2, {n:,} particles, f64 mass U[1,2] and speed |N(0,1)|, 64x64 mesh, "
                  "count/sum/min/max/avg"),
    "uniform64_at_scale": ("uniform", 2 ** 27, 64, 2, "f64",
                           "uniform [0,1)^2, {n:,} particles, f64 mass U[1,2] and speed |N(0,1)|, "
                           "64x64 mesh, count/sum/min/max/avg"),
    "gaussians4096": ("gaussians", 2 ** 27, 4096, 2, "f32",
                      "16-Gaussian mixture in [0,1)^2, {n:,} f32 particles, 2 f32 attributes "
                      "U[0,1e4], 4096x4096 mesh, count/sum/min/max/avg"),
}
# kernel sources whose ncu traffic record applies, per particle-pass strategy
KERNEL_SOURCES = {
    "global": ["paper_2310_02926_gb300/csrc/k_global.cu"],
    "private": ["paper_2310_02926_gb300/csrc/k_private.cu", "paper_2310_02926_gb300/csrc/bn_device.cuh"],
    "sort": ["paper_2310_02926_gb300/csrc/k_sort.cu", "paper_2310_02926_gb300/csrc/bn_device.cuh"],
}
COMMON_SOURCES = ["paper_2310_02926_gb300/csrc/bn_internal.cuh"]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured hbm_gbs (MEASURED_PEAKS.json, copy)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def kernel_source_sha(strategy: str) -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES.get(strategy, []) + COMMON_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, strategy: str, n: int):
    """DRAM bytes per launch of the particle pass from the committed ncu
    record for this workload and strategy, if it was taken on the current
    kernel source and at this size."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            recs = json.load(f)
        for t in recs if isinstance(recs, list) else [recs]:
            if (t.get("workload") == workload and t.get("strategy") == strategy
                    and t.get("full_n") == n and t.get("source_sha") == kernel_source_sha(strategy)):
                return t.get("dram_bytes_per_launch_full"), t.get("note")
    except Exception:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons every 100 ms in the background."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        inside = [s for s in self.samples if t0 - 0.15 <= s[0] <= t1 + 0.15] or self.samples
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[2]) for _, p in inside if num(p[2]) is not None]
        mx = [num(p[3]) for _, p in inside if num(p[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, p in inside for k in range(4)
                          if p[5 + k].lower() in ("active", "1", "yes")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, n: int, seed: int):
    import numpy as np
    import workloads
    gen, _, side, _, dt, _ = WORKLOADS[name]
    dtype = np.float64 if dt == "f64" else np.float32
    return getattr(workloads, gen)(n, seed=seed, dtype=dtype, res=side)


def workload_config(name: str, n: int, input_bytes: int):
    gen, _, side, n_attrs, dt, desc = WORKLOADS[name]
    l2 = (f"inputs {input_bytes / 1e9:.2f} GB > 129 MB L2: no flush between steps"
          if input_bytes > 129e6 else
          f"inputs {input_bytes / 1e6:.1f} MB fit in L2: L2-resident latency case, not an HBM figure")
    return {"workload": desc.format(n=n), "name": name, "n_particles": n, "grid": [side, side],
            "n_attrs": n_attrs, "dtype": dt, "l2": l2}


def time_oracle(w, min_seconds: float, max_reps: int):
    import oracle
    oracle.bin_workload(w.__class__(w.name, w.x[:1000], w.y[:1000], [a[:1000] for a in w.attrs],
                                    w.lo, w.hi, w.res))  # load + warm
    reps, t = 0, 0.0
    while reps < max_reps and (t < min_seconds or reps == 0):
        t0 = time.perf_counter()
        oracle.bin_workload(w)
        t += time.perf_counter() - t0
        reps += 1
    return w.n * reps / t, reps, t


def run_reference(args):
    """The CPU oracle as the reference arm (bounded sample per step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import workloads
    sample_n = min(args.reference_sample, WORKLOADS[args.workload][1])
    w = make_workload(args.workload, sample_n, seed=0)
    import oracle
    oracle.build()
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.bin_workload(w)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.bin_workload(w)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sample_n * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": WORKLOADS[args.workload][4],
            "data": "synthetic", "impl": "reference",
            "config": workload_config(args.workload, WORKLOADS[args.workload][1], w.bytes_read()),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample_n:,} particles of the same workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    global N_PART
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-sample", type=int, default=2_000_000)
    ap.add_argument("--strategy", default="auto", choices=["auto", "global", "private", "sort"])
    ap.add_argument("--workload", default="plummer1024", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0,
                    help="particles (0 = the workload's size; smaller cases for profiling runs)")
    ap.add_argument("--sum", default="f32c", choices=["f32c", "f32", "f64"],
                    help="sum mode for f32 workloads")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    N_PART = args.n or WORKLOADS[args.workload][1]

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as bn
    import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    w = make_workload(args.workload, N_PART, seed=rank)
    RES = w.res[0]
    N_ATTR = len(w.attrs)
    B = RES * RES
    tdtype = torch.float64 if w.x.dtype == np.float64 else torch.float32
    dt_label = WORKLOADS[args.workload][4]
    stream = torch.cuda.Stream(device=dev)
    cols = [torch.from_numpy(c).to(dev) for c in (w.x, w.y, *w.attrs)]
    ctx = bn.Context(local, stream=stream.cuda_stream, profile=True)
    flags = {"auto": 0, "global": bn.STRATEGY_GLOBAL, "private": bn.STRATEGY_PRIVATE,
             "sort": bn.STRATEGY_SORT}[args.strategy]
    ops = bn.OP_ALL | flags | {"f32c": bn.SUM_F32C, "f32": bn.SUM_F32, "f64": bn.SUM_F64}[args.sum]
    g = bn.grid(w.lo, w.hi, w.res)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        out = bn.alloc_outputs(N_ATTR, B, tdtype, dev)
        res_struct = bn.result_struct(out)

        def step():
            return bn.bn_bin_particles(ctx.handle, cols[0], cols[1], cols[2:], g, ops,
                                       res_struct, sync=False)

        clocks = ClockSampler(local).start()
        for _ in range(args.warmup):
            bn.bn_request_release(step())
        stream.synchronize()
        bn.bn_context_profile(ctx.handle)  # forget warm-up launches
        launches0 = ctx.launches
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_wall0 = time.time()
        ev0.record(stream)
        reqs = [step() for _ in range(args.steps)]
        ev1.record(stream)
        ev1.synchronize()
        t_wall1 = time.time()
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        for r in reqs:
            bn.bn_request_release(r)
        elapsed_ms = ev0.elapsed_time(ev1)
        gpu_launches = ctx.launches - launches0
        kern_ms, kern_launches, strategy = bn.bn_context_profile(ctx.handle)
        time.sleep(0.3)
        clocks.stop()
        clk = clocks.summary(t_wall0, t_wall1)
    if pg:
        t = torch.tensor([elapsed_ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    value = N_PART * args.steps * world / (elapsed_ms / 1e3)
    bytes_in = w.bytes_read()
    tsz = w.x.dtype.itemsize
    bytes_state = B * (8 + N_ATTR * (8 + 2 * tsz))   # count, sum, min, max
    bytes_out = w.bytes_written()                    # + avg
    hbm, peak_src = peaks()
    step_gbs = (bytes_in + bytes_out) / (elapsed_ms / args.steps / 1e3) / 1e9
    kern_avg_ms = kern_ms / max(1, kern_launches)
    kern_bytes = bytes_in + bytes_state
    achieved = kern_bytes / (kern_avg_ms / 1e3) / 1e9 if kern_launches else None
    traffic, traffic_note = ncu_traffic(args.workload, strategy, N_PART)

    # end to end through the public API with pinned host buffers
    e2e = None
    if args.e2e_steps > 0 and rank == 0:
        hcols = [torch.from_numpy(c).pin_memory() for c in (w.x, w.y, *w.attrs)]
        hout = bn.alloc_outputs(N_ATTR, B, tdtype, torch.device("cpu"))
        for k in ("count",):
            hout[k] = hout[k].pin_memory()
        for k in ("sum", "min", "max", "avg"):
            hout[k] = [t.pin_memory() for t in hout[k]]
        ctx.bin_particles(hcols[0], hcols[1], hcols[2:], w.lo, w.hi, w.res, ops=ops, out=hout)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.bin_particles(hcols[0], hcols[1], hcols[2:], w.lo, w.hi, w.res, ops=ops, out=hout)
        t_e2e = (time.perf_counter() - t0) / args.e2e_steps
        bn.bn_context_profile(ctx.handle)
        e2e = {"value": N_PART / t_e2e, "unit": UNIT, "h2d_bytes_per_step": bytes_in,
               "d2h_bytes_per_step": bytes_out, "ms_per_step": 1e3 * t_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, reps, secs = time_oracle(w, min_seconds=10.0, max_reps=4)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the full workload ({N_PART:,} particles) x {reps}, {secs:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dt_label, "data": "synthetic",
            "config": dict(workload_config(args.workload, N_PART, bytes_in), strategy=strategy,
                           sum_mode=args.sum if dt_label == "f32" else "f64",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "hbm_frac_step": step_gbs / hbm,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                         "kernel": f"particle pass ({strategy} strategy)",
                         "algorithmic_bytes_per_launch": kern_bytes,
                         "avg_launch_ms": kern_avg_ms, "peak_source": peak_src,
                         "traffic_note": traffic_note},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
