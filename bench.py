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
import hashlib
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
    "batch256": ("batch", 256, 0, 2, "f32",
                 "{n} blocks of log-uniform 1e3..1e7 f32 particles (uniform or Plummer per block), "
                 "square meshes log-uniform 32..2048, 2 attributes, one bn_bin_batch call"),
    "multigrid": ("multigrid", 2 ** 22, 256, 10, "f64",
                  "{n:,} f64 particles of a Plummer snapshot (positions, velocities, 4 derived "
                  "scalars), 10 variables binned in 9 coordinate systems on 256x256 meshes, "
                  "one fused bn_bin_multi call vs 9 bn_bin_particles calls"),
    "serving": ("serving", 10_000, 0, 3, "f32",
                "Poisson stream of {n:,} requests (mean 2 ms apart, log-uniform 1e4..2e7 f32 "
                "particles, meshes 64^2..1024^2) under a 40 GB budget beside a direct-sum "
                "gravity producer (N=65,536 f32)"),
}
# kernel sources whose ncu traffic record applies, per particle-pass strategy
KERNEL_SOURCES = {
    "global": ["paper_2310_02926_gb300/csrc/k_global.cu", "paper_2310_02926_gb300/csrc/bn_device.cuh"],
    "private": ["paper_2310_02926_gb300/csrc/k_private.cu", "paper_2310_02926_gb300/csrc/bn_device.cuh"],
    "sort": ["paper_2310_02926_gb300/csrc/k_sort.cu", "paper_2310_02926_gb300/csrc/bn_device.cuh"],
    "hybrid": ["paper_2310_02926_gb300/csrc/k_window.cu", "paper_2310_02926_gb300/csrc/bn_device.cuh"],
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
            "config": {k: v for k, v in workload_config(args.workload, WORKLOADS[args.workload][1],
                                                         w.bytes_read()).items() if k != "l2"} | {
                "sample_particles_per_step": sample_n,
                "timed": f"the CPU oracle (single thread) on a {sample_n:,}-particle draw of the same "
                         f"workload (same generator and seed) per step; particles/s is sample "
                         f"particles / time"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"a {sample_n:,}-particle draw of the same workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def compare_with_oracle(w, out, bn):
    """Per-bin error of the GPU result against the CPU oracle: counts, min
    and max must match exactly; for sums, |gpu - oracle| / sum|a| over
    non-empty bins (max and 99th percentile)."""
    import numpy as np
    import oracle
    ref = oracle.bin_workload(w)
    sabs = oracle.bin_particles(w.x, w.y, [np.abs(a) for a in w.attrs], w.lo, w.hi, w.res)["sum"]
    cnt = out["count"].cpu().numpy().astype(np.uint64)
    res = {"count_exact": bool(np.array_equal(cnt, ref["count"]))}
    ne = ref["count"] > 0
    rel_all = []
    for a in range(len(w.attrs)):
        g = out["sum"][a].cpu().numpy()
        mn = out["min"][a].cpu().numpy()
        mx = out["max"][a].cpu().numpy()
        res[f"min{a}_exact"] = bool(np.array_equal(mn.view(np.int64 if mn.itemsize == 8 else np.int32),
                                                   ref["min"][a].view(np.int64 if mn.itemsize == 8 else np.int32)))
        res[f"max{a}_exact"] = bool(np.array_equal(mx.view(np.int64 if mx.itemsize == 8 else np.int32),
                                                   ref["max"][a].view(np.int64 if mx.itemsize == 8 else np.int32)))
        rel = np.abs(g[ne] - ref["sum"][a][ne]) / sabs[a][ne]
        rel_all.append(rel)
    rel = np.concatenate(rel_all) if rel_all else np.zeros(1)
    res["sum_rel_err_max"] = float(rel.max())
    res["sum_rel_err_p99"] = float(np.percentile(rel, 99))
    res["bins_checked"] = int(ne.sum())
    return res


def run_batch(args, n_blocks):
    """Batching: every block of the plan binned in one bn_bin_batch call
    (f32 columns, compensated FP32 sums), against the same blocks in f64
    binned one bn_bin_particles call after another (the plain FP64 form)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as bn
    import workloads
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    plan = workloads.batch(n_blocks=n_blocks, seed=0)
    ctx = bn.Context(0, stream=stream.cuda_stream)
    blocks32, keep, outs64, cols64 = [], [], [], []
    total = 0
    t0 = time.time()
    with torch.cuda.stream(stream):
        for k in range(plan.n_blocks):
            w = plan.block(k)
            total += w.n
            c32 = [torch.from_numpy(c).to(dev) for c in (w.x, w.y, *w.attrs)]
            o32 = bn.alloc_outputs(2, w.res[0] * w.res[1], torch.float32, dev)
            r32 = bn.result_struct(o32)
            keep.append((c32, o32, r32))
            blocks32.append(bn.block(c32[0], c32[1], c32[2:], bn.grid(w.lo, w.hi, w.res), r32))
            c64 = [c.double() for c in c32]
            o64 = bn.alloc_outputs(2, w.res[0] * w.res[1], torch.float64, dev)
            cols64.append((c64, bn.grid(w.lo, w.hi, w.res), bn.result_struct(o64), o64))
        gen_s = time.time() - t0
        ops = bn.OP_ALL | bn.SUM_F32C | {"auto": 0, "global": bn.STRATEGY_GLOBAL,
                                         "private": bn.STRATEGY_PRIVATE,
                                         "sort": bn.STRATEGY_SORT, "hybrid": bn.STRATEGY_HYBRID}[args.strategy]

        clocks = ClockSampler(0).start()
        walls = {}

        def timed(fn, steps, warm, key):
            for _ in range(warm):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = ctx.launches
            t_a = time.time()
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            e1.synchronize()
            walls[key] = (t_a, time.time())
            return e0.elapsed_time(e1) / steps, (ctx.launches - l0) // steps

        # request handles of asynchronous calls are freed as they complete
        def batched():
            r = bn.bn_bin_batch(ctx.handle, blocks32, ops, sync=False)
            bn.bn_request_release(r)

        def plain():
            for c64, g, r, _ in cols64:
                q = bn.bn_bin_particles(ctx.handle, c64[0], c64[1], c64[2:], g, bn.OP_ALL, r, sync=False)
                bn.bn_request_release(q)

        ms_b, launches_b = timed(batched, args.steps, args.warmup, "batched")
        ms_p, launches_p = timed(plain, max(3, args.steps // 4), 3, "plain")
        time.sleep(0.3)
        clocks.stop()
        clk = clocks.summary(walls["batched"][0], walls["plain"][1])
    bytes32 = total * 16
    bins_total = sum(int(plan.sides[k]) ** 2 for k in range(plan.n_blocks))
    out_bytes = bins_total * (8 + 2 * (8 + 4 + 4 + 8))   # count, and sum/min/max/avg per attribute
    hbm, peak_src = peaks()
    tuning = bn.bn_context_autotune_report(ctx.handle).strip().splitlines()
    line = {"metric": METRIC, "value": total / (ms_b / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["batch256"][5].format(n=plan.n_blocks),
                       "name": "batch256", "n_particles": total, "n_blocks": plan.n_blocks,
                       "sum_mode": "f32c", "l2": "inputs 4+ GB > L2"},
            "batched_fp32": {"particles_per_s": total / (ms_b / 1e3), "ms": ms_b,
                             "hbm_frac_read": bytes32 / (ms_b / 1e3) / 1e9 / hbm,
                             "hbm_frac_algorithmic": (bytes32 + out_bytes) / (ms_b / 1e3) / 1e9 / hbm,
                             "gpu_launches_per_step": launches_b},
            "plain_fp64": {"particles_per_s": total / (ms_p / 1e3), "ms": ms_p,
                           "gpu_launches_per_step": launches_p},
            "speedup_batched_fp32_vs_plain_fp64": ms_p / ms_b,
            "bins_total": bins_total, "output_bytes": out_bytes,
            "autotuner": tuning,
            "data_generation_s": gen_s,
            "gpu_launches": launches_b * args.steps,
            "clocks": clk}
    if args.check:
        # blocks in a seeded random order, each against the oracle, until the
        # time budget is spent (the sample is stated in the result)
        import numpy as np
        order = np.random.default_rng(7).permutation(plan.n_blocks)
        worst, exact, checked, parts = 0.0, True, 0, 0
        t_chk = time.time()
        for k in order:
            if checked and time.time() - t_chk > args.check_seconds:
                break
            w = plan.block(int(k))
            o = {kk: vv for kk, vv in keep[int(k)][1].items()}
            e = compare_with_oracle(w, o, bn)
            worst = max(worst, e["sum_rel_err_max"])
            exact = exact and e["count_exact"] and all(v for kk, v in e.items() if kk.endswith("_exact"))
            checked += 1
            parts += w.n
        line["errors_vs_oracle"] = {
            "exact_count_min_max": exact, "sum_rel_err_max": worst, "tolerance": 1e-6,
            "sample": f"{checked} of {plan.n_blocks} blocks ({parts:,} of {total:,} particles), "
                      f"seeded random order, {args.check_seconds:.0f} s budget"}
    ctx.close()
    return line


def run_multigrid(args, n):
    """Fused multi-grid pass: 10 variables in 9 coordinate systems (Sec. 4.3)
    binned by one bn_bin_multi call, against the same 90 binnings as 9
    bn_bin_particles calls. Both read the columns from HBM."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as bn
    import workloads
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    ctx = bn.Context(0, stream=stream.cuda_stream)
    cols = workloads.phase_space(n, seed=0)
    names = list(cols)
    res = (args.multigrid_res, args.multigrid_res)
    with torch.cuda.stream(stream):
        tcols = [torch.from_numpy(cols[k]).to(dev) for k in names]
        specs, outs, keep, sep = [], [], [], []
        variables = [names.index(v) for v in workloads.PHASE_SPACE_VARIABLES[:args.multigrid_vars]]
        for (a, b) in workloads.PHASE_SPACE_SYSTEMS:
            ha, hb = workloads.PHASE_SPACE_BOUNDS[a], workloads.PHASE_SPACE_BOUNDS[b]
            g = bn.grid((-ha, -hb), (ha, hb), res)
            specs.append(bn.grid_spec(names.index(a), names.index(b), variables, g))
            o = bn.alloc_outputs(len(variables), res[0] * res[1], torch.float64, dev)
            keep.append(o)
            outs.append(bn.result_struct(o))
            o2 = bn.alloc_outputs(len(variables), res[0] * res[1], torch.float64, dev)
            sep.append((names.index(a), names.index(b), g, bn.result_struct(o2), o2))

        def timed(fn, steps, warm):
            for _ in range(warm):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = ctx.launches
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / steps, (ctx.launches - l0) // steps

        def fused():
            r = bn.bn_bin_multi(ctx.handle, tcols, specs, bn.OP_ALL, outs, sync=False)
            bn.bn_request_release(r)

        sep_ops = bn.OP_ALL | {"auto": 0, "global": bn.STRATEGY_GLOBAL, "private": bn.STRATEGY_PRIVATE,
                               "sort": bn.STRATEGY_SORT, "hybrid": bn.STRATEGY_HYBRID}[args.strategy]

        def separate():
            for (ia, ib, g, r, _) in sep:
                q = bn.bn_bin_particles(ctx.handle, tcols[ia], tcols[ib], [tcols[v] for v in variables],
                                        g, sep_ops, r, sync=False)
                bn.bn_request_release(q)

        ms_f, launches_f = timed(fused, args.steps, args.warmup)
        ms_s, launches_s = timed(separate, max(1, args.steps // 4), args.warmup)
    B = res[0] * res[1]
    nv = len(variables)
    bytes_in = n * 8 * len(names)                     # every column once
    bytes_out = len(specs) * B * (8 + nv * 4 * 8)     # count, and sum/min/max/avg per variable
    hbm, peak_src = peaks()
    achieved = (bytes_in + bytes_out) / (ms_f / 1e3) / 1e9
    line = {"metric": METRIC, "value": n / (ms_f / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_f,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["multigrid"][5].format(n=n).replace(
                           "10 variables", f"{nv} variables").replace("256x256", f"{res[0]}x{res[1]}"),
                       "name": "multigrid",
                       "n_particles": n, "columns": len(names), "systems": len(specs),
                       "variables": nv, "grid": list(res), "l2": "inputs 0.44 GB > L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": "whole step (fused pass + per-spec set-up and finalise)",
                         "algorithmic_bytes_per_launch": bytes_in + bytes_out,
                         "peak_source": peak_src},
            "fused": {"ms": ms_f, "particles_per_s": n / (ms_f / 1e3), "gpu_launches_per_step": launches_f},
            "separate": {"ms": ms_s, "particles_per_s": n / (ms_s / 1e3), "gpu_launches_per_step": launches_s},
            "speedup_fused_vs_separate": ms_s / ms_f,
            "separate_strategy": args.strategy,
            "autotuner": bn.bn_context_autotune_report(ctx.handle).strip().splitlines(),
            "gpu_launches": launches_f * args.steps, "e2e": None, "cpu_baseline": None}
    if args.check:
        worst, exact = 0.0, True
        for k, (a, b) in enumerate(workloads.PHASE_SPACE_SYSTEMS):
            ha, hb = workloads.PHASE_SPACE_BOUNDS[a], workloads.PHASE_SPACE_BOUNDS[b]
            w = workloads.Workload(f"{a}-{b}", cols[a], cols[b],
                                   [cols[v] for v in workloads.PHASE_SPACE_VARIABLES[:args.multigrid_vars]],
                                   (-ha, -hb), (ha, hb), res)
            e = compare_with_oracle(w, dict(keep[k]), bn)
            worst = max(worst, e["sum_rel_err_max"])
            exact = exact and all(v for kk, v in e.items() if kk.endswith("_exact"))
        line["errors_vs_oracle"] = {"exact_count_min_max": exact, "sum_rel_err_max": worst}
    ctx.close()
    return line


def run_serving(args, n_requests):
    """Serving: a Poisson stream of requests submitted to a bn_server at
    their arrival times while the n-body producer runs on its own stream;
    latency is arrival -> completion seen by the submitting thread."""
    import ctypes
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as bn
    import workloads
    dev = torch.device("cuda", 0)
    plan = workloads.serving(n_requests=n_requests, seed=0)
    pool = [torch.from_numpy(c).to(dev) for c in (plan.pool.x, plan.pool.y, *plan.pool.attrs)]
    ctx = bn.Context(0)
    try:
        lo_prio, hi_prio = torch.cuda.Stream.priority_range()
    except Exception:
        lo_prio, hi_prio = 0, -1
    prio = hi_prio if args.serving_priority == "high" else lo_prio
    srv = bn.bn_server_create(ctx.handle, 40 << 30, max_inflight=4, max_batch=32, priority=prio)
    # output slots, reused once their request has completed
    max_side = int(plan.sides.max())
    n_slots = 128
    slots = [bn.alloc_outputs(3, max_side * max_side, torch.float32, dev) for _ in range(n_slots)]
    free = list(range(n_slots))
    # producer: direct-sum gravity, N = 65,536, its own stream
    prod_stream = torch.cuda.Stream(device=dev)
    g = torch.Generator().manual_seed(1)
    nb = 65_536
    pos = torch.zeros(nb, 4)
    pos[:, :3] = torch.randn(nb, 3, generator=g)
    pos[:, 3] = 1.0 / nb
    pos, vel, acc = pos.to(dev), torch.zeros(nb, 4, device=dev), torch.zeros(nb, 4, device=dev)
    acc_ok = ctypes.c_int(0)
    stop = threading.Event()
    prod_times = []

    def producer():
        torch.cuda.set_device(dev)
        evs = []
        while not stop.is_set():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(prod_stream)
            bn.bn_nbody_step(pos, vel, acc, acc_ok, 1e-3, 1e-3, prod_stream.cuda_stream)
            e1.record(prod_stream)
            evs.append((e0, e1))
            if len(evs) > 2:
                a, b = evs.pop(0)
                b.synchronize()
                prod_times.append(a.elapsed_time(b))

    def producer_alone(seconds):
        th = threading.Thread(target=producer)
        th.start()
        time.sleep(seconds)
        stop.set()
        th.join()
        stop.clear()
        t = list(prod_times)
        prod_times.clear()
        return t

    alone = producer_alone(2.0) if not args.no_producer else []
    th = threading.Thread(target=producer)
    if not args.no_producer:
        th.start()
        time.sleep(0.5)
    prod_times.clear()
    lat, outstanding, served, parts = [], [], 0, []
    clocks = ClockSampler(0).start()
    t_wall0 = time.time()
    t_start = time.perf_counter()
    i = 0
    while i < plan.n_requests or outstanding:
        now = time.perf_counter() - t_start
        while i < plan.n_requests and plan.arrival_s[i] <= now and free:
            o0, n, side = int(plan.offsets[i]), int(plan.sizes[i]), int(plan.sides[i])
            sl = free.pop()
            o = {k: (v[:side * side] if not isinstance(v, list) else [t[:side * side] for t in v])
                 for k, v in slots[sl].items()}
            r = bn.result_struct(o, stream=0)
            blk = bn.block(*[c[o0:o0 + n] for c in pool[:2]], [c[o0:o0 + n] for c in pool[2:]],
                           bn.grid((-10, -10), (10, 10), (side, side)), r, stream=0)
            t_call = time.perf_counter() - t_start
            req = bn.bn_server_submit(srv, blk, bn.OP_ALL)
            outstanding.append((req, plan.arrival_s[i], n, sl, r, blk, t_call - plan.arrival_s[i]))
            i += 1
        keep = []
        now = time.perf_counter() - t_start
        for item in outstanding:
            st = bn.lib().bn_query(item[0])
            if st == bn.NOT_READY:
                keep.append(item)
                continue
            if st < 0:
                raise RuntimeError(f"request failed: {st}")
            lat.append(now - item[1])
            tm = bn.bn_server_request_timing(item[0]) or {}
            tm["lag_us"] = 1e6 * item[6]
            parts.append(tm)
            served += item[2]
            free.append(item[3])
            bn.bn_request_release(item[0])
        outstanding = keep
    wall = time.perf_counter() - t_start
    t_wall1 = time.time()
    time.sleep(0.3)
    clocks.stop()
    clk = clocks.summary(t_wall0, t_wall1)
    stop.set()
    if not args.no_producer:
        th.join()
    with_serving = list(prod_times)
    stats = bn.bn_server_stats_get(srv)
    bn.bn_server_destroy(srv)
    ctx.close()
    lat_ms = np.array(lat) * 1e3
    # where the time goes: the bench's own lag before submit (an output slot
    # to reuse, the polling loop), then the server's record of each stage
    comp = {"bench_lag": "lag_us", "submit": "submit_us", "queue": "queue_us", "launch": "launch_us",
            "complete": "complete_us", "batch_gpu": "batch_gpu_us"}
    cols = {k: np.array([p.get(v, 0.0) for p in parts]) / 1e3 for k, v in comp.items()}
    accounted = sum(cols[k] for k in ("bench_lag", "submit", "queue", "launch", "complete"))
    cols["poll"] = np.maximum(lat_ms - accounted, 0.0)
    tail = lat_ms >= np.percentile(lat_ms, 99)
    split = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)),
                 "mean_in_p99_tail": float(v[tail].mean())} for k, v in cols.items()}
    split["batch_size"] = {"p50": float(np.percentile([p.get("batch_size", 0) for p in parts], 50)),
                           "max": float(max(p.get("batch_size", 0) for p in parts))}
    line = {"metric": METRIC, "value": served / wall, "unit": UNIT, "n_gpus": 1,
            "steps": plan.n_requests, "warmup": 0, "ms_per_step": wall * 1e3 / plan.n_requests,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["serving"][5].format(n=plan.n_requests),
                       "name": "serving", "budget_gb": 40, "max_inflight": 4, "max_batch": 32,
                       "server_priority": args.serving_priority, "producer": not args.no_producer},
            "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                           "max": float(lat_ms.max()), "mean": float(lat_ms.mean())},
            "particles_served": int(served), "wall_s": wall,
            "producer_step_ms": {"alone": float(np.median(alone)) if alone else None,
                                 "with_serving": float(np.median(with_serving)) if with_serving else None},
            "latency_split_ms": split,
            "server": stats,
            "clocks": clk}
    return line


def host_link_gbs(dev, nbytes: int = 1 << 30, reps: int = 5):
    """Page-locked host <-> device copy rates (GB/s, best of reps)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = None
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        out[name] = nbytes / (best / 1e3) / 1e9
    del h, d
    return out


def time_threaded_baseline(w, min_seconds: float, max_reps: int):
    """The all-core CPU baseline (oracle/binning_threaded.c) on the whole
    workload: particles/s and the threads it used."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    oracle.bin_particles_threaded(w.x[:1000], w.y[:1000], [a[:1000] for a in w.attrs], w.lo, w.hi,
                                  w.res, threads=threads)  # load + warm
    reps, t = 0, 0.0
    while reps < max_reps and (t < min_seconds or reps == 0):
        t0 = time.perf_counter()
        oracle.bin_particles_threaded(w.x, w.y, w.attrs, w.lo, w.hi, w.res, threads=threads)
        t += time.perf_counter() - t0
        reps += 1
    return w.n * reps / t, reps, t, threads


def run_single(args, name, n, env, with_e2e=True, with_cpu=True, check=False, steps=None):
    """One bn_bin_particles call per step on a single workload; returns the
    JSON object (the headline line, or a sub-object of it)."""
    import numpy as np
    import torch
    import paper_2310_02926_gb300 as bn

    rank, world, local, pg = env
    steps = steps or args.steps
    dev = torch.device("cuda", local)
    w = make_workload(name, n, seed=rank)
    B = w.res[0] * w.res[1]
    n_attr = len(w.attrs)
    tdtype = torch.float64 if w.x.dtype == np.float64 else torch.float32
    dt_label = WORKLOADS[name][4]
    stream = torch.cuda.Stream(device=dev)
    cols = [torch.from_numpy(c).to(dev) for c in (w.x, w.y, *w.attrs)]
    ctx = bn.Context(local, stream=stream.cuda_stream, profile=True)
    flags = {"auto": 0, "global": bn.STRATEGY_GLOBAL, "private": bn.STRATEGY_PRIVATE,
             "sort": bn.STRATEGY_SORT, "hybrid": bn.STRATEGY_HYBRID}[args.strategy]
    op_bits = {"all": bn.OP_ALL, "count": bn.OP_COUNT, "count+sum": bn.OP_COUNT | bn.OP_SUM,
               "count+minmax": bn.OP_COUNT | bn.OP_MIN | bn.OP_MAX}[args.ops]
    ops = op_bits | flags | {"f32c": bn.SUM_F32C, "f32": bn.SUM_F32, "f64": bn.SUM_F64}[args.sum]
    g = bn.grid(w.lo, w.hi, w.res)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        out = bn.alloc_outputs(n_attr, B, tdtype, dev, ops=op_bits)
        res_struct = bn.result_struct(out)
        exchange = None
        if world > 1 and op_bits == bn.OP_ALL:
            # every rank bins its own particles onto the same mesh; each step
            # ends with the one exchange the path has: the partial meshes
            # combine (SUM, SUM, MIN, MAX over NCCL), then avg is recomputed
            exchange = torch.empty(bn.bn_exchange_bytes(B, n_attr), dtype=torch.uint8, device=dev)
            whole = bn.alloc_outputs(n_attr, B, tdtype, dev)
            whole_struct = bn.result_struct(whole)
            code = bn.F64 if dt_label == "f64" else bn.F32

        def step():
            # request handles of the step's asynchronous calls, released later
            rs = [bn.bn_bin_particles(ctx.handle, cols[0], cols[1], cols[2:], g, ops, res_struct,
                                      sync=False)]
            if exchange is not None:  # all on the context's stream, in order
                rs.append(bn.bn_exchange_pack(ctx.handle, res_struct, code, n_attr, B, exchange, sync=False))
                bn.allreduce_exchange(exchange, B, n_attr)
                rs.append(bn.bn_exchange_unpack(ctx.handle, exchange, code, n_attr, B, bn.OP_ALL,
                                                whole_struct, sync=False))
            return rs

        def release(rs):
            for r in rs:
                bn.bn_request_release(r)

        clocks = ClockSampler(local).start()
        for _ in range(args.warmup):
            release(step())
        stream.synchronize()
        bn.bn_context_profile(ctx.handle)  # forget warm-up launches
        launches0 = ctx.launches
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_wall0 = time.time()
        ev0.record(stream)
        reqs = [step() for _ in range(steps)]
        ev1.record(stream)
        ev1.synchronize()
        t_wall1 = time.time()
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        for rs in reqs:
            release(rs)
        elapsed_ms = ev0.elapsed_time(ev1)
        gpu_launches = ctx.launches - launches0
        kern_ms, kern_launches, strategy = bn.bn_context_profile(ctx.handle)
        tuning = bn.bn_context_autotune_report(ctx.handle).strip().splitlines()
        time.sleep(0.3)
        clocks.stop()
        clk = clocks.summary(t_wall0, t_wall1)
    if pg:
        t = torch.tensor([elapsed_ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    value = n * steps * world / (elapsed_ms / 1e3)
    bytes_in = w.bytes_read()
    tsz = w.x.dtype.itemsize
    bytes_state = B * (8 + n_attr * (8 + 2 * tsz))   # count, sum, min, max
    bytes_out = w.bytes_written()                    # + avg
    hbm, peak_src = peaks()
    step_gbs = (bytes_in + bytes_out) / (elapsed_ms / steps / 1e3) / 1e9
    kern_avg_ms = kern_ms / max(1, kern_launches)
    kern_bytes = bytes_in + bytes_state
    achieved = kern_bytes / (kern_avg_ms / 1e3) / 1e9 if kern_launches else None
    traffic, traffic_note = ncu_traffic(name, strategy, n)

    # end to end through the public API with pinned host buffers
    e2e = None
    if with_e2e and args.e2e_steps > 0 and rank == 0:
        hcols = [torch.from_numpy(c).pin_memory() for c in (w.x, w.y, *w.attrs)]
        hout = bn.alloc_outputs(n_attr, B, tdtype, torch.device("cpu"), ops=op_bits)
        for k in list(hout):
            hout[k] = [t.pin_memory() for t in hout[k]] if isinstance(hout[k], list) else hout[k].pin_memory()
        ctx.bin_particles(hcols[0], hcols[1], hcols[2:], w.lo, w.hi, w.res, ops=ops, out=hout)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.bin_particles(hcols[0], hcols[1], hcols[2:], w.lo, w.hi, w.res, ops=ops, out=hout)
        t_e2e = (time.perf_counter() - t0) / args.e2e_steps
        bn.bn_context_profile(ctx.handle)
        link = host_link_gbs(dev)
        moved = (bytes_in + bytes_out) / t_e2e / 1e9
        # the host link bounds end to end: the inputs cross it once (read in
        # place from page-locked memory) and the outputs once
        bound_s = bytes_in / (link["h2d_gbs"] * 1e9) + bytes_out / (link["d2h_gbs"] * 1e9)
        e2e = {"value": n / t_e2e, "unit": UNIT, "h2d_bytes_per_step": bytes_in,
               "d2h_bytes_per_step": bytes_out, "ms_per_step": 1e3 * t_e2e,
               "roofline": {"bound": "host link", "achieved_gbs": moved, "host_link": link,
                            "frac": bound_s / t_e2e,
                            "note": "frac = (h2d bytes / h2d copy rate + d2h bytes / d2h copy rate) / "
                                    "e2e step time; rates are page-locked cudaMemcpy copies of 1 GiB"}}

    errors = None
    if check and rank == 0:
        errors = compare_with_oracle(w, out, bn)
        errors["tolerance"] = 1e-12 if dt_label == "f64" else 1e-6

    cpu = cpu1 = None
    if with_cpu and rank == 0 and world == 1:
        v, reps, secs, threads = time_threaded_baseline(w, min_seconds=5.0, max_reps=20)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "variant": "all-core FP64 oracle: per-thread private meshes, then a merge "
                          "(oracle/binning_threaded.c)",
               "sample": f"the full workload ({n:,} particles) x {reps}, {secs:.1f} s"}
        v1, reps1, secs1 = time_oracle(w, min_seconds=5.0, max_reps=4)
        cpu1 = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the full workload ({n:,} particles) x {reps1}, {secs1:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dt_label, "data": "synthetic",
        "config": dict(workload_config(name, n, bytes_in), strategy=strategy,
                       autotuner=tuning, ops=args.ops,
                       sum_mode=args.sum if dt_label == "f32" else "f64",
                       parallelism=(f"{world} ranks, each binning its own {n:,} particles; partial meshes combined "
                     f"every step (exchange buffer, NCCL all-reduce)") if world > 1 else "single GPU"),
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
    if cpu1 is not None:
        line["cpu_baseline_1core"] = cpu1
    if errors is not None:
        line["errors_vs_oracle"] = errors
    ctx.close()
    del cols, out
    torch.cuda.empty_cache()
    return line


def sub_object(line, keep=("value", "unit", "ms_per_step", "steps", "dtype", "config", "roofline",
                           "clocks", "errors_vs_oracle", "gpu_launches")):
    return {k: line[k] for k in keep if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the uniform-at-scale, batch and serving sub-objects")
    ap.add_argument("--reference-sample", type=int, default=2_000_000)
    ap.add_argument("--strategy", default="auto", choices=["auto", "global", "private", "sort", "hybrid"])
    ap.add_argument("--workload", default="plummer1024", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0,
                    help="particles (0 = the workload's size; smaller cases for profiling runs)")
    ap.add_argument("--sum", default="f32c", choices=["f32c", "f32", "f64"],
                    help="sum mode for f32 workloads")
    ap.add_argument("--serving-priority", default="high", choices=["low", "high"],
                    help="stream priority of the server relative to the producer")
    ap.add_argument("--no-producer", action="store_true", help="serving without the producer")
    ap.add_argument("--ops", default="all", choices=["all", "count", "count+sum", "count+minmax"],
                    help="reductions to compute (all = count/sum/min/max/avg, the benchmark's)")
    ap.add_argument("--multigrid-vars", type=int, default=10, choices=range(1, 11),
                    help="multigrid workload: variables binned in every coordinate system")
    ap.add_argument("--multigrid-res", type=int, default=256,
                    help="multigrid workload: mesh side of every coordinate system")
    ap.add_argument("--check", action="store_true",
                    help="compare the last step with the CPU oracle and report per-bin errors")
    ap.add_argument("--check-seconds", type=float, default=40.0,
                    help="time budget of the batch workload's oracle check")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    n = args.n or WORKLOADS[args.workload][1]
    if args.ops != "all":
        args.check = False
    standalone = {"batch256": run_batch, "serving": run_serving, "multigrid": run_multigrid}
    if args.workload in standalone:
        print(json.dumps(standalone[args.workload](args, n)), flush=True)
        return 0

    import torch
    import __graft_entry__
    __graft_entry__.build()

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    env = (rank, world, local, pg)
    line = run_single(args, args.workload, n, env, with_e2e=True,
                      with_cpu=not args.no_cpu_baseline, check=args.check)
    headline_default = args.workload == "plummer1024" and not args.n and args.ops == "all"
    if headline_default and not args.no_extras and world == 1:
        # the other targets of the benchmark's metric, each measured on its
        # own full-size workload with its own clocks record
        sub = run_single(args, "uniform64_at_scale", WORKLOADS["uniform64_at_scale"][1], env,
                         with_e2e=False, with_cpu=False, check=True, steps=50)
        line["uniform64_at_scale"] = sub_object(sub)
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup, bargs.check, bargs.strategy = 5, 3, True, "auto"
        line["batch256"] = run_batch(bargs, WORKLOADS["batch256"][1])
        sargs = argparse.Namespace(**vars(args))
        sargs.serving_priority, sargs.no_producer = "high", False
        line["serving"] = run_serving(sargs, WORKLOADS["serving"][1])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
