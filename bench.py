#!/usr/bin/env python
"""Throughput of the bilateral solver hot path on GB300.

One step = the whole forward path on one synthetic 1920 x 1080 image with a
3-channel target (sigma = (16, 8, 8), lambda = 128): grid build (quantised
keys, canonical vertices, splat map, neighbour tables), 2 bistochastisation
sweeps, splat / diag(A) / flat init, 25 Jacobi-PCG iterations and the slice.
Metric: solved Mpix/s.  Each rank solves its own image (independent problems:
weak scaling, no data-path collective).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  `--impl reference` times the FP64 CPU
oracle (the only other implementation of this method here) on the host.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solved Mpix/s (25-iter PCG, 1080p & batched), fwd+bwd Mpix/s; % HBM peak"
WORKLOAD = ("plain solve, 1920x1080 reference, C=3 piecewise-planar target, c~U[0,1], "
            "sigma=(16,8,8), lambda=128, 2 bistochastisation sweeps, 25 Jacobi-PCG iterations")
BISTOCH_ITERS = 2
PCG_ITERS = 25


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="host time spent timing the oracle for cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------ distributed --

class Dist:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local_rank)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, value: float) -> float:
        if self.pg is None:
            return value
        import torch
        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # wait (bounded) for the first sample so the timed region is covered
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None:
            self.out.flush()
            if os.fstat(self.out.fileno()).st_size > 0:
                break
            time.sleep(0.02)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle ---

def oracle_step(inst):
    import oracle
    g = oracle.build_grid(inst.yuv, inst.sigma_xy, inst.sigma_l, inst.sigma_uv, BISTOCH_ITERS)
    oracle.solve(g, inst.t, inst.c, inst.lam, PCG_ITERS)


def cpu_baseline(inst, seconds: float):
    """The FP64 oracle, as it stands, single-threaded on the host."""
    times = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        oracle_step(inst)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() >= t_end and len(times) >= 1:
            break
    mpix = inst.n_pixels * len(times) / sum(times) / 1e6
    return {"value": mpix, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": f"full {inst.width}x{inst.height} C={inst.channels} image (the bench "
                      f"workload), grid+bistochastisation+solve, {len(times)} repeats, "
                      f"{sum(times):.1f} s, single-threaded FP64 C"}


def run_reference(args, dist):
    if dist.rank != 0:
        return
    from paper_1511_03296_gb300 import synth
    inst = synth.plain_1080p().instances[0]
    budget = 150.0
    t0 = time.perf_counter()
    oracle_step(inst)
    t_full = time.perf_counter() - t0
    # each step a bounded sample: full image if it fits the budget, else a band of rows
    per_step = budget / max(1, args.steps + args.warmup)
    frac = min(1.0, per_step / max(t_full, 1e-3))
    rows = max(16, int(inst.height * frac))
    sample = inst if rows >= inst.height else synth.crop(inst, 0, 0, rows, inst.width)
    for _ in range(args.warmup):
        oracle_step(sample)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(sample)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample.n_pixels * len(times) / total / 1e6
    desc = (f"{'full' if sample is inst else f'top {rows}-row band of the'} "
            f"{inst.width}x{inst.height} C=3 image per step, single-threaded FP64 C oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pixels_per_step": sample.n_pixels},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours ---

def algorithmic_bytes_per_pcg_iteration(V: int, C: int) -> int:
    """48 + 40 C bytes per vertex: 10 neighbour ids, diag(A) and n, plus per
    channel the two-pass minimum of the CG vector traffic."""
    return V * (48 + 40 * C)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def run_ours(args, dist):
    import numpy as np
    import torch

    from paper_1511_03296_gb300 import build as fbs_build
    from paper_1511_03296_gb300 import fbs, synth

    dev = dist.local_rank if torch.cuda.device_count() > 1 else 0
    torch.cuda.set_device(dev)
    fbs_build.build()
    fbs.load()
    inst = synth.plain_1080p(seed=2 + dist.rank).instances[0]
    stream = torch.cuda.current_stream()
    d_yuv = torch.from_numpy(inst.yuv).cuda()
    d_t = torch.from_numpy(inst.t).cuda()
    d_c = torch.from_numpy(inst.c).cuda()
    d_x = torch.empty_like(d_t)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    V_holder = {}

    def step(yuv, t, c, x):
        g = fbs.grid_build([yuv], inst.sigma_xy, inst.sigma_l, inst.sigma_uv)
        fbs.bistochastize(g, BISTOCH_ITERS)
        fbs.solve(g, [t], [c], inst.lam, PCG_ITERS, x=[x])
        V_holder["V"] = g.vertex_counts[0]
        g.destroy()

    for _ in range(args.warmup):
        flush.zero_()
        step(d_yuv, d_t, d_c, d_x)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fbs.profile_enable(2)                 # region events only (2 per phase)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step(d_yuv, d_t, d_c, d_x)
            ends[i].record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    regions = fbs.profile_read()
    fbs.profile_enable(0)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_local = sum(step_ms) / len(step_ms)
    ms = dist.max(ms_local)
    value = dist.world * inst.n_pixels / (ms / 1e3) / 1e6
    V = V_holder["V"]

    # ---- per-kernel launch list of a few steps (separate pass)
    fbs.profile_enable(1)
    nprof = 3
    for _ in range(nprof):
        flush.zero_()
        step(d_yuv, d_t, d_c, d_x)
    torch.cuda.synchronize()
    kernels = fbs.profile_read()
    fbs.profile_enable(0)
    launches_per_step = sum(n for n, _ in kernels.values()) / nprof
    total_kernel_ms = sum(t for _, t in kernels.values())
    shares = {k: round(t / total_kernel_ms, 4) for k, (n, t) in kernels.items() if n}

    # ---- e2e through the public API with pinned host buffers
    h_yuv = torch.from_numpy(inst.yuv).pin_memory()
    h_t = torch.from_numpy(inst.t).pin_memory()
    h_c = torch.from_numpy(inst.c).pin_memory()
    h_x = torch.empty(inst.t.shape, dtype=torch.float32).pin_memory()
    e_yuv, e_t, e_c, e_x = (torch.empty_like(d_yuv), torch.empty_like(d_t),
                            torch.empty_like(d_c), torch.empty_like(d_x))
    e2e_steps = max(3, min(args.steps, 20))
    es = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps)]
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps)]
    for i in range(e2e_steps + 2):
        flush.zero_()
        j = i - 2
        if j >= 0:
            es[j].record(stream)
        e_yuv.copy_(h_yuv, non_blocking=True)
        e_t.copy_(h_t, non_blocking=True)
        e_c.copy_(h_c, non_blocking=True)
        step(e_yuv, e_t, e_c, e_x)
        h_x.copy_(e_x, non_blocking=True)
        if j >= 0:
            ee[j].record(stream)
    torch.cuda.synchronize()
    e2e_ms = dist.max(sum(s.elapsed_time(e) for s, e in zip(es, ee)) / e2e_steps)
    assert np.allclose(h_x.numpy(), d_x.cpu().numpy())
    h2d = inst.yuv.nbytes + inst.t.nbytes + inst.c.nbytes
    d2h = inst.t.nbytes

    # ---- roofline: the PCG iteration (apply + update), timed as a region
    loop_n, loop_ms = regions.get("region:pcg_loop", (0, 0.0))
    iter_ms = loop_ms / max(1, loop_n) / PCG_ITERS
    bytes_iter = algorithmic_bytes_per_pcg_iteration(V, inst.channels)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = bytes_iter / (iter_ms / 1e3) / 1e9 if iter_ms > 0 else None
    region_share = {k: round(t / max(1e-9, sum(tt for _, tt in regions.values())), 4)
                    for k, (n, t) in regions.items() if n}

    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "pixels_per_gpu": inst.n_pixels, "vertices": V,
                   "channels": inst.channels, "parallelism": f"replicas x{dist.world}",
                   "l2": "flushed between steps (256 MiB write outside the step events)",
                   "precision": "FP32 vectors, FP64-accurate CG dot products, FP64 "
                                "bistochastisation"},
        "clocks": clk.summary(),
        "e2e": {"value": dist.world * inst.n_pixels / (e2e_ms / 1e3) / 1e6, "unit": "Mpix/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": {"kernel": "pcg iteration (pcg_apply + pcg_update)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "peak_source": "measured" if peaks else "fallback",
                     "bytes_per_launch": bytes_iter, "iter_us": iter_ms * 1e3,
                     "note": "working set L2-resident at this size (see design notes)"},
        "phase_share": region_share,
        "kernel_share": shares,
    }
    if dist.rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(synth.plain_1080p().instances[0], args.cpu_seconds)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
