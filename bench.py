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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solved Mpix/s (25-iter PCG, 1080p & batched), fwd+bwd Mpix/s; % HBM peak"
WORKLOAD = ("plain solve, 1920x1080 reference, C=3 piecewise-planar target, c~U[0,1], "
            "sigma=(16,8,8), lambda=128, 2 bistochastisation sweeps, 25 Jacobi-PCG iterations")
L2_NOTE = ("GPU arm: L2 flushed between steps by a 256 MiB write outside the step events; "
           "CPU oracle arm: host memory, no flush")
BISTOCH_ITERS = 2
PCG_ITERS = 25


def bench_config():
    """The config object both arms print (same keys and values)."""
    return {"workload": WORKLOAD, "l2": L2_NOTE}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="host time spent timing the oracle for cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the batched and forward+backward workloads")
    p.add_argument("--precond", choices=["jacobi", "hierarchical"], default="jacobi",
                   help="preconditioner of the --only batched workload")
    p.add_argument("--only", choices=["batched", "fwd_bwd", "lowrank", "dt"], default=None,
                   help="run one extra workload alone (for profiling) and print its line")
    p.add_argument("--images", type=int, default=None,
                   help="image count of the --only workload (default: its full size)")
    p.add_argument("--tune-cache", default=None,
                   help="JSON file of autotuner choices: read when it holds the workload's "
                        "shape class, else written after timing (a profiled run then uses "
                        "the choice of a plain run)")
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


TUNE_CACHE = None     # --tune-cache


def tune(fbs, yuv, sig, t, c, lam, x):
    """The library's autotuner on one grid of the workload (its choice is then
    set on every step's grid; tuning happens outside the timed region).  Every
    step builds a new grid and solves it once, so the tuner times first solves
    on a grid (no graph replay)."""
    g = fbs.grid_build(yuv, *sig)
    fbs.bistochastize(g, BISTOCH_ITERS)
    r = fbs.autotune(g, t, c, lam, PCG_ITERS, x=x, single_solve=True, cache=TUNE_CACHE)
    g.destroy()
    return r


def rank_seed(base: int, rank: int) -> int:
    """Each rank draws its own independent problems (weak scaling)."""
    return base + rank


def whole_job_mpix(world: int, pixels_per_rank: int, ms_max: float) -> float:
    """Whole-job Mpix/s: every rank's pixels over the slowest rank's step time."""
    return world * pixels_per_rank / (ms_max / 1e3) / 1e6


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


def _oracle_worker(args):
    """One host process: repeats the oracle's 1080p step for `seconds`."""
    seconds, = args
    from paper_1511_03296_gb300 import synth
    inst = synth.plain_1080p().instances[0]
    n, t_all = 0, 0.0
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        oracle_step(inst)
        t_all += time.perf_counter() - t0
        n += 1
        if time.perf_counter() >= t_end:
            break
    return n * inst.n_pixels, t_all


def cpu_baseline_all_cores(seconds: float):
    """The oracle on every host core at once, one independent image per process
    (spawned: the parent holds a CUDA context).  Whole-host Mpix/s."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(seconds,)] * cores)
    wall = time.perf_counter() - t0
    pix = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": pix / busy / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each repeating the 1920x1080 C=3 step for about "
                      f"{seconds:.0f} s ({pix / 2073600:.0f} steps in all, {wall:.1f} s wall)"}


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
            "config": bench_config(),
            "sample_pixels_per_step": sample.n_pixels,
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


def time_steps(step, steps, warmup, flush, stream):
    """Device time (ms) of each of `steps` calls of step(), after `warmup`
    untimed calls; L2 is flushed before every call, outside the events."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]


# DRAM traffic of one PCG iteration (both phases) from one ncu capture of the
# current kernels (dram__bytes_read.sum + dram__bytes_write.sum; the summaries
# and commands are in profiles/pcg_*_batched16.md and
# profiles/pcg_resident_single_1080p.md).  ncu flushes the caches before each
# captured launch.  The 64-image batch is too large to capture under the
# profiling size rule: its 16-image prefix was captured (the z-form apply of
# an iteration >= 1 and the update, four launches each, averaged) and the
# traffic is scaled by its ratio to the algorithmic bytes (below 1: the
# gathers read 12 B of packed 8- and 16-bit neighbour offsets per vertex, not
# the 40 B of 32-bit ids the algorithmic count assumes, and the updates'
# writes stay in L2 within the captured launch).  None: the kernel changed
# since its last capture.
PCG_TRAFFIC_1080P = None
PCG_TRAFFIC_1080P_RESIDENT = None
# The resident loop of the single-reduction form at 1080p (all 25 iterations
# in one cooperative launch): dram__bytes over the launch (rate x duration),
# per iteration; after the first iteration the working set is served from L2.
PCG_TRAFFIC_1080P_RESIDENT_SINGLE = 23.025889e9 * 404.192e-6 / 25
PCG_TRAFFIC_RATIO_BATCHED = (85614656 + 2921600 + 66437824 + 509312) / 235835472


def pcg_roofline(regions, solves_per_step, steps, bytes_per_iter, peak):
    """Achieved GB/s of the PCG iteration from the region events of the
    timed steps (all PCG iterations of a step share the same byte count)."""
    n, ms = regions.get("region:pcg_loop", (0, 0.0))
    if not n:
        return None
    iter_ms = ms / n / PCG_ITERS
    achieved = bytes_per_iter / (iter_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "bytes_per_iter": bytes_per_iter, "iter_us": iter_ms * 1e3}


def run_extra_batched(dist, flush, stream, peak, steps, warmup, n_images=64, sequential=True,
                      precond="jacobi"):
    """64 images of uneven size in one grid and one batched solve, against the
    same images solved one at a time (optionally with the hierarchical
    preconditioner instead of Jacobi)."""
    import torch
    from paper_1511_03296_gb300 import fbs, synth
    wl = synth.batched_64(seed=rank_seed(4, dist.rank), n_images=n_images)
    insts = wl.instances
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    yuv = [dev(i.yuv) for i in insts]
    t = [dev(i.t) for i in insts]
    c = [dev(i.c) for i in insts]
    x = [torch.empty_like(tt) for tt in t]
    sig = ([i.sigma_xy for i in insts], [i.sigma_l for i in insts], [i.sigma_uv for i in insts])
    lam = [i.lam for i in insts]
    info = {}
    tuning = tune(fbs, yuv, sig, t, c, lam, x)

    pc = fbs.PRECOND_HIERARCHICAL if precond == "hierarchical" else fbs.PRECOND_JACOBI

    def batched():
        g = fbs.grid_build(yuv, *sig)
        fbs.apply_tuning(g, tuning)
        fbs.set_option(g, fbs.OPT_PRECONDITIONER, pc)
        fbs.bistochastize(g, BISTOCH_ITERS)
        fbs.solve(g, t, c, lam, PCG_ITERS, x=x)
        info["V"] = g.vertex_counts
        g.destroy()

    def one_at_a_time():
        for k in range(len(insts)):
            g = fbs.grid_build([yuv[k]], sig[0][k], sig[1][k], sig[2][k])
            fbs.bistochastize(g, BISTOCH_ITERS)
            fbs.solve(g, [t[k]], [c[k]], lam[k], PCG_ITERS, x=[x[k]])
            g.destroy()

    fbs.profile_enable(2)
    ms_b = time_steps(batched, steps, warmup, flush, stream)
    regions = fbs.profile_read()
    fbs.profile_enable(0)
    ms_s = time_steps(one_at_a_time, max(2, steps // 4), 1, flush, stream) if sequential else [0.0]
    npix = wl.n_pixels
    mb = dist.max(sum(ms_b) / len(ms_b))
    ms1 = dist.max(sum(ms_s) / len(ms_s)) or float("nan")
    bytes_iter = sum(V * (48 + 40 * i.channels) for V, i in zip(info["V"], insts))
    return {"workload": "64 images, sizes U{320..1920} x U{240..1080}, half depth (C=1), half "
                        "chroma (C=2, c=1 on 2% of pixels), sigma_xy in {8,16}, lambda in {32,128}",
            "preconditioner": precond,
            "pixels": npix, "vertices": int(sum(info["V"])),
            "batched_mpix_s": whole_job_mpix(dist.world, npix, mb), "batched_ms": mb,
            "tuning": tuning,
            "one_at_a_time_mpix_s": whole_job_mpix(dist.world, npix, ms1),
            "one_at_a_time_ms": ms1,
            "phase_share": {k: round(v[1] / max(1e-9, sum(w[1] for w in regions.values())), 4)
                            for k, v in regions.items() if v[0]},
            "pcg_roofline": dict(pcg_roofline(regions, 1, steps, bytes_iter, peak) or {},
                                 traffic=PCG_TRAFFIC_RATIO_BATCHED * bytes_iter
                                 if precond == "jacobi" else None,
                                 traffic_source="ncu of the first 16 images, scaled by "
                                                "traffic / algorithmic bytes"
                                 if precond == "jacobi" else None,
                                 bytes_basis="Jacobi PCG iteration, 48 + 40 C per vertex"
                                 if precond == "jacobi" else
                                 "Jacobi-byte equivalent: 48 + 40 C per vertex; the pyramid "
                                 "sweeps' bytes are not counted, their time is")}


def run_extra_robust(dist, flush, stream, peak, steps, warmup):
    """The robust solver on a 1400 x 1000 disparity target (5 % outliers, c = 0
    on a 10 % mask): grid, 2 bistochastisation sweeps, 10 IRLS x 25 PCG."""
    import torch
    from paper_1511_03296_gb300 import fbs, synth
    wl = synth.robust_1400x1000(seed=rank_seed(3, dist.rank))
    inst = wl.instances[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    yuv, t, c = dev(inst.yuv), dev(inst.t), dev(inst.c)
    x = torch.empty_like(t)
    info = {}

    def step():
        g = fbs.grid_build([yuv], inst.sigma_xy, inst.sigma_l, inst.sigma_uv)
        fbs.bistochastize(g, BISTOCH_ITERS)
        fbs.solve_robust(g, [t], [c], inst.lam, wl.sigma_gm, wl.irls_iters, PCG_ITERS, x=[x])
        info["V"] = g.vertex_counts[0]
        g.destroy()

    fbs.profile_enable(2)
    ms = time_steps(step, steps, warmup, flush, stream)
    regions = fbs.profile_read()
    fbs.profile_enable(0)
    m = dist.max(sum(ms) / len(ms))
    bytes_iter = algorithmic_bytes_per_pcg_iteration(info["V"], 1)
    return {"workload": "robust 1400x1000, C=1, sigma=(4,4,4), lambda=0.25, sigma_gm=1, "
                        "10 IRLS x 25 PCG iterations",
            "pixels": inst.n_pixels, "vertices": info["V"],
            "robust_mpix_s": whole_job_mpix(dist.world, inst.n_pixels, m), "ms_per_step": m,
            "phase_share": {k: round(v[1] / max(1e-9, sum(w[1] for w in regions.values())), 4)
                            for k, v in regions.items() if v[0]},
            "pcg_roofline": dict(pcg_roofline(regions, wl.irls_iters, steps, bytes_iter, peak)
                                 or {}, traffic=None)}


def run_extra_fwd_bwd(dist, flush, stream, peak, steps, warmup, n_images=16):
    """16 images 640x480, 21-channel softmax targets, through the library's
    autograd Function for a batch (BilateralSolveBatch): one forward solve of
    all images, the MSE loss against a label map, loss.backward() -- one
    backward solve of all images giving dL/dt and dL/dc."""
    import torch
    from paper_1511_03296_gb300 import fbs, synth
    wl = synth.segmentation_16(seed=rank_seed(5, dist.rank), n_images=n_images)
    insts = wl.instances
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    yuv = [dev(i.yuv) for i in insts]
    t = [dev(i.t).requires_grad_(True) for i in insts]
    c = [dev(i.c).requires_grad_(True) for i in insts]
    lab = [dev(i.label) for i in insts]
    x0 = [torch.empty_like(tt) for tt in t]
    sig = ([i.sigma_xy for i in insts], [i.sigma_l for i in insts], [i.sigma_uv for i in insts])
    lam = [i.lam for i in insts]
    numel = sum(tt.numel() for tt in t)
    info = {}
    tuning = tune(fbs, yuv, sig, [tt.detach() for tt in t], [cc.detach() for cc in c], lam, x0)

    def step():
        g = fbs.grid_build(yuv, *sig)
        fbs.apply_tuning(g, tuning)
        fbs.bistochastize(g, BISTOCH_ITERS)
        for tt, cc in zip(t, c):
            tt.grad = None
            cc.grad = None
        xs = fbs.bilateral_solve(t, c, g, lam, PCG_ITERS)
        loss = sum(((xx - ll) ** 2).sum() for xx, ll in zip(xs, lab)) / numel
        loss.backward()
        info["V"] = g.vertex_counts
        g.destroy()

    fbs.profile_enable(2)
    ms = time_steps(step, steps, warmup, flush, stream)
    regions = fbs.profile_read()
    fbs.profile_enable(0)
    m = dist.max(sum(ms) / len(ms))
    npix = wl.n_pixels
    bytes_iter = sum(V * (48 + 40 * i.channels) for V, i in zip(info["V"], insts))
    return {"workload": "16 images 640x480, C=21 softmax targets, c~U[0,1], sigma=(8,4,3), "
                        "lambda=128, forward + backward through the autograd Function "
                        "(2 x 25 PCG iterations)",
            "pixels": npix, "vertices": int(sum(info["V"])),
            "fwd_bwd_mpix_s": whole_job_mpix(dist.world, npix, m), "ms_per_step": m,
            "tuning": tuning,
            "phase_share": {k: round(v[1] / max(1e-9, sum(w[1] for w in regions.values())), 4)
                            for k, v in regions.items() if v[0]},
            "pcg_roofline": dict(pcg_roofline(regions, 2, steps, bytes_iter, peak) or {},
                                 traffic=None)}


def run_extra_lowrank(dist, flush, stream, steps, warmup, n_images=16, eps=0.01):
    """16 scenes 640x480 with 21-channel softmax targets of which 2-6 classes
    occur: the full 21-channel forward solve against the low-rank reduction
    (eps = 0.01), each with its grid build and bistochastisation."""
    import torch
    from paper_1511_03296_gb300 import fbs, synth
    wl = synth.segmentation_scenes_16(seed=rank_seed(6, dist.rank), n_images=n_images)
    insts = wl.instances
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    yuv = [dev(i.yuv) for i in insts]
    t = [dev(i.t) for i in insts]
    c = [dev(i.c) for i in insts]
    x_full = [torch.empty_like(tt) for tt in t]
    x_lr = [torch.empty_like(tt) for tt in t]
    sig = ([i.sigma_xy for i in insts], [i.sigma_l for i in insts], [i.sigma_uv for i in insts])
    lam = [i.lam for i in insts]
    info = {}

    def full():
        g = fbs.grid_build(yuv, *sig)
        fbs.bistochastize(g, BISTOCH_ITERS)
        fbs.solve(g, t, c, lam, PCG_ITERS, x=x_full)
        g.destroy()

    def lowrank():
        g = fbs.grid_build(yuv, *sig)
        fbs.bistochastize(g, BISTOCH_ITERS)
        info["ranks"] = fbs.solve_lowrank(g, t, c, lam, PCG_ITERS, eps, x=x_lr)
        g.destroy()

    ms_f = time_steps(full, steps, warmup, flush, stream)
    ms_l = time_steps(lowrank, steps, warmup, flush, stream)
    num = sum(float(((a - b) ** 2).sum()) for a, b in zip(x_lr, x_full))
    den = sum(float((b ** 2).sum()) for b in x_full)
    mf, ml = dist.max(sum(ms_f) / len(ms_f)), dist.max(sum(ms_l) / len(ms_l))
    npix = wl.n_pixels
    return {"workload": f"{n_images} scenes 640x480, C=21 softmax targets with 2-6 classes "
                        "present, c~U[0,1], sigma=(8,4,3), lambda=128, 25 PCG iterations",
            "pixels": npix, "eps": eps, "ranks": info["ranks"],
            "full_ms": mf, "full_mpix_s": whole_job_mpix(dist.world, npix, mf),
            "lowrank_ms": ml, "lowrank_mpix_s": whole_job_mpix(dist.world, npix, ml),
            "speedup": mf / ml, "rel_l2_vs_full": (num / den) ** 0.5}


def run_extra_dt(dist, flush, stream, steps, warmup):
    """The domain transform post-filter on the 1080p workload's 3-channel
    output (sigma_s = 32, sigma_r = 64, 3 iterations, the reference as the
    guide), timed alone: the paper includes it in every runtime."""
    import torch
    from paper_1511_03296_gb300 import fbs, synth
    inst = synth.plain_1080p(seed=rank_seed(2, dist.rank)).instances[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    guide, x0 = dev(inst.yuv), dev(inst.t)
    x = torch.empty_like(x0)

    def step():
        x.copy_(x0)
        fbs.domain_transform(guide, x, 32.0, 64.0, 3)

    def copy_only():
        x.copy_(x0)

    ms = time_steps(step, steps, warmup, flush, stream)
    mc = time_steps(copy_only, steps, warmup, flush, stream)
    m = dist.max(sum(ms) / len(ms) - sum(mc) / len(mc))
    return {"workload": "domain transform of a 1920x1080 3-channel image, sigma_s=32, "
                        "sigma_r=64, 3 iterations (rows: parallel affine scans per row; "
                        "columns: affine scans over 8 row segments per column)",
            "ms": m, "mpix_s": whole_job_mpix(dist.world, inst.n_pixels, m)}


def run_only(args, dist):
    """One extra workload alone (a profiling aid): prints its own JSON line."""
    import torch
    from paper_1511_03296_gb300 import build as fbs_build
    from paper_1511_03296_gb300 import fbs
    torch.cuda.set_device(dist.local_rank if torch.cuda.device_count() > 1 else 0)
    fbs_build.build()
    fbs.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    if args.only == "batched":
        out = run_extra_batched(dist, flush, stream, peak, args.steps, args.warmup,
                                n_images=args.images or 64, sequential=False,
                                precond=args.precond)
    elif args.only == "dt":
        out = run_extra_dt(dist, flush, stream, args.steps, args.warmup)
    elif args.only == "lowrank":
        out = run_extra_lowrank(dist, flush, stream, args.steps, args.warmup,
                                n_images=args.images or 16)
    else:
        out = run_extra_fwd_bwd(dist, flush, stream, peak, args.steps, args.warmup,
                                n_images=args.images or 16)
    if dist.rank == 0:
        print(json.dumps({"only": args.only, **out}), flush=True)


def e2e_pipelined(step, host_in, dev_like, steps, stream):
    """End to end through the public API, as a stream of steps: step i's
    inputs are copied from pinned host memory on a copy stream while step
    i - 1 computes, and its result is copied back while step i + 1
    computes (two sets of device buffers).  Every step still moves its own
    inputs in and its result out inside the timed region.  Returns (ms per
    step, the last step's host result)."""
    import torch
    sx = torch.cuda.Stream()
    sc = stream
    d_yuv, d_t, d_c, d_x = dev_like
    ins = [(torch.empty_like(d_yuv), torch.empty_like(d_t), torch.empty_like(d_c))
           for _ in range(2)]
    outs = [torch.empty_like(d_x) for _ in range(2)]
    hx = [torch.empty(tuple(d_x.shape), dtype=torch.float32).pin_memory() for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def copy_in(b, after=None):
        with torch.cuda.stream(sx):
            if after is not None:
                sx.wait_event(after)          # the step that last used these buffers
            for dst, src in zip(ins[b], host_in):
                dst.copy_(src, non_blocking=True)
            ev_in[b].record(sx)

    def run(k):
        copy_in(0)
        for i in range(k):
            b = i % 2
            if i + 1 < k:
                copy_in(b ^ 1, ev_done[b ^ 1] if i >= 1 else None)
            sc.wait_event(ev_in[b])
            if i >= 2:
                sc.wait_event(ev_out[b])      # step i - 2's result has been read back
            step(*ins[b], outs[b])
            ev_done[b].record(sc)
            with torch.cuda.stream(sx):
                sx.wait_event(ev_done[b])
                hx[b].copy_(outs[b], non_blocking=True)
                ev_out[b].record(sx)
        for b in range(min(k, 2)):
            sc.wait_event(ev_out[b])

    run(3)                                    # warm-up
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(sc)
    run(steps)
    t1.record(sc)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps, hx[(steps - 1) % 2]


def summary(line):
    """The headline figures of every workload, compact, last on the line."""
    frac = lambda rec: round(rec.get("pcg_roofline", {}).get("frac", float("nan")), 3)
    b, f, r = line["batched"], line["fwd_bwd"], line["robust"]
    h, lr = line["batched_hierarchical"], line["lowrank"]
    return {
        "1080p_mpix_s": round(line["value"], 1),
        "1080p_pcg_frac": round(line["roofline"].get("frac", float("nan")), 3),
        "batched_mpix_s": round(b["batched_mpix_s"], 1),
        "one_at_a_time_mpix_s": round(b["one_at_a_time_mpix_s"], 1),
        "batched_speedup": round(b["batched_mpix_s"] / b["one_at_a_time_mpix_s"], 2),
        "batched_pcg_frac": frac(b),
        "fwd_bwd_mpix_s": round(f["fwd_bwd_mpix_s"], 1), "fwd_bwd_pcg_frac": frac(f),
        "robust_mpix_s": round(r["robust_mpix_s"], 1), "robust_pcg_frac": frac(r),
        "hierarchical_batched_mpix_s": round(h["batched_mpix_s"], 1),
        "lowrank_speedup": round(lr["speedup"], 2),
        "domain_transform_mpix_s": round(line["domain_transform"]["mpix_s"], 1),
        "cpu_oracle_1core_mpix_s": round(line.get("cpu_baseline", {}).get("value", float("nan")), 2),
    }


def run_ours(args, dist):
    import torch

    from paper_1511_03296_gb300 import build as fbs_build
    from paper_1511_03296_gb300 import fbs, synth

    dev = dist.local_rank if torch.cuda.device_count() > 1 else 0
    torch.cuda.set_device(dev)
    fbs_build.build()
    fbs.load()
    inst = synth.plain_1080p(seed=rank_seed(2, dist.rank)).instances[0]
    stream = torch.cuda.current_stream()
    d_yuv = torch.from_numpy(inst.yuv).cuda()
    d_t = torch.from_numpy(inst.t).cuda()
    d_c = torch.from_numpy(inst.c).cuda()
    d_x = torch.empty_like(d_t)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    V_holder = {}

    tuning = tune(fbs, [d_yuv], (inst.sigma_xy, inst.sigma_l, inst.sigma_uv), [d_t], [d_c],
                  inst.lam, [d_x])

    def step(yuv, t, c, x):
        g = fbs.grid_build([yuv], inst.sigma_xy, inst.sigma_l, inst.sigma_uv)
        fbs.apply_tuning(g, tuning)
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
    value = whole_job_mpix(dist.world, inst.n_pixels, ms)
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

    def e2e_step():
        e_yuv.copy_(h_yuv, non_blocking=True)
        e_t.copy_(h_t, non_blocking=True)
        e_c.copy_(h_c, non_blocking=True)
        step(e_yuv, e_t, e_c, e_x)
        h_x.copy_(e_x, non_blocking=True)

    e2e = time_steps(e2e_step, max(3, min(args.steps, 20)), 2, flush, stream)
    e2e_serial_ms = dist.max(sum(e2e) / len(e2e))
    assert np.allclose(h_x.numpy(), d_x.cpu().numpy())
    e2e_ms, hx_last = e2e_pipelined(step, (h_yuv, h_t, h_c), (d_yuv, d_t, d_c, d_x),
                                    max(6, min(args.steps, 40)), stream)
    e2e_ms = dist.max(e2e_ms)
    assert np.allclose(hx_last.numpy(), d_x.cpu().numpy())
    h2d = inst.yuv.nbytes + inst.t.nbytes + inst.c.nbytes
    d2h = inst.t.nbytes

    # ---- roofline: the PCG iteration (both phases), timed as a region
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    bytes_iter = algorithmic_bytes_per_pcg_iteration(V, inst.channels)
    roof = pcg_roofline(regions, 1, args.steps, bytes_iter, peak)
    resident = tuning.get("pcg_launch") == fbs.PCG_PERSISTENT
    single = tuning.get("pcg_form") == fbs.PCG_FORM_SINGLE
    region_share = {k: round(t / max(1e-9, sum(tt for _, tt in regions.values())), 4)
                    for k, (n, t) in regions.items() if n}

    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(),
        "details": {"pixels_per_gpu": inst.n_pixels, "vertices": V, "channels": inst.channels,
                    "parallelism": f"replicas x{dist.world}",
                    "precision": "FP32 vectors, FP64-accurate CG dot products, FP64 "
                                 "bistochastisation",
                    "tuning": tuning, "phase_share": None, "kernel_share": None},
        "clocks": clk.summary(),
        "e2e": {"value": whole_job_mpix(dist.world, inst.n_pixels, e2e_ms), "unit": "Mpix/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms,
                "pipelining": "each step copies its inputs from pinned host memory and its "
                              "result back on a second stream, overlapping the neighbouring "
                              "steps' compute; no L2 flush",
                "serial": {"value": whole_job_mpix(dist.world, inst.n_pixels, e2e_serial_ms),
                           "ms_per_step": e2e_serial_ms,
                           "note": "copies and compute one after another, L2 flushed between "
                                   "steps outside the events"}},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": dict(roof or {}, kernel="pcg iteration" + (
                             ", resident loop of the single-reduction form" if resident and single
                             else ", resident loop" if resident else
                             ", single-reduction form, per-iteration launches" if single else
                             " (both CG phases), per-phase launches"),
                         traffic=(PCG_TRAFFIC_1080P_RESIDENT_SINGLE if resident and single else
                                  PCG_TRAFFIC_1080P_RESIDENT if resident else
                                  None if single else PCG_TRAFFIC_1080P),
                         traffic_source=("ncu, one 25-iteration launch of the resident loop, "
                                         "per iteration" if resident else
                                         "ncu, cold caches, one iteration (apply + update)"),
                         peak_source="measured" if peaks else "fallback",
                         note="working set L2-resident at this size; see batched / fwd_bwd "
                              "for the HBM-bound sizes"),
    }
    line["details"]["phase_share"] = region_share
    line["details"]["kernel_share"] = shares
    if not args.no_extra:
        xs = max(3, min(args.steps // 10, 20))
        extra = {
            "batched": run_extra_batched(dist, flush, stream, peak, xs, 3),
            "fwd_bwd": run_extra_fwd_bwd(dist, flush, stream, peak, xs, 3),
            "robust": run_extra_robust(dist, flush, stream, peak, max(3, xs // 2), 3),
            "batched_hierarchical": run_extra_batched(dist, flush, stream, peak,
                                                      max(3, xs // 2), 3, sequential=False,
                                                      precond="hierarchical"),
            "lowrank": run_extra_lowrank(dist, flush, stream, max(3, xs // 2), 3),
            "domain_transform": run_extra_dt(dist, flush, stream, xs, 3),
        }
        # long per-workload records (phase shares, tuning) go to details, so the
        # results themselves stay near the end of the line
        for name, rec in extra.items():
            line["details"][name] = {k: rec.pop(k) for k in ("phase_share", "tuning") if k in rec}
        line.update(extra)
    if dist.rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(synth.plain_1080p().instances[0], args.cpu_seconds)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.cpu_seconds / 2)
    if not args.no_extra:
        line["summary"] = summary(line)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    global TUNE_CACHE
    args = parse_args()
    TUNE_CACHE = args.tune_cache
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.only:
            run_only(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
