#!/usr/bin/env python
"""Throughput of the coarse-to-fine visual-hull path on GB300.

One step = one batched pass of the whole path over a batch of consecutive
volleyball-shaped frames (16 cameras 1920x1080, 400x220x80 coarse voxels of
5 cm, 1 cm fine voxels in the ROIs, 10 bisection steps): silhouette packing
from device-resident masks, reconstruction of all frames in one
fvv_reconstruct call (coarse hull, CCL + Eq. (1) filter + ROIs, fine hull,
marching cubes with bisection, depth images) and one fvv_colour call.

Printed (rank 0, one JSON line): batched frames/s (`value`), voxel-camera
tests/s, the plain per-frame path on the same GPU (frames/s and p50/p99
frame latency), per-stage times, the roofline of the dominant kernel, the
CPU oracle timed on the host cores (`cpu_baseline`), the end-to-end number
through the public API with host buffers (`e2e`), clocks and launch count.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--frames F]
    python bench.py --impl reference ...    # the CPU oracle as the reference arm

Multi-GPU: frames are independent, so N GPUs run N replicas on different
frames (no collective on the data path); `value` is the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s & G voxel-camera tests/s on 1 GB300, batched vs plain; p50/p99 frame latency"
CONFIG = "volleyball"
WORKLOAD = ("volleyball-shaped frames: 16 cameras 1920x1080 (f=1800), 12 players + ball, volume 20x11x4 m, "
            "coarse 5 cm (400x220x80), fine 1 cm in ROIs, 10 bisection steps, 0.1% silhouette flips")
# FP32 floating-point operations of one camera test by definition: x', y', w'
# (9 fused multiply-adds, 2 operations each), u and v (2 divisions), two floors.
FLOPS_PER_TEST = 22
# FP32 floating-point operations of one (triangle, camera) pair of the depth
# images by definition: three vertex projections (27 fused multiply-adds), the
# squared centroid distance (3 subtractions, 3 multiplications, 2 additions),
# u and v of the three vertices (6 divisions).  The per-pixel edge tests are
# not counted (they depend on how many pixel centres a triangle covers).
FLOPS_PER_PAIR = 68
# FP32 lanes per SM (Blackwell): the nominal FP32 peak is the SM count (queried
# at run time) x 128 lanes x 2 operations per fused multiply-add x the maximum
# SM clock; the roofline's `peak` is the rate fvv_probe_fma measures instead.
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per frame of each large kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of a 4-frame launch of
# the current kernels, scaled to a launch by its frame count.  None for a
# kernel changed since that capture.
DRAM_BYTES_PER_FRAME = {"k_fine_carve": 7.28576e6 / 4, "k_bisect": 17.22496e6 / 4,
                        "k_coarse_carve": (4.332032e6 + 5120) / 4,
                        "k_zbuffer<1>": None, "k_zbuffer<2>": None,
                        "k_zbuffer<4>": (179.26144e6 + 9.915392e6) / 4}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--frames", type=int, default=64, help="frames per batched step")
    ap.add_argument("--plain-frames", type=int, default=16)
    ap.add_argument("--cpu-frames", type=int, default=4, help="frames in the CPU-oracle sample")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving leg (4 rigs at 30 Hz each; 0 skips it)")
    ap.add_argument("--serve-pool", type=int, default=8, help="frames per rig in the serving pool")
    ap.add_argument("--serve-masks", choices=("in_place", "copies"), default="in_place",
                    help="serving: pinned masks read in place by the packing kernel, or copied by the copy engines")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--tuning-cache", default=None,
                    help="JSON file of tuned launch shapes: reuse the entry for this GPU and workload, "
                         "or autotune and add it")
    ap.add_argument("--zbuffer-cams", type=int, choices=(1, 2, 4), default=None,
                    help="cameras per z-buffer block, set after any tuning (for profiling one variant)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--study", choices=("surface", "fig10", "table1", "view"), default=None,
                    help="instead of the benchmark line: surface-rule errors (Sec. II-C), the coarse/fine "
                         "voxel-size sweeps of Fig. 10, the Table I capture shapes, or novel-view rendering")
    ap.add_argument("--study-frames", type=int, default=4)
    ap.add_argument("--study-image", default=None, help="--study view: write the first view here (PPM)")
    return ap.parse_args()


def first_frame(rank, frames_per_rank):
    """Replicas only: rank r reconstructs its own consecutive frames, disjoint
    from every other rank's (frames are independent; no data-path collective)."""
    return rank * frames_per_rank


def max_over_ranks(x, world, device):
    """The slowest rank's time (the job's time); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, frames_per_rank, seconds):
    """Whole-job throughput: the frames all ranks processed over the job's time."""
    return world * frames_per_rank / seconds


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows, self.proc, self.gpu = [], None, gpu_index

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu is not None:
                cmd[1:1] = ["-i", str(self.gpu)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return self.summary()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ inputs

def make_batch(n_frames, offset, device):
    import torch
    from synth import make_frame, make_rig
    rig = make_rig(CONFIG)
    masks, rgbs, vps = [], [], []
    for i in range(n_frames):
        _, fr = make_frame(CONFIG, offset + i, device=device, rig=rig)
        masks.append(fr.masks)
        rgbs.append(fr.rgb)
        vps.append(fr.viewpoint)
    return rig, torch.stack(masks), torch.stack(rgbs), np.stack(vps)


# ------------------------------------------------------------------ CPU oracle

def oracle_frames_per_s(rig, masks_cpu, rgb_cpu, vps):
    """The oracle as it stands (single thread), full path per frame."""
    from oracle import Oracle
    o = Oracle(rig)
    t0 = time.perf_counter()
    tests = 0
    for m, c, vp in zip(masks_cpu, rgb_cpu, vps):
        ref = o.reconstruct(m)
        d = o.depth(ref.verts, ref.tris)
        o.colour(c, vp, d, ref.verts)
        tests += ref.tests
    dt = time.perf_counter() - t0
    return len(masks_cpu) / dt, tests / dt, dt


def _oracle_worker(job):
    """One frame of the full oracle path in a worker process (frame-parallel
    CPU baseline); inputs are read from .npy files written by the parent."""
    path, i = job
    from oracle import Oracle
    from synth import make_rig
    masks = np.load(os.path.join(path, "masks.npy"), mmap_mode="r")
    rgb = np.load(os.path.join(path, "rgb.npy"), mmap_mode="r")
    vps = np.load(os.path.join(path, "vps.npy"))
    o = Oracle(make_rig(CONFIG))
    j = i % len(masks)
    t0 = time.perf_counter()
    ref = o.reconstruct(np.asarray(masks[j]))
    d = o.depth(ref.verts, ref.tris)
    o.colour(np.asarray(rgb[j]), vps[j], d, ref.verts)
    return time.perf_counter() - t0, ref.tests


def oracle_all_cores(masks_cpu, rgb_cpu, vps):
    """The same oracle as independent processes, one frame per host core
    (frames are independent, so this needs no change to the oracle).
    Returns (frames/s, processes, seconds)."""
    import multiprocessing as mp
    import shutil
    import tempfile
    from oracle import build as build_oracle
    build_oracle()
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    tmp = tempfile.mkdtemp(prefix="fvv_oracle_")
    try:
        np.save(os.path.join(tmp, "masks.npy"), masks_cpu)
        np.save(os.path.join(tmp, "rgb.npy"), rgb_cpu)
        np.save(os.path.join(tmp, "vps.npy"), np.asarray(vps))
        with mp.get_context("spawn").Pool(n) as pool:
            pool.map(_oracle_worker, [(tmp, i) for i in range(n)], chunksize=1)      # imports, page-in
            t0 = time.perf_counter()
            pool.map(_oracle_worker, [(tmp, i) for i in range(n)], chunksize=1)
            dt = time.perf_counter() - t0
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return n / dt, n, dt


def oracle_configs_single_core(frames):
    """Per-frame milliseconds of the single-threaded oracle (full path) on
    each scene configuration: {config: (masks list, rgb list, viewpoints)}."""
    from oracle import Oracle
    from synth import make_rig
    out = {}
    for cfg, (ms, cs, vps) in frames.items():
        o = Oracle(make_rig(cfg))
        t0 = time.perf_counter()
        tests = 0
        for m, c, vp in zip(ms, cs, vps):
            ref = o.reconstruct(m)
            d = o.depth(ref.verts, ref.tris)
            o.colour(c, vp, d, ref.verts)
            tests += ref.tests
        dt = time.perf_counter() - t0
        out[cfg] = {"ms_per_frame": 1000 * dt / len(ms), "frames": len(ms), "tests_per_frame": tests / len(ms)}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from synth import make_frame, make_rig
    rig = make_rig(CONFIG)
    n = args.warmup + args.steps
    frames = [make_frame(CONFIG, i, rig=rig)[1] for i in range(n)]
    times, tests = [], 0
    for i, fr in enumerate(frames):
        fps, tps, dt = oracle_frames_per_s(rig, [fr.masks.numpy()], [fr.rgb.numpy()], [fr.viewpoint])
        if i >= args.warmup:
            times.append(dt)
            tests += tps * dt
    total = sum(times)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "gtests_per_s": tests / total / 1e9,
            "config": {"workload": WORKLOAD, "frames_per_step": 1, "parallelism": "single host thread"},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed volleyball-shaped frames, one per step, full path "
                                       "(reconstruct + depth + colour), single thread"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving

SERVE_RIGS = (("volleyball", 1000), ("volleyball", 2000), ("judo", 0), ("hd720", 0))   # (config, first frame)


def run_serving(args, rank):
    """Requests from four rigs (two volleyball-shaped 16x1080p with one
    calibration, one judo-shaped 12x4K, one 8x720p), Poisson arrivals at 30 Hz
    per rig, admitted under a 40 GB memory budget with slot capacities fitted
    to each rig's frames, and served with continuous batching (the two
    volleyball rigs share batches).  Run once at the offered rate and once
    with all arrivals compressed 1000x (saturation)."""
    import torch
    from paper_1903_11785_gb300.serve import RigPool, Server, poisson_schedule, summarize, summarize_per_rig
    from synth import make_frame, make_rig
    pools = []
    for cfg, first in SERVE_RIGS:
        rig = make_rig(cfg)
        frames = [make_frame(cfg, first + rank * 100 + i, device="cuda", rig=rig)[1] for i in range(args.serve_pool)]
        pools.append(RigPool(scene_rig=rig, masks=[f.masks.cpu().pin_memory() for f in frames],
                             rgb=[f.rgb.cpu().pin_memory() for f in frames],
                             viewpoints=np.stack([f.viewpoint for f in frames])))
        del frames
        torch.cuda.empty_cache()
    srv = Server(pools, budget_bytes=40 << 30, mask_copies=args.serve_masks == "copies")
    try:
        out = {"rigs": [c for c, _ in SERVE_RIGS], "offered_fps": 4 * 30.0, "masks": args.serve_masks}
        out.update(srv.describe())
        warm = poisson_schedule(len(pools), 30.0, 40, seed=7, pool_sizes=[args.serve_pool] * len(pools))
        srv.run(warm, time_scale=1000.0)
        reqs = poisson_schedule(len(pools), 30.0, args.serve_requests, seed=1903,
                                pool_sizes=[args.serve_pool] * len(pools))
        done = srv.run(reqs)
        out.update(summarize(done))
        out["per_rig"] = summarize_per_rig(done, len(pools))
        reqs = poisson_schedule(len(pools), 30.0, args.serve_requests, seed=1904,
                                pool_sizes=[args.serve_pool] * len(pools))
        sat = srv.run(reqs, time_scale=1000.0)
        out["saturated"] = summarize(sat, time_scale=1000.0)
        out["saturated"]["per_rig"] = summarize_per_rig(sat, len(pools), time_scale=1000.0)
        return out
    finally:
        srv.close()


# ------------------------------------------------------------------ GPU path

def measure_l2(fvv, torch, sms):
    """L2 peaks for the memory side of the hull tests' roofline: a coalesced
    read of a 32 MiB buffer and random 32-bit gathers from a 4 MiB one (the
    size of one frame's packed silhouettes), both L2-resident, both through
    the library's fvv_probe_l2, timed by events on the launching stream."""
    blocks, threads = sms * 8, 256
    out = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(190311785)
    rd = torch.randint(-2 ** 31, 2 ** 31 - 1, (8 << 20,), dtype=torch.int32, device="cuda", generator=g)
    ga = torch.randint(-2 ** 31, 2 ** 31 - 1, (1 << 20,), dtype=torch.int32, device="cuda", generator=g)
    stream = torch.cuda.current_stream()
    res = {}
    for name, mode, buf, reps in (("read", 0, rd, 64), ("gather", 1, ga, 1024)):
        for _ in range(3):
            fvv.fvv_probe_l2(mode, buf, reps, out, blocks, threads)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 10
        a.record(stream)
        for _ in range(n):
            fvv.fvv_probe_l2(mode, buf, reps, out, blocks, threads)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1000.0 / n
        units = buf.numel() * 4 * reps if mode == 0 else blocks * threads * reps
        res[name] = units / sec
    return {"read_GBps": res["read"] / 1e9, "gather_Gwords_per_s": res["gather"] / 1e9,
            "gather_sector_GBps": res["gather"] * 32 / 1e9,
            "how": "fvv_probe_l2: ld.global.cg coalesced read of 32 MiB x64, and random 32-bit gathers (1024 per "
                   f"thread, {blocks}x{threads} threads) from 4 MiB; mean of 10 launches after 3"}


def measure_alu(fvv, torch, sms):
    """FP32 ceiling: fvv_probe_fma, 16 independent fused multiply-add chains
    per thread on sms x 8 blocks of 256 threads, timed by events on the
    launching stream (mean of 10 launches after 3)."""
    blocks, threads, reps = sms * 8, 256, 8192
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    for _ in range(3):
        fvv.fvv_probe_fma(reps, 1.0, 0.5, out, blocks, threads)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    a.record(stream)
    for _ in range(n):
        fvv.fvv_probe_fma(reps, 1.0, 0.5, out, blocks, threads)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1000.0 / n
    return {"tflops": blocks * threads * reps * 16 * 2 / sec / 1e12,
            "how": f"fvv_probe_fma: {blocks}x{threads} threads, 16 fused multiply-add chains of {reps} steps each; "
                   "mean of 10 launches after 3"}


def max_sm_clock_mhz(gpu_index):
    try:
        cmd = ["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"]
        if gpu_index is not None:
            cmd[1:1] = ["-i", str(gpu_index)]
        return float(subprocess.check_output(cmd, text=True, timeout=20).split()[0])
    except Exception:
        return None


def fp64_flips(rig, masks):
    """Sec. II-B: voxels whose occupancy differs between the binary32 oracle
    (the parity target) and the binary64 one, on one frame: over the coarse
    grid, and over the fine samples of the ROIs whose grown box is the same in
    both precisions."""
    from oracle import Oracle
    a = Oracle(rig, "f32").reconstruct(masks)
    b = Oracle(rig, "f64").reconstruct(masks)
    same, fine_n, fine_flips = 0, 0, 0
    boxes_b = {(r.gmin, r.gmax): k for k, r in enumerate(b.rois)}
    for k, r in enumerate(a.rois):
        kb = boxes_b.get((r.gmin, r.gmax))
        if kb is not None and a.fine[k].shape == b.fine[kb].shape:
            same += 1
            fine_n += a.fine[k].size
            fine_flips += int((a.fine[k] != b.fine[kb]).sum())
    return {"frames": 1, "coarse_voxels": int(a.coarse.size), "coarse_flips": int((a.coarse != b.coarse).sum()),
            "coarse_on_f32": int(a.coarse.sum()), "rois_f32": len(a.rois), "rois_f64": len(b.rois),
            "rois_same_box": same, "fine_samples_compared": fine_n, "fine_flips": fine_flips}


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1903_11785_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    from paper_1903_11785_gb300 import fvv

    F = args.frames
    rig, masks, rgb, vps = make_batch(F, first_frame(rank, F), "cuda")
    mask_bytes, rgb_bytes = masks.numel(), rgb.numel()
    N, H, W = masks.shape[1:]
    r = fvv.Rig(rig, max_slots=F, host_staging=0 if args.no_e2e else 2)   # 2: mask staging only
    slots = list(range(F))
    stream = torch.cuda.current_stream()

    def step():
        r.upload_silhouettes_batch(slots, masks)
        r.reconstruct(slots)
        r.colour(slots, rgb, vps)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tuning = None
    if not args.no_tune:
        if args.tuning_cache:               # shapes an earlier run picked for this GPU and workload
            from paper_1903_11785_gb300 import tuning_cache
            tuning, cached = tuning_cache.tuned(r, rig, slots, args.tuning_cache, torch.cuda.get_device_name(local))
            tuning = dict(tuning, from_cache=cached)
        else:
            tuning = r.autotune(slots)      # launch shapes picked on this batch
        step()
        torch.cuda.synchronize()
    if args.zbuffer_cams is not None:
        tuning = dict(r.get_tuning(), zbuffer_cams=args.zbuffer_cams)
        r.set_tuning(tuning)
        step()
        torch.cuda.synchronize()
    counts = [r.counts(i) for i in slots]
    tests = sum(c["tests_coarse"] + c["tests_fine"] + c["tests_bisect"] for c in counts)
    tsum = {k: sum(c[k] for c in counts) for k in ("tests_coarse", "tests_fine", "tests_bisect", "n_verts",
                                                    "n_tris", "lookups_fine", "lookups_bisect")}

    # ---- timed region (batched)
    gpu_index = None
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd and cvd.split(",")[0].strip().isdigit():
        gpu_index = int(cvd.split(",")[local].strip()) if len(cvd.split(",")) > local else None
    # the whole step (one packing launch, the reconstruction's launches, the
    # colour launches) captured once as a CUDA graph and replayed per step;
    # every call only enqueues work on the current stream, so it captures
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index).start()
    time.sleep(0.4)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, "cuda")
    value = job_rate(world, F, ms / 1000.0)
    # per-stage device times: the same step run eagerly with stage events, after
    # the timed region (untimed); these are the Table II buckets
    r.set_timing(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    stages = r.timing()
    r.set_timing(False)
    eager_ms = sum(v[0] for v in stages.values()) / args.steps

    # ---- plain path: one frame per call (slot 0, reconstruction replayed as a
    # CUDA graph on a side stream), per-frame latency by events
    lat = []
    P = min(args.plain_frames, F)
    r.set_graphs(True)
    ps = torch.cuda.Stream()
    with torch.cuda.stream(ps):
        for i in range(P + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ps)
            r.upload_silhouettes(0, masks[i % F])
            r.reconstruct([0])
            r.colour([0], rgb[i % F:i % F + 1], vps[i % F:i % F + 1])
            b.record(ps)
            b.synchronize()
            if i >= 2:
                lat.append(a.elapsed_time(b))
    r.set_graphs(False)
    torch.cuda.synchronize()
    plain_fps = len(lat) / (sum(lat) / 1000.0)

    # ---- per-stage times and the rooflines of the four large kernels; the
    # `roofline` object is the one of the stage that takes longest
    per_step = {k: v[0] / args.steps for k, v in stages.items()}
    launches = {k: v[1] / args.steps for k, v in stages.items()}
    units = {  # algorithmic units per step, and FP32 operations per unit
        "coarse": (tsum["tests_coarse"], FLOPS_PER_TEST, "camera tests"),
        "fine": (tsum["tests_fine"], FLOPS_PER_TEST, "camera tests"),
        "bisect": (tsum["tests_bisect"] + tsum["n_verts"] * 6 * (rig.bisect_steps + 1) / FLOPS_PER_TEST,
                   FLOPS_PER_TEST, "camera tests (+ midpoints as test equivalents)"),
        "depth": (tsum["n_tris"] * rig.n_cams, FLOPS_PER_PAIR, "(triangle, camera) pairs"),
    }
    zc = r.get_tuning()["zbuffer_cams"]
    kernel_of = {"coarse": "k_coarse_carve", "fine": "k_fine_carve", "bisect": "k_bisect",
                 "depth": f"k_zbuffer<{zc}>"}

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu = measure_alu(fvv, torch, sms)
    max_mhz = max_sm_clock_mhz(gpu_index)
    alu["nominal_tflops"] = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12 if max_mhz else None
    alu["nominal_from"] = f"{sms} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz} MHz (max SM clock)"

    def alu_roofline(k):
        n_units, fpu, what = units[k]
        launch_ms = per_step[k] / max(launches[k], 1)
        achieved = n_units * fpu / max(launches[k], 1) / (launch_ms / 1000.0) / 1e12
        traffic = DRAM_BYTES_PER_FRAME.get(kernel_of[k])
        return {"bound": "alu", "kernel": kernel_of[k], "achieved": achieved, "peak": alu["tflops"],
                "unit": "TFLOP/s", "frac": achieved / alu["tflops"],
                "traffic": traffic * F if traffic is not None else None,
                "peak_source": "measured (fvv_probe_fma)", "launch_ms": launch_ms,
                "units_per_launch": n_units / max(launches[k], 1), "unit_of_work": what, "flops_per_unit": fpu}
    rooflines = {k: alu_roofline(k) for k in units}
    roofline = rooflines[max(units, key=lambda k: per_step[k])]
    dom = max(("coarse", "fine", "bisect"), key=lambda k: per_step[k])   # the largest hull kernel
    launch_ms = rooflines[dom]["launch_ms"]

    # ---- memory side: the silhouette words the dominant kernel actually
    # read (the fine hull and the bisection settle most tests for a whole tile
    # or edge without a read; the coarse hull reads one word per test),
    # against the measured L2 random-gather rate
    l2 = measure_l2(fvv, torch, sms)
    reads_dom = {"coarse": tsum["tests_coarse"], "fine": tsum["lookups_fine"], "bisect": tsum["lookups_bisect"]}[dom]
    gathers = reads_dom / max(launches[dom], 1) / (launch_ms / 1000.0)
    tests_rate = tsum["tests_" + dom] / max(launches[dom], 1) / (launch_ms / 1000.0)
    # the whole step's camera tests (a1, a5, a7) at the algorithmic 4 bytes
    # (one 32-bit silhouette word) and at one 32-byte L2 sector per test,
    # against the measured coalesced L2 read rate
    step_tests_per_s = tests / (ms / 1000.0) / world
    l2_roofline = {"bound": "l2", "kernel": kernel_of[dom], "achieved": gathers / 1e9,
                   "peak": l2["gather_Gwords_per_s"], "unit": "G silhouette-word gathers/s",
                   "frac": gathers / 1e9 / l2["gather_Gwords_per_s"],
                   "definition": "silhouette words the kernel actually reads per second over the measured random "
                                 "32-bit gather rate of L2: the utilisation of the L2 path the hull tests use, "
                                 "the reading taken for a 50% L2-roofline target",
                   "algorithmic_tests_G_per_s": tests_rate / 1e9,
                   "reads_per_test": reads_dom / max(tsum["tests_" + dom], 1),
                   "step_algorithmic": {"tests_G_per_s": step_tests_per_s / 1e9,
                                        "frac_at_4B": step_tests_per_s * 4 / (l2["read_GBps"] * 1e9),
                                        "frac_at_32B_sector": step_tests_per_s * 32 / (l2["read_GBps"] * 1e9),
                                        "peak_read_GBps": l2["read_GBps"]},
                   "probe": l2}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        masks_h = masks.cpu().pin_memory()
        rgb_h = rgb.cpu().pin_memory()
        step()                      # the plain path reused slot 0: put the batch back before sizing outputs
        torch.cuda.synchronize()
        cnt = [r.counts(i) for i in slots]
        outs = [dict(verts=torch.empty((c["n_verts"], 3), dtype=torch.float32).pin_memory(),
                     tris=torch.empty((c["n_tris"], 3), dtype=torch.int32).pin_memory(),
                     rgb=torch.empty((c["n_verts"], 3), dtype=torch.uint8).pin_memory(),
                     cam=torch.empty((c["n_verts"],), dtype=torch.int32).pin_memory()) for c in cnt]
        # masks and RGB stay in pinned host memory: the masks are copied to
        # the slots' staging by the copy engines (which need no SMs, so the
        # copies overlap other groups' kernels), the colour kernel reads only
        # the RGB pixels it needs (FVV_MAPPED_HOST)
        h2d = int(masks_h.numel())
        d2h = int(sum(sum(t.numel() * t.element_size() for t in o.values()) for o in outs))

        # groups of frames on three rotating streams, so that one group's
        # copies (copy engines) overlap the other groups' kernels (calls on
        # disjoint slots may run concurrently)
        E2E_GROUP, E2E_STREAMS = 8, 3
        e2e_streams = [torch.cuda.Stream() for _ in range(E2E_STREAMS)]
        groups = [slots[g:g + E2E_GROUP] for g in range(0, F, E2E_GROUP)]

        def e2e_step():
            # reading a group back waits for its work (it reads the counts),
            # so the next group is queued before the previous one is read back
            def compute(grp, st):
                with torch.cuda.stream(st):
                    r.upload_silhouettes_batch(grp, masks_h[grp[0]:grp[-1] + 1], stream=st)
                    r.reconstruct(grp, stream=st)
                    r.colour(grp, rgb_h[grp[0]:grp[-1] + 1], vps[grp[0]:grp[-1] + 1], stream=st, in_place=True)

            def read_back(grp, st):
                # one wait for the group's counts, then its copies (fvv_get_results_batch)
                fvv.fvv_get_results_batch(r.ptr, grp, [outs[i] for i in grp], stream=st)
            pending = []
            for gi, grp in enumerate(groups):
                st = e2e_streams[gi % E2E_STREAMS]
                compute(grp, st)
                pending.append((grp, st))
                if len(pending) == E2E_STREAMS:
                    read_back(*pending.pop(0))
            for grp, st in pending:
                read_back(grp, st)
            torch.cuda.synchronize()

        for _ in range(3):
            e2e_step()
        ok = all(torch.equal(o["verts"], r.results(i)["verts"].cpu()) for i, o in zip(slots[:2], outs[:2]))
        ks = max(30, args.steps)   # single slow steps (35-55 ms) occur; more steps dilute them
        torch.cuda.synchronize()
        per = []
        t0 = time.perf_counter()
        for _ in range(ks):
            t1 = time.perf_counter()
            e2e_step()
            per.append(time.perf_counter() - t1)
        dt = (time.perf_counter() - t0) / ks
        dt = max_over_ranks(dt, world, "cuda")
        e2e = {"value": job_rate(world, F, dt), "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": ks, "step_ms": {"mean": 1000 * dt, "median": 1000 * float(np.median(per)),
                                        "min": 1000 * min(per), "max": 1000 * max(per)},
               "results_match_device": bool(ok),
               "pipelining": f"{len(groups)} groups of {E2E_GROUP} frames on {E2E_STREAMS} rotating streams, "
                             f"each group read back while the next {E2E_STREAMS - 1} run",
               "inputs": f"{masks_h.numel() / 1e9:.2f} GB of pinned host masks per step copied by the copy engines "
                         f"into the slots' staging; {rgb_h.numel() / 1e9:.2f} GB of pinned host RGB read in place "
                         "by the colour kernel (only the pixels it needs cross the host link)"}

    S = min(args.cpu_frames, F)
    cpu_sample = (masks[:S].cpu().numpy(), rgb[:S].cpu().numpy(), vps[:S])
    cfg_frames = {}
    if rank == 0 and world == 1 and not args.no_cpu:
        from synth import make_frame
        from synth import make_rig as _make_rig
        for cfg, n_cfg in (("tiny", 4), ("judo", 1), ("hd720", 2)):
            rg = _make_rig(cfg)
            frs = [make_frame(cfg, i, device="cuda", rig=rg)[1] for i in range(n_cfg)]
            cfg_frames[cfg] = ([f.masks.cpu().numpy() for f in frs], [f.rgb.cpu().numpy() for f in frs],
                               [f.viewpoint for f in frs])
            del frs

    # ---- serving: 4 rigs, Poisson arrivals, continuous batching under a memory budget
    serving = None
    if args.serve_requests > 0:
        r.close()
        del masks, rgb
        torch.cuda.empty_cache()
        serving = run_serving(args, rank)
        r = None

    # ---- CPU oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    flips = None
    if rank == 0 and world == 1 and not args.no_cpu:
        S = min(args.cpu_frames, F)
        fps, tps, dt = oracle_frames_per_s(rig, *cpu_sample)
        cpu = {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle", "gtests_per_s": tps / 1e9,
               "sample": f"{S} volleyball-shaped frames of the batch, full path (reconstruct + depth + colour), "
                         f"single thread, {dt:.1f} s"}
        pfps, nproc, pdt = oracle_all_cores(*cpu_sample)
        cpu["all_cores"] = {"value": pfps, "unit": "frames/s", "cores": nproc, "kind": "oracle",
                            "sample": f"{nproc} processes, one volleyball-shaped frame each (cycling over the "
                                      f"{S} sampled frames), full path, {pdt:.1f} s"}
        per_cfg = oracle_configs_single_core(cfg_frames)
        per_cfg["volleyball"] = {"ms_per_frame": 1000 * dt / S, "frames": S, "tests_per_frame": tps * dt / S}
        cpu["single_core_per_config"] = per_cfg
        flips = fp64_flips(rig, cpu_sample[0][0])

    # kernels per step: one packing launch per 128 frames; the reconstruction's 15
    # (info reset; coarse hull; 5 for CCL, boxes and filter; fine-grid clear
    # and fine hull; MC compaction; bisection; triangles; depth clear, box and
    # z-buffer); one colour launch per 48 frames
    n_launch = args.steps * ((F + 127) // 128 + 15 + (F + 47) // 48)
    p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step": F, "cameras": int(N), "image": [int(W), int(H)],
                       "l2": f"inputs larger than L2: {mask_bytes / 1e9:.2f} GB masks + "
                             f"{rgb_bytes / 1e9:.2f} GB RGB per step",
                       "timed": "the whole step captured once as a CUDA graph, replayed once per step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "gpu_launches": n_launch,
            "cpu_baseline": cpu, "serving": serving, "tuning": tuning,
            "rooflines": {kernel_of[k]: v for k, v in rooflines.items()}, "alu_probe": alu,
            "l2_roofline": l2_roofline, "fp64_flips": flips,
            "stages_ms_per_frame": {k: v / F for k, v in per_step.items()},
            "eager_ms_per_step": eager_ms,
            "gtests_per_s": world * tests / (ms / 1000.0) / 1e9, "tests_per_frame": tests / F,
            "plain": {"frames_per_s": plain_fps, "latency_ms_p50": p50, "latency_ms_p99": p99, "frames": len(lat),
                      "cuda_graph": True},
            "roofline": roofline, "e2e": e2e, "clocks": clk,
            "device": {"name": torch.cuda.get_device_name(local), "sms": int(sms)}}
    # the figures a reader of the last lines of the output needs, at the end
    line["headline"] = {
        "batched_fps": value, "graph": True, "gtests_per_s": line["gtests_per_s"],
        "plain_fps": plain_fps, "plain_p50_ms": p50, "plain_p99_ms": p99,
        "e2e_fps": e2e["value"] if e2e else None,
        "serving_fps": serving["throughput_fps"] if serving else None,
        "serving_p50_ms": serving["latency_ms_p50"] if serving else None,
        "serving_p99_ms": serving["latency_ms_p99"] if serving else None,
        "serving_frames": serving["frames"] if serving else None,
        "depth_alu_frac": rooflines["depth"]["frac"], "l2_gather_frac": l2_roofline["frac"],
        "fp64_coarse_flips": flips["coarse_flips"] if flips else None,
        "cpu_oracle_fps": cpu["value"] if cpu else None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if r is not None:
        r.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ studies

PAPER_STAGES = (("B-1", ("coarse",)), ("B-2", ("ccl",)), ("B-3", ("fine",)), ("C", ("mc", "bisect")),
                ("D-1", ("depth",)), ("D-2", ("colour",)))


def _timed_reconstruction(fvv, torch, rig, frames, reps=3, keep_results=False):
    """Reconstruct and colour `frames` (one slot each, one batched call) on
    the default launch shapes; per-stage device ms per frame (Table II
    buckets) over `reps` timed repetitions, frames/s, counts and results."""
    F = len(frames)
    r = fvv.Rig(rig, max_slots=F, host_staging=0)
    try:
        slots = list(range(F))
        masks = [f.masks.cuda() for f in frames]
        rgb = torch.stack([f.rgb.cuda() for f in frames])
        vps = np.stack([f.viewpoint for f in frames])

        def step():
            r.upload_silhouettes_batch(slots, masks)
            r.reconstruct(slots)
            r.colour(slots, rgb, vps)
        step()
        torch.cuda.synchronize()
        r.set_timing(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            step()
        b.record()
        torch.cuda.synchronize()
        st = r.timing()
        r.set_timing(False)
        ms = a.elapsed_time(b) / reps
        counts = [r.counts(i) for i in slots]
        res = [r.results(i) for i in slots] if keep_results else None
        stages = {k: v[0] / reps / F for k, v in st.items()}
        paper = {name: sum(stages[k] for k in ks) for name, ks in PAPER_STAGES}
        return {"frames_per_s": F / (ms / 1000.0), "ms_per_frame": ms / F, "stages_ms_per_frame": stages,
                "paper_buckets_ms_per_frame": paper,
                "per_frame": {k: sum(c[k] for c in counts) / F for k in
                              ("n_rois", "n_verts", "n_tris", "tests_coarse", "tests_fine", "tests_bisect")}}, res
    finally:
        r.close()


def _ellipsoid_distance(torch, p, e):
    """Euclidean distance from points p (M,3, float64 tensor) to the surface
    of ellipsoid e, and whether each point is inside it.  The closest point
    of an ellipsoid with semi-axes a to a local point y is a^2 y / (t + a^2)
    where t solves sum (a_i y_i / (t + a_i^2))^2 = 1 (t > -min a_i^2); t is
    found by bisection."""
    dev = p.device
    c = torch.as_tensor(e.centre, dtype=torch.float64, device=dev)
    rot = torch.as_tensor(e.rot, dtype=torch.float64, device=dev)
    a = torch.as_tensor(e.axes, dtype=torch.float64, device=dev)
    y = ((p - c) @ rot).abs().clamp_min(1e-12)     # an exact zero would leave the root unbracketed
    g0 = ((y / a) ** 2).sum(1)
    inside = g0 <= 1.0
    amin2 = float(a.min()) ** 2
    lo = torch.where(inside, torch.full_like(g0, -amin2), torch.zeros_like(g0))
    hi = torch.where(inside, torch.zeros_like(g0), (a * y).norm(dim=1))
    a2 = a * a
    for _ in range(100):
        t = 0.5 * (lo + hi)
        f = ((a * y / (t[:, None] + a2)) ** 2).sum(1) - 1.0
        lo = torch.where(f > 0, t, lo)
        hi = torch.where(f > 0, hi, t)
    t = 0.5 * (lo + hi)
    x = torch.nan_to_num(a2 * y / (t[:, None] + a2))
    return (y - x).norm(dim=1), inside


def _surface_error(torch, verts, ellipsoids):
    """Unsigned distance (m) from each vertex to the surface of the union of
    the ellipsoids: outside all of them, the nearest surface; inside some,
    the largest distance to the surface of one that holds it (a lower bound
    of the distance to the union's boundary)."""
    p = torch.as_tensor(np.asarray(verts, np.float64), device="cuda")
    out_d = torch.full((len(p),), float("inf"), dtype=torch.float64, device="cuda")
    in_d = torch.zeros(len(p), dtype=torch.float64, device="cuda")
    any_in = torch.zeros(len(p), dtype=torch.bool, device="cuda")
    for e in ellipsoids:
        near = ((p - torch.as_tensor(e.centre, device="cuda")).norm(dim=1) <= float(np.max(e.axes)) + 0.3)
        idx = near.nonzero().squeeze(1)
        if len(idx) == 0:
            continue
        d, ins = _ellipsoid_distance(torch, p[idx], e)
        out_d[idx] = torch.minimum(out_d[idx], torch.where(ins, torch.full_like(d, float("inf")), d))
        in_d[idx] = torch.where(ins, torch.maximum(in_d[idx], d), in_d[idx])
        any_in[idx] |= ins
    return torch.where(any_in, in_d, out_d).cpu().numpy()


def _stats_mm(x):
    x = np.asarray(x, np.float64) * 1000.0
    return {"mean": float(x.mean()), "median": float(np.median(x)), "p95": float(np.percentile(x, 95)),
            "max": float(x.max())}


def study_surface(fvv, torch, args):
    """Sec. II-C: where the three surface rules put the vertices.  Rules:
    bisection with the configured 10 steps, the paper's pixel walk and
    minimum ratio (Eqs. (2)-(3)), and the edge midpoint (0 steps, the
    isovalue 0.5 of conventional marching cubes).  Errors against (i) the
    crossing of the all-camera predicate along each edge, found by 24
    bisection steps (within 1 cm / 2^24 of it), and (ii) the analytic
    surfaces of the ellipsoids the silhouettes were rendered from (which
    also holds the visual hull's own excess over the objects)."""
    from dataclasses import replace
    from synth import make_frame, make_rig
    base = make_rig(CONFIG)
    frames = [make_frame(CONFIG, i, device="cuda", rig=base)[1] for i in range(args.study_frames)]
    rules = {"bisect_10": replace(base, bisect_steps=10), "lambda_eq2_eq3": replace(base, surface_rule=1),
             "midpoint": replace(base, bisect_steps=0), "_crossing": replace(base, bisect_steps=24)}
    runs = {k: _timed_reconstruction(fvv, torch, rig, frames, keep_results=True) for k, rig in rules.items()}
    ref = runs["_crossing"][1]
    out = {"study": "surface", "workload": WORKLOAD, "frames": len(frames), "rules": {}}
    for k in ("bisect_10", "lambda_eq2_eq3", "midpoint"):
        timing, res = runs[k]
        cross, surf = [], []
        for fr, rr, r0 in zip(frames, res, ref):
            v, v0 = rr["verts"].double(), r0["verts"].double()
            assert v.shape == v0.shape, "the rules share the mesh topology"
            cross.append((v - v0).norm(dim=1).cpu().numpy())
            surf.append(_surface_error(torch, rr["verts"].cpu().numpy(), fr.ellipsoids))
        out["rules"][k] = {"crossing_error_mm": _stats_mm(np.concatenate(cross)),
                           "object_surface_error_mm": _stats_mm(np.concatenate(surf)),
                           "surface_step_ms_per_frame": timing["stages_ms_per_frame"]["bisect"],
                           "surface_step_tests_per_frame": timing["per_frame"]["tests_bisect"],
                           "verts_per_frame": timing["per_frame"]["n_verts"]}
    return out


def study_fig10(fvv, torch, args):
    """Fig. 10: per-stage time against the coarse voxel size (20-60 mm, fine
    20 mm; coarse = fine = 20 mm is the coarse-to-fine scheme switched off)
    and against the fine voxel size (15-35 mm, coarse 50 mm), on the
    volleyball-shaped scene."""
    from dataclasses import replace
    from synth import make_frame, make_rig
    base = make_rig(CONFIG)
    frames = [make_frame(CONFIG, i, device="cuda", rig=base)[1] for i in range(args.study_frames)]
    out = {"study": "fig10", "workload": WORKLOAD, "frames": len(frames), "coarse_sweep": {}, "fine_sweep": {}}
    for c in (0.02, 0.03, 0.04, 0.05, 0.06):
        t, _ = _timed_reconstruction(fvv, torch, replace(base, coarse_m=c, fine_m=0.02), frames)
        out["coarse_sweep"][f"{round(c * 1000)}mm"] = t
    for f in (0.015, 0.02, 0.025, 0.03, 0.035):
        t, _ = _timed_reconstruction(fvv, torch, replace(base, coarse_m=0.05, fine_m=f), frames)
        out["fine_sweep"][f"{round(f * 1000)}mm"] = t
    return out


# the paper's own per-stage times (Table II) and totals (Table I), GTX 1080 Ti,
# real footage: context for the Table I shapes, not a target
PAPER_TABLE = {"volleyball_t1": {"B-1": 0.54, "B-2": 21.49, "B-3": 1.23, "C": 3.90, "D-1": 5.93, "D-2": 3.30,
                                 "total": 36.39},
               "judo_t1": {"B-1": 0.06, "B-2": 2.11, "B-3": 0.23, "C": 0.65, "D-1": 2.99, "D-2": 1.26,
                           "total": 7.30}}


def study_table1(fvv, torch, args):
    """The capture shapes of Table I on synthetic scenes: volleyball (10
    cameras 4K, 18 x 18 x 9 m, 50/20 mm) and judo (16 cameras 1080p,
    5 x 6 x 2.1 m, 80/40 mm); per-stage time in the Table II buckets beside
    the paper's numbers (GTX 1080 Ti, real footage: context only)."""
    from synth import make_frame, make_rig
    out = {"study": "table1", "frames": args.study_frames, "shapes": {}}
    for cfg in ("volleyball_t1", "judo_t1"):
        rig = make_rig(cfg)
        frames = [make_frame(cfg, i, device="cuda", rig=rig)[1] for i in range(args.study_frames)]
        t, _ = _timed_reconstruction(fvv, torch, rig, frames)
        t["paper_gtx1080ti_ms"] = PAPER_TABLE[cfg]
        out["shapes"][cfg] = t
    return out


def study_view(fvv, torch, args):
    """Step E (Sec. II-E): novel 1920x1080 views of reconstructed
    volleyball-shaped frames from a virtual camera between two capture
    cameras; device time per view (events), covered pixels and how many
    pixels each capture camera coloured."""
    from synth import default_viewpoint, look_at_camera, make_frame, make_rig
    rig = make_rig(CONFIG)
    F = args.study_frames
    frames = [make_frame(CONFIG, i, device="cuda", rig=rig)[1] for i in range(F)]
    W, H = 1920, 1080
    r = fvv.Rig(rig, max_slots=F, host_staging=0)
    try:
        for i, fr in enumerate(frames):
            r.upload_silhouettes(i, fr.masks)
        r.reconstruct(list(range(F)))
        views = []
        for i in range(F):
            C = default_viewpoint(rig, i)
            _, _, P = look_at_camera(np.asarray(C, np.float64), np.array([0.0, 0.0, 1.0]), 1800.0, W, H)
            views.append((P.astype(np.float32), np.asarray(C, np.float32)))
        for i in range(F):                                      # warm-up
            r.render_view(i, frames[i].rgb, *views[i], W, H)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record()
        for _ in range(reps):
            for i in range(F):
                key, img, cam = r.render_view(i, frames[i].rgb, *views[i], W, H)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / (reps * F)
        key, img, cam = r.render_view(0, frames[0].rgb, *views[0], W, H)
        cam = cam.cpu().numpy()
        covered = int((key != -1).sum())
        if args.study_image:
            with open(args.study_image, "wb") as fh:
                fh.write(b"P6 %d %d 255\n" % (W, H))
                fh.write(img.cpu().numpy().tobytes())
        return {"study": "view", "workload": WORKLOAD, "view": [W, H], "frames": F, "ms_per_view": ms,
                "views_per_s": 1000.0 / ms, "covered_pixels": covered,
                "pixels_per_capture_camera": {int(c): int((cam == c).sum()) for c in np.unique(cam) if c >= 0},
                "uncoloured_pixels": int(((cam < 0) & (key.cpu().numpy() != -1)).sum())}
    finally:
        r.close()


def run_study(args):
    import torch
    assert torch.cuda.is_available(), "the studies need a CUDA GPU"
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300 import fvv
    fn = {"surface": study_surface, "fig10": study_fig10, "table1": study_table1, "view": study_view}[args.study]
    print(json.dumps(fn(fvv, torch, args)), flush=True)
    return 0


def main():
    args = parse_args()
    if args.study:
        return run_study(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
