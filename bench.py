#!/usr/bin/env python3
"""Depth-map throughput of the PatchMatch + plane-hypothesis-inference path.

One step = one full depth map of the high-resolution workload: a 3072 x 2048
uint8 reference with 10 source views, 21 x 21 window at dilation 2 (11 x 11
samples), random initialisation, 8 red/black iterations, then plane
hypothesis inference with the 4-label MRF on the unrecovered pixels.
Inputs are seeded synthetic scenes (stand-ins for ETH3D high-res).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle as it stands (a deliberately
slow program, the CPU baseline) on bounded crops of the same workload.
Under torchrun (N > 1) every rank computes its own depth map (views are
independent units; no data exchange), value = pixels of all ranks / max time.
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
sys.path.insert(0, ROOT)

WORKLOAD = dict(W=3072, H=2048, n_src=10, win_radius=10.0, win_samples=11, iters=8, sigma_s=5.0, sigma_c=0.2)
# smaller case of the same kernels for profiler captures (inputs still larger than L2)
WORKLOADS = {"highres": WORKLOAD, "mid": dict(WORKLOAD, W=1536, H=1024), "batch24": dict(WORKLOAD),
             "sparse": dict(WORKLOAD),
             "learned": dict(WORKLOAD, W=1536, H=1024, iters=4), "table3": dict(WORKLOAD),
             "table1": dict(WORKLOAD), "pipeline": dict(WORKLOAD), "combined": dict(WORKLOAD, W=1536, H=1024)}
BATCH_SIZES = ((3072, 2048),) * 8 + ((2048, 1365),) * 8 + ((1536, 1024),) * 8
FLOP_PER_SAMPLE = 26          # algorithmic FP32 flops per window sample of one ZNCC (FMA = 2)
GATHERS_PER_SAMPLE = 1        # one 8-byte coefficient texel per window sample


def l2_bytes_per_sample(n, step):
    """Algorithmic L2 bytes per window sample when each (pixel, view) pair
    fetches its window's rows from L2 once (no reuse across pairs): a row of
    n samples `step` texels apart spans (n - 1) step + 1 texels of 8 bytes,
    counted in 32-byte sectors (one more for alignment)."""
    span = (n - 1) * step + 1
    sectors = int(np.ceil(span * 8 / 32)) + 1
    return n * sectors * 32 / (n * n)


def measured_peaks(mvs, device):
    """FP32 flop/s, L1 gathers/s and L2 bytes/s of this GPU, measured by the
    library's own micro-benchmarks (mvs_measure_peaks) right before the
    timed region, with the SM clock sampled while they run."""
    with ClockSampler(device) as clk:
        f, g, b = mvs.mvs_measure_peaks(device)
    return {"fp32_tflops": f / 1e12, "l1_gathers_per_s": g, "l2_gbs": b / 1e9, "clocks": clk.summary(),
            "how": "mvs_measure_peaks: FFMA chains, 8-byte L1 gathers in the window-sample pattern, "
                   "64 MB L2-resident stream; fastest of five timed launches each after a warm-up"}


def roofline_fractions(sample_evals_per_s, peaks, n, step):
    """Fractions of the three rooflines of the phase kernel from algorithmic
    counts per window sample; the binding one is the largest."""
    fr = {"fp32": FLOP_PER_SAMPLE * sample_evals_per_s / (peaks["fp32_tflops"] * 1e12),
          "l1": GATHERS_PER_SAMPLE * sample_evals_per_s / peaks["l1_gathers_per_s"],
          "l2": l2_bytes_per_sample(n, step) * sample_evals_per_s / (peaks["l2_gbs"] * 1e9)}
    return fr, max(fr, key=fr.get)


def _oracle_worker(args):
    """One oracle process of the N-core CPU baseline: the full path on one
    crop of the shared scene (images read from shared memory)."""
    shm_name, shapes, K, R, t, params, crop, seed = args
    from multiprocessing import shared_memory
    import oracle
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        imgs, off = [], 0
        for (h, w) in shapes:
            imgs.append(np.ndarray((h, w), np.uint8, buffer=shm.buf, offset=off).copy())
            off += h * w
    finally:
        shm.close()

    class _S:
        pass
    sc = _S()
    sc.K, sc.R, sc.t, sc.images = K, R, t, imgs
    return oracle_sample(sc, params, crop, n_crops=1, seed=seed)


def oracle_throughput(sc, params, crop, crops_per_core=2, seed=0):
    """N-core CPU baseline: one oracle process per host core (spawned, after
    CUDA is up in this process), each on independent crops.  Returns
    (pixels per second over the wall time of the parallel section, cores,
    pixels)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    cores = os.cpu_count() or 1
    total = sum(im.size for im in sc.images)
    shm = shared_memory.SharedMemory(create=True, size=total)
    try:
        off = 0
        for im in sc.images:
            np.ndarray(im.shape, np.uint8, buffer=shm.buf, offset=off)[...] = im
            off += im.size
        shapes = [im.shape for im in sc.images]
        jobs = [(shm.name, shapes, sc.K, sc.R, sc.t, params, crop, seed + k) for k in range(cores * crops_per_core)]
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_worker, jobs[:cores])       # start-up (imports, oracle build check) untimed
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, jobs)
            wall = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    px = sum(r[1] for r in res)
    return px / wall, cores, px


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up can hold up CUDA calls of this process for
            # hundreds of ms: begin the warm-up only once it reports
            t0 = time.perf_counter()
            while not self.rows and self.proc.poll() is None and time.perf_counter() - t0 < 10.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_params(mvs, seed, lanes=0, precision=0):
    w = WORKLOAD
    return mvs.PMParams(win_radius=w["win_radius"], win_samples=w["win_samples"], sigma_s=w["sigma_s"],
                        sigma_c=w["sigma_c"], d_lo=2.0, d_hi=8.0, iters=w["iters"], seed=seed,
                        lanes_per_pixel=lanes, precision=precision)


# ---------------------------------------------------------------------------
# CPU oracle on a crop of the reference view (cpu_baseline / --impl reference)
# ---------------------------------------------------------------------------
def crop_scene(sc, x0, y0, cw, ch):
    """The reference view cut to a cw x ch window at (x0, y0): same camera
    with its principal point moved; the sources stay whole."""
    K = sc.K.copy()
    K[0, 0, 2] -= x0
    K[0, 1, 2] -= y0
    imgs = [np.ascontiguousarray(sc.images[0][y0:y0 + ch, x0:x0 + cw])] + list(sc.images[1:])
    return K, imgs


def oracle_sample(sc, params, crop, n_crops=1, seed=0):
    """Full oracle path (init, iterations, plane inference) on n_crops crops
    of the reference placed uniformly at random over the image (so textured
    and texture-less areas appear in their proportions); returns (seconds,
    pixels)."""
    import oracle
    cw, ch = crop
    H, W = sc.images[0].shape
    rng = np.random.default_rng(seed)
    tot, px = 0.0, 0
    for _ in range(n_crops):
        x0 = int(rng.integers(0, W - cw))
        y0 = int(rng.integers(0, H - ch))
        K, imgs = crop_scene(sc, x0, y0, cw, ch)
        osc = oracle.Scene(K, sc.R, sc.t, imgs)
        srcs = list(range(1, len(imgs)))
        t = time.perf_counter()
        pl, co = oracle.patchmatch(osc, 0, srcs, params, params.iters)
        known = ((pl[..., 3] > 0) & (co < 0.5)).astype(np.uint8)
        oracle.plane_infer(osc, 0, srcs, params, known, pl)
        tot += time.perf_counter() - t
        px += cw * ch
    return tot, px


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from paper_2104_06165_gb300 import mvs, scenes
    w = WORKLOAD
    sc = scenes.scene_highres(seed=0, W=w["W"], H=w["H"], n_src=w["n_src"])
    params = make_params(mvs, 0)
    crop = (24, 16)
    for i in range(args.warmup):
        oracle_sample(sc, params, crop, n_crops=1, seed=100 + i)
    tot_t, tot_px = 0.0, 0
    for i in range(args.steps):
        t, px = oracle_sample(sc, params, crop, n_crops=1, seed=i)
        tot_t += t
        tot_px += px
    value = tot_px / tot_t / 1e6
    line = {"impl": "reference", "metric": "depth-map Mpix/s (full PatchMatch + PHI)", "value": value,
            "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "highres 3072x2048 + 10 sources, 21x21 dil 2, 8 iters, PHI+MRF",
                       "sample": f"one random {crop[0]}x{crop[1]} reference crop per step, full-size sources"},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": f"one random {crop[0]}x{crop[1]} crop of the 3072x2048 reference per step"},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, scenes
    mvs.load()
    w = WORKLOAD
    t0 = time.perf_counter()
    sc = scenes.scene_highres(seed=rank, W=w["W"], H=w["H"], n_src=w["n_src"])
    t_render = time.perf_counter() - t0
    H, W = sc.images[0].shape
    srcs = list(range(1, len(sc.images)))
    params = make_params(mvs, seed=1 + rank, lanes=args.lanes, precision=1 if args.precision == "mixed" else 0)
    phi = mvs.PhiParams()
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    plane = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    cost = torch.empty((H, W), dtype=torch.float32, device=dev)

    def step():
        mvs.mvs_patchmatch(ctx.h, 0, srcs, params, plane, cost)
        mvs.mvs_plane_infer(ctx.h, 0, srcs, params, phi, None, plane, cost)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    peaks = measured_peaks(mvs, local)
    if world > 1:
        dist.barrier()
    mvs.mvs_profile(ctx.h, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    phase_ms, phase_n, launches, evals = mvs.mvs_profile_read(ctx.h)
    mvs.mvs_profile(ctx.h, 0)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the public API: host images (pinned) in, host depth map out
    ctx.close()
    pinned = []
    for im in sc.images:
        t_ = torch.empty(im.shape, dtype=torch.uint8, pin_memory=True)
        t_.numpy()[...] = im
        pinned.append(t_.numpy())
    h_plane_t = torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 3))

    def e2e_step_host():
        c2 = mvs.Context(sc.K, sc.R, sc.t, pinned, stream=stream)     # H2D of the images
        mvs.mvs_patchmatch(c2.h, 0, srcs, params, plane, cost)
        mvs.mvs_plane_infer(c2.h, 0, srcs, params, phi, None, plane, cost)
        h_plane_t.copy_(plane, non_blocking=True)                       # D2H of the depth/normal map
        stream.synchronize()
        c2.close()

    e2e_step_host()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step_host()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = int(sum(im.nbytes for im in sc.images))
    d2h = int(h_plane_t.numel() * 4)

    mpix = H * W / 1e6
    value = world * mpix * args.steps / (ms / 1e3)
    # roofline of the dominant kernel (checkerboard phase): algorithmic FP32
    # flops = evaluated ZNCCs x window samples x FLOP_PER_SAMPLE
    n2 = w["win_samples"] ** 2
    phase_flops = evals * n2 * FLOP_PER_SAMPLE
    achieved = phase_flops / (phase_ms / 1e3) / 1e12 if phase_ms > 0 else None
    peak = peaks["fp32_tflops"]
    step_px = w["win_radius"] / (0.5 * (w["win_samples"] - 1))
    fracs, binding = roofline_fractions(evals * n2 / (phase_ms / 1e3), peaks, w["win_samples"], step_px)
    line = {
        "metric": "depth-map Mpix/s (full PatchMatch + PHI)",
        "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f16/f32 mixed", "data": "synthetic",
        "config": {"precision": args.precision, "workload": f"{args.workload} {W}x{H} uint8 ref + {len(srcs)} sources, 21x21 window dil 2 "
                               "(11x11 samples), 8 iterations, PHI + 4-label MRF", "parallelism": f"replicas{world}",
                   "lanes_per_pixel": args.lanes,
                   "l2": f"inputs larger than L2 ({len(sc.images)} textures of {(W + 1) * (H + 1) * 8 / 1e6:.0f} MB)",
                   "render_s": round(t_render, 1)},
        "e2e": {"value": world * mpix / e2e_s, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "ncc_evals_per_s": evals / (phase_ms / 1e3) if phase_ms > 0 else None,
        "phase_kernel_ms": phase_ms / max(1, phase_n),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": (tpp * H * W if (tpp := phase_traffic_per_pixel()) else None),
                     "traffic_unit": "bytes per launch (ncu dram read+write, 1536x1024 capture scaled by pixels)",
                     "kernel": "k_phase (checkerboard propagation + refinement)",
                     "peak_basis": "measured FFMA rate of this GPU (mvs_measure_peaks), see peaks",
                     "fractions": {k: round(v, 4) for k, v in fracs.items()}, "binding": binding,
                     "binding_note": "the largest of the three fractions from algorithmic counts; the L2 count "
                                     "assumes no L1 reuse across pairs, while the kernel's measured limiter is "
                                     "instruction issue (ncu: 75 % of issue slots, L2 at 20 % of its peak)",
                     "fraction_basis": {"fp32": f"{FLOP_PER_SAMPLE} flop per window sample / measured FFMA peak",
                                        "l1": f"{GATHERS_PER_SAMPLE} 8-byte gather per window sample / measured "
                                              "L1 gather peak in the same pattern",
                                        "l2": f"{l2_bytes_per_sample(w['win_samples'], step_px):.1f} bytes per "
                                              "window sample (each pair's window rows from L2 once) / measured "
                                              "L2 read bandwidth"},
                     "peaks": peaks},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        try:
            t_, px = oracle_sample(sc, params, (24, 16), n_crops=4, seed=7)
            line["cpu_baseline"] = {"value": px / t_ / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                                    "sample": "4 random 24x16 crops of the 3072x2048 reference, full-size "
                                              "sources, full path (init, 8 iterations, PHI)"}
            v_n, cores, px_n = oracle_throughput(sc, params, (24, 16), crops_per_core=2, seed=11)
            line["cpu_baseline_all_cores"] = {"value": v_n / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                                              "sample": f"{2 * cores} random 24x16 crops, one oracle process per "
                                                        f"host core (os.cpu_count() = {cores}), full path"}
        except Exception as e:  # the baseline is informative only
            line["cpu_baseline"] = line.get("cpu_baseline") or {"error": str(e)[:200]}
            line["cpu_baseline_all_cores"] = {"error": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """24 reference views at mixed resolutions, each with 10 sources, in one
    captured CUDA graph (autotuned work layout), then the geometric filter of
    every view against its sources.  Under several ranks the 24 views are
    sharded by pixel count (dist.filter_sharded: each rank's views in one
    graph, the plane maps exchanged over NCCL, each rank filters its own
    views): strong scaling of the one scene."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2104_06165_gb300 import dist as pdist, mvs, scenes
    mvs.load()
    t0 = time.perf_counter()
    sc, srcs = scenes.scene_batch(seed=0, sizes=BATCH_SIZES)
    t_render = time.perf_counter() - t0
    n = len(sc.images)
    refs = list(range(n))
    params = make_params(mvs, seed=1 + rank, lanes=-1 if args.lanes == 0 else args.lanes)
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    planes = [torch.empty(im.shape + (4,), dtype=torch.float32, device=dev) for im in sc.images]
    costs = [torch.empty(im.shape, dtype=torch.float32, device=dev) for im in sc.images]
    keeps = [torch.empty(im.shape, dtype=torch.uint8, device=dev) for im in sc.images]
    fp = mvs.FilterParams()

    shapes = [im.shape for im in sc.images]

    def step():
        if world > 1:
            ks, _ = pdist.filter_sharded(mvs, ctx, shapes, srcs, params, fp, device=dev)
            for v, k in ks.items():
                keeps[v] = k
            return
        mvs.mvs_patchmatch_batch(ctx.h, refs, srcs, params, planes, costs)
        for r in refs:
            mvs.mvs_geo_filter(ctx.h, r, srcs[r], fp, keeps[r])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mvs.mvs_profile(ctx.h, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    _, _, launches, _ = mvs.mvs_profile_read(ctx.h)
    mpix = sum(im.size for im in sc.images) / 1e6
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        if rank == 0:
            print(json.dumps({"metric": "depth-map Mpix/s (batched PatchMatch + geometric filter, views sharded)",
                              "value": mpix * args.steps / (ms / 1e3), "unit": "Mpix/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                              "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic", "gpu_launches": int(launches),
                              "config": {"workload": "batch24, views sharded by pixel count over the ranks "
                                                     "(dist.filter_sharded), one exchange of the plane maps",
                                         "total_mpix": round(mpix, 2)},
                              "clocks": clk.summary()}), flush=True)
        ctx.close()
        dist.destroy_process_group()
        return
    kept = float(sum(k.float().mean().item() * k.numel() for k in keeps) / (mpix * 1e6))
    # depth-map fusion (Sec. III-F) of the 24 filtered maps into one cloud
    cap = int(mpix * 1e6)
    pts = torch.empty((cap, 4), dtype=torch.float32, device=dev)
    n_pts = mvs.mvs_fuse(ctx.h, refs, pts, None, keep_masks=keeps)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    f0.record(stream)
    for _ in range(reps):
        mvs.mvs_fuse(ctx.h, refs, pts, None, keep_masks=keeps)
    f1.record(stream)
    torch.cuda.synchronize()
    fuse_ms = f0.elapsed_time(f1) / reps
    merged = float(pts[:n_pts, 3].mean().item()) if n_pts else 0.0
    # neighbouring-image selection (Sec. III-A) from synthetic SfM points
    sp = scenes.sparse_points(sc, 20000, seed=7 + rank)
    masks = np.zeros(len(sp["X"]), np.uint64)
    for v in range(n):
        masks |= sp["vis"][:, v].astype(np.uint64) << np.uint64(v)
    d_X = torch.from_numpy(np.ascontiguousarray(sp["X"])).to(dev)
    d_m = torch.from_numpy(masks.view(np.int64)).to(dev)
    nbr = torch.zeros((n, 8), dtype=torch.int32, device=dev)
    mvs.mvs_select_neighbors(ctx.h, d_X, d_m, nbr)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(reps):
        mvs.mvs_select_neighbors(ctx.h, d_X, d_m, nbr)
    s1.record(stream)
    torch.cuda.synchronize()
    sel_ms = s0.elapsed_time(s1) / reps
    nb = nbr.cpu().numpy()
    agree = float(np.mean([len(set(nb[v][nb[v] >= 0].tolist()) & set(srcs[v])) / 8.0 for v in range(n)]))
    line = {"metric": "depth-map Mpix/s (batched PatchMatch + geometric filter)", "value": mpix * args.steps / (ms / 1e3),
            "unit": "Mpix/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch24: 8x3072x2048 + 8x2048x1365 + 8x1536x1024 reference views, 10 sources "
                                   "each, 21x21 window dil 2, 8 iterations, one CUDA graph, geometric filter",
                       "lanes_per_pixel": params.lanes_per_pixel, "render_s": round(t_render, 1),
                       "total_mpix": round(mpix, 2)},
            "gpu_launches": int(launches), "kept_fraction": kept,
            "fusion": {"ms": fuse_ms, "input_mpix": round(mpix, 2), "kept_mpix": round(kept * mpix, 2),
                       "mpix_per_s": mpix / (fuse_ms / 1e3), "points": int(n_pts), "mean_merged": merged,
                       "views": len(refs), "note": "mvs_fuse of the 24 geometric-filter-masked maps, after the "
                                                   "timed steps (not inside them)"},
            "neighbor_selection": {"ms": sel_ms, "points": int(len(sp["X"])), "views": n, "k": 8,
                                   "shared_with_angle_rule": agree,
                                   "note": "mvs_select_neighbors (Eqs. 1-3) from synthetic SfM points, after the "
                                           "timed steps; shared_with_angle_rule = mean fraction of the 8 chosen "
                                           "sources that are among the 10 the bench's 15-40 degree rule uses"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_pipeline(args):
    """The paper's whole Algorithm 1 on the 24-view scene of batch24, every
    stage on the GPU inside one timed step: neighbouring-image selection
    (Eqs. 1-3, top 8) from 20 k synthetic SfM points, per-view depth ranges
    from the sparse features (Sec. III-B), PatchMatch of all 24 views in one
    graph from those ranges (8 iterations), the geometric filter, plane
    hypothesis inference on the filtered maps, the filter again, and the
    fusion of the 24 maps into one point cloud (Sec. III-F).  value = input
    Mpix/s of the whole algorithm."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, scenes
    mvs.load()
    t0 = time.perf_counter()
    sc, angle_srcs = scenes.scene_batch(seed=rank, sizes=BATCH_SIZES, want_gt=True)
    t_render = time.perf_counter() - t0
    n = len(sc.images)
    refs = list(range(n))
    k_nbr = 8
    sp = scenes.sparse_points(sc, 20000, seed=7 + rank)
    masks = np.zeros(len(sp["X"]), np.uint64)
    for v in range(n):
        masks |= sp["vis"][:, v].astype(np.uint64) << np.uint64(v)
    d_X = torch.from_numpy(np.ascontiguousarray(sp["X"])).to(dev)
    d_m = torch.from_numpy(masks.view(np.int64)).to(dev)
    d_rep = torch.from_numpy(np.ascontiguousarray(sp["reproj"])).to(dev)
    d_obs = [torch.from_numpy(np.ascontiguousarray(sp["obs"][:, v])).to(dev) for v in refs]
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    sizes = [im.shape for im in sc.images]
    offs = np.concatenate([[0], np.cumsum([h * w for h, w in sizes])])
    ranges = torch.empty((int(offs[-1]) * 2,), dtype=torch.float32, device=dev)
    rng_views = [ranges[2 * int(offs[v]):2 * int(offs[v + 1])].view(sizes[v][0], sizes[v][1], 2) for v in refs]
    planes = [torch.empty(hw + (4,), dtype=torch.float32, device=dev) for hw in sizes]
    costs = [torch.empty(hw, dtype=torch.float32, device=dev) for hw in sizes]
    keeps = [torch.empty(hw, dtype=torch.uint8, device=dev) for hw in sizes]
    nbr = torch.zeros((n, k_nbr), dtype=torch.int32, device=dev)
    cap = int(offs[-1])
    pts = torch.empty((cap, 4), dtype=torch.float32, device=dev)
    params = make_params(mvs, seed=1 + rank)
    params.init_mode, params.init_range = mvs.MVS_INIT_RANGE, ranges
    phi = mvs.PhiParams()
    fp = mvs.FilterParams()
    evs = {}
    n_sel = []

    def mark(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        evs.setdefault(name, []).append(e)

    def step():
        mark("select")
        mvs.mvs_select_neighbors(ctx.h, d_X, d_m, nbr)
        nb = nbr.cpu().numpy()
        srcs = []
        for v in refs:     # pad a short list with the nearest views by angle
            lst = [int(u) for u in nb[v] if u >= 0]
            n_sel.append(len(lst))
            lst += [u for u in angle_srcs[v] if u not in lst][:k_nbr - len(lst)]
            srcs.append(lst)
        mark("sparse_range")
        for v in refs:
            mvs.mvs_sparse_depth_range(ctx.h, v, d_X, d_m, d_rep, d_obs[v], rng_views[v])
        mark("patchmatch")
        mvs.mvs_patchmatch_batch(ctx.h, refs, srcs, params, planes, costs)
        mark("filter1")
        for v in refs:
            mvs.mvs_geo_filter(ctx.h, v, srcs[v], fp, keeps[v])
        mark("phi")
        for v in refs:
            mvs.mvs_plane_infer(ctx.h, v, srcs[v], params, phi, keeps[v], planes[v], costs[v])
        mark("filter2")
        for v in refs:
            mvs.mvs_geo_filter(ctx.h, v, srcs[v], fp, keeps[v])
        mark("fusion")
        n_pts = mvs.mvs_fuse(ctx.h, refs, pts, None, keep_masks=keeps)
        mark("end")
        return n_pts, srcs

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs.clear()
    mvs.mvs_profile(ctx.h, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            n_pts, srcs = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    _, _, launches, _ = mvs.mvs_profile_read(ctx.h)
    mvs.mvs_profile(ctx.h, 0)
    order = ["select", "sparse_range", "patchmatch", "filter1", "phi", "filter2", "fusion", "end"]
    stage_ms = {a: float(np.mean([evs[a][i].elapsed_time(evs[b][i]) for i in range(args.steps)]))
                for a, b in zip(order[:-1], order[1:])}
    # quality against the rendered truth: final kept depths within 1 %
    comp, acc = [], []
    for v in refs:
        g = sc.gt_views[v]["depth"]
        d = planes[v][..., 3].cpu().numpy()
        k = keeps[v].cpu().numpy().astype(bool)
        good = k & (np.abs(d - g) <= 0.01 * g)
        comp.append(good.mean())
        acc.append(good.sum() / max(1, k.sum()))
    mpix = sum(h * w for h, w in sizes) / 1e6
    line = {"metric": "Algorithm 1 input Mpix/s (selection, sparse init, PatchMatch, filter, PHI, filter, fusion)",
            "value": mpix * args.steps / (ms / 1e3), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "pipeline: 8x3072x2048 + 8x2048x1365 + 8x1536x1024 views of one scene, "
                                   f"{k_nbr} selected sources each, 20 k synthetic SfM points, 21x21 window "
                                   "dil 2, 8 iterations, PHI + 4-label MRF, two geometric filters, fusion",
                       "render_s": round(t_render, 1), "total_mpix": round(mpix, 2)},
            "gpu_launches": int(launches), "stage_ms": stage_ms,
            "quality": {"completeness": float(np.mean(comp)), "kept_within_1pct": float(np.mean(acc)),
                        "points": int(n_pts),
                        "note": "per-view means over the 24 final maps: completeness = kept pixels within 1 % of "
                                "the rendered depth / all pixels; kept_within_1pct = the same / kept pixels"},
            "sources_from_selection": float(np.mean(n_sel)),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


PHASE_SOURCES = ["paper_2104_06165_gb300/csrc/pm_kernels.cu", "paper_2104_06165_gb300/csrc/pm_device.cuh",
                 "paper_2104_06165_gb300/csrc/mvs_internal.h"]


def phase_traffic_per_pixel():
    """DRAM bytes per reference pixel of one k_phase launch from the committed
    ncu summary, or None when the kernel sources changed since the capture."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", "k_phase_mid_full.md")).read()
        vals = dict(l.split(": ", 1) for l in txt.splitlines() if l.startswith(("traffic_bytes_per_pixel:",
                                                                                "sources_sha256:")))
        h = hashlib.sha256()
        for f in PHASE_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != vals["sources_sha256"].strip():
            return None
        return float(vals["traffic_bytes_per_pixel"])
    except Exception:
        return None


def _peak_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def run_learned(args):
    """Learned plane proposals on 1536 x 1024 scenes with about half of the
    image texture-less: one step = initialisation, one plain iteration, the
    proposal network on that state, three iterations with K = 4 proposals
    per pixel.  The plain 8-iteration depth map of the same scene is timed
    the same way; both are scored by completeness (depth within 1 % of the
    ground truth)."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, proposals as P
    mvs.load()
    t0 = time.perf_counter()
    sc = P.scene(2000 + rank)
    t_render = time.perf_counter() - t0
    H, W = sc.images[0].shape
    srcs = list(range(1, len(sc.images)))
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    net = mvs.mvs_cnn_create(W, H, 2.0, 8.0, 0, stream)
    P.load_weights(net)
    plane = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    cost = torch.empty((H, W), dtype=torch.float32, device=dev)
    props = torch.empty((H, W, P.K_PROP, 4), dtype=torch.float32, device=dev)
    learned = lambda: P.learned_patchmatch(ctx, 0, srcs, P.pm_params(1 + rank), net, plane, cost, props, iters=4)
    plain8 = lambda: mvs.mvs_patchmatch(ctx.h, 0, srcs, P.pm_params(1 + rank, iters=8), plane, cost)

    def timed(fn, clk=None):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        mvs.mvs_profile(ctx.h, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        prof = mvs.mvs_profile_read(ctx.h)
        mvs.mvs_profile(ctx.h, 0)
        return e0.elapsed_time(e1) / args.steps, prof, P.completeness(plane.cpu().numpy(), sc.gt_depth)

    with ClockSampler(local) as clk:
        ms_l, prof_l, comp_l = timed(learned)
        ms_p, prof_p, comp_p = timed(plain8)
    # the proposal network alone (forward + decode) on the learned state
    learned()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        mvs.mvs_propose(ctx.h, 0, net, props)
    e1.record(stream)
    torch.cuda.synchronize()
    cnn_ms = e0.elapsed_time(e1) / reps
    from paper_2104_06165_gb300.proposals import cnn_flops
    peak_bf16, peak_kind = _peak_bf16()
    cnn_tf = cnn_flops(W, H) / (cnn_ms / 1e3) / 1e12
    phase_ms, phase_n, launches, evals = prof_l
    n2 = WORKLOAD["win_samples"] ** 2
    achieved = evals * n2 * FLOP_PER_SAMPLE / (phase_ms / 1e3) / 1e12 if phase_ms > 0 else None
    peaks = measured_peaks(mvs, local)
    peak = peaks["fp32_tflops"]
    mpix = H * W / 1e6
    line = {
        "metric": "depth-map Mpix/s (learned proposals + 4-iteration PatchMatch)", "value": mpix / (ms_l / 1e3),
        "unit": "Mpix/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_l,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (network bf16)",
        "data": "synthetic",
        "config": {"workload": f"learned {W}x{H} uint8 ref + {len(srcs)} sources, ~50% texture-less, 21x21 window "
                               "dil 2, 1 plain iteration + proposal network + 3 iterations with 4 proposals/pixel",
                   "render_s": round(t_render, 1), "l2": "inputs larger than L2 (11 textures of 13 MB)"},
        "completeness": comp_l,
        "plain8": {"value": mpix / (ms_p / 1e3), "ms_per_step": ms_p, "completeness": comp_p},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "kernel": "k_phase (propagation + proposals + refinement)",
                     "peak_basis": "measured FFMA rate of this GPU (mvs_measure_peaks)"},
        "cnn": {"ms": cnn_ms, "achieved_tflops": cnn_tf, "peak_tflops": peak_bf16, "peak": peak_kind,
                "frac": cnn_tf / peak_bf16, "bound": "tensor"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    mvs.mvs_cnn_destroy(net)
    ctx.close()


def run_combined(args):
    """The three additions together against plain PatchMatch on one scene of
    eight 1536 x 1024 reference views (about half of the surface
    texture-less, 10 sources each, 21 x 21 window at dilation 2):
      plain-k:    FP32 PatchMatch view by view, k = 1..4 iterations;
      batched-k:  the same eight views in one captured graph;
      combined-k: the eight views batched, mixed precision, one iteration,
                  the trained proposal network on every view's state, then
                  k - 1 iterations with K = 4 proposals per pixel (k = 2, 4);
      batched-learned-2: the combined form in FP32 (no mixed precision).
    Completeness: pixels within 1 % of the rendered depth over all eight
    views.  value = the combined form with the best Mpix/s among those at
    least as complete as plain-2; `versus` names the fastest plain or batched
    schedule that reaches that completeness and the ratio."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, proposals as P, scenes
    mvs.load()
    t0 = time.perf_counter()
    n, W, H = 8, 1536, 1024
    sc, srcs = scenes.scene_batch(seed=2000 + rank, sizes=((W, H),) * n, flat_frac=0.5, want_gt=True)
    t_render = time.perf_counter() - t0
    refs = list(range(n))
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    net = mvs.mvs_cnn_create(W, H, 2.0, 8.0, 0, stream)
    P.load_weights(net)
    planes = [torch.empty((H, W, 4), dtype=torch.float32, device=dev) for _ in refs]
    costs = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in refs]
    props = torch.empty((n, H, W, P.K_PROP, 4), dtype=torch.float32, device=dev)
    gts = [sc.gt_views[v]["depth"] for v in refs]

    def completeness():
        return float(np.mean([P.completeness(planes[v].cpu().numpy(), gts[v]) for v in refs]))

    def plain(k):
        for v in refs:
            mvs.mvs_patchmatch(ctx.h, v, srcs[v], P.pm_params(1, iters=k), planes[v], costs[v])

    def batched(k):
        mvs.mvs_patchmatch_batch(ctx.h, refs, srcs, P.pm_params(1, iters=k), planes, costs)

    def combined(k, precision=1):
        mvs.mvs_patchmatch_batch(ctx.h, refs, srcs,
                                 P.pm_params(1, iters=k, phase_begin=0, phase_end=2, precision=precision),
                                 planes, costs)
        for v in refs:
            mvs.mvs_propose(ctx.h, v, net, props[v])
        mvs.mvs_patchmatch_batch(ctx.h, refs, srcs,
                                 P.pm_params(1, iters=k, phase_begin=2, phase_end=2 * k, precision=precision,
                                             init_mode=mvs.MVS_INIT_GIVEN, n_prop=P.K_PROP, proposals=props),
                                 planes, costs)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        return {"ms_per_step": ms, "mpix_s": n * W * H / 1e6 / (ms / 1e3), "completeness": round(completeness(), 4)}

    arms = {}
    with ClockSampler(local) as clk:
        for k in (1, 2, 3, 4):
            arms[f"plain-{k}"] = timed(lambda: plain(k))
        for k in (1, 2, 3, 4):
            arms[f"batched-{k}"] = timed(lambda: batched(k))
        for k in (2, 4):
            arms[f"combined-{k}"] = timed(lambda: combined(k))
        # the same without the mixed-precision ZNCC (batched + learned, FP32)
        arms["batched-learned-2"] = timed(lambda: combined(2, precision=0))
    target = arms["plain-2"]["completeness"]
    good = [a for a in ("combined-2", "combined-4") if arms[a]["completeness"] >= target - 0.001]
    best = max(good or ["combined-2", "combined-4"], key=lambda a: arms[a]["mpix_s"])
    need = arms[best]["completeness"] - 0.001
    rivals = [a for a in arms if a.startswith(("plain", "batched-")) and "learned" not in a
              and arms[a]["completeness"] >= need]
    rival = max(rivals, key=lambda a: arms[a]["mpix_s"]) if rivals else None
    line = {
        "metric": "depth-map Mpix/s (batched + mixed precision + learned proposals) vs plain PatchMatch",
        "value": arms[best]["mpix_s"], "unit": "Mpix/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": arms[best]["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16/f32 mixed (network bf16)", "data": "synthetic",
        "config": {"workload": f"combined: {n} reference views {W}x{H} of one scene (about half texture-less), "
                               "10 sources each, 21x21 window dil 2", "form": best,
                   "render_s": round(t_render, 1)},
        "completeness": arms[best]["completeness"],
        "versus": {"schedule": rival, "mpix_s": arms[rival]["mpix_s"] if rival else None,
                   "completeness": arms[rival]["completeness"] if rival else None,
                   "ratio": arms[best]["mpix_s"] / arms[rival]["mpix_s"] if rival else None,
                   "note": "the fastest plain or batched FP32 schedule at least as complete as the combined form"},
        "arms": arms,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    mvs.mvs_cnn_destroy(net)
    ctx.close()


def run_sparse(args):
    """Sparse-feature depth initialisation (Sec. III-B) on the
    high-resolution workload: synthetic SfM points (20 k, 0.5 px noise, 2 %
    outliers), per-pixel depth ranges by mvs_sparse_depth_range, then
    PatchMatch from that initialisation and from the random one for 1, 2, 4
    and 8 iterations; completeness = pixels within 1 % of the true depth.
    value = Mpix/s of the sparse-initialised run with the fewest iterations
    that reaches the random 8-iteration completeness (range computation
    included)."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, scenes
    mvs.load()
    w = WORKLOAD
    sc = scenes.scene_highres(seed=rank, W=w["W"], H=w["H"], n_src=w["n_src"])
    H, W = sc.images[0].shape
    srcs = list(range(1, len(sc.images)))
    sp = scenes.sparse_points(sc, 20000, seed=3 + rank)
    masks = np.zeros(len(sp["X"]), np.uint64)
    for v in range(len(sc.images)):
        masks |= sp["vis"][:, v].astype(np.uint64) << np.uint64(v)
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
            (sp["X"], masks.view(np.int64), sp["reproj"], sp["obs"][:, 0])]
    rng = torch.empty((H, W, 2), dtype=torch.float32, device=dev)
    plane = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    cost = torch.empty((H, W), dtype=torch.float32, device=dev)
    gt = sc.gt_depth

    def run(iters, sparse):
        p = make_params(mvs, 1 + rank)
        p.iters = iters
        if sparse:
            mvs.mvs_sparse_depth_range(ctx.h, 0, *d_in, rng)
            p.init_mode, p.init_range = mvs.MVS_INIT_RANGE, rng
        mvs.mvs_patchmatch(ctx.h, 0, srcs, p, plane, cost)

    rows = []
    with ClockSampler(local) as clk:
        for sparse in (False, True):
            for iters in (1, 2, 4, 8):
                for _ in range(args.warmup):
                    run(iters, sparse)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    run(iters, sparse)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                d = plane[..., 3].cpu().numpy()
                comp = float((np.abs(d - gt) <= 0.01 * gt).mean())
                rows.append({"init": "sparse" if sparse else "random", "iters": iters, "ms": ms,
                             "mpix_s": H * W / 1e3 / ms, "completeness": comp})
    target = [r for r in rows if r["init"] == "random" and r["iters"] == 8][0]
    ok = [r for r in rows if r["init"] == "sparse" and r["completeness"] >= target["completeness"] - 0.005]
    best = min(ok, key=lambda r: r["iters"]) if ok else [r for r in rows if r["init"] == "sparse"][-1]
    line = {"metric": "depth-map Mpix/s (sparse-feature initialisation, PatchMatch only)", "value": best["mpix_s"],
            "unit": "Mpix/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"sparse {W}x{H} uint8 ref + {len(srcs)} sources, 21x21 window dil 2, "
                                   "20 k synthetic SfM points, PatchMatch without PHI",
                       "chosen": {"iters": best["iters"], "completeness": best["completeness"]},
                       "random_8_iters": {"mpix_s": target["mpix_s"], "completeness": target["completeness"]}},
            "rows": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_table1(args):
    """The paper's PHI ablation (Sec. IV, Table I) on the high-resolution
    synthetic workload: PatchMatch alone (PHI-MVS/P: pixels whose cost
    passes the hole threshold), PHI selecting each hole's hypothesis of
    minimal matching cost (PHI-MVS/M) and PHI with the MRF (PHI-MVS), all
    from the same 8-iteration PatchMatch map.  Completeness = pixels within
    1 % of the true depth, over all pixels and over the texture-less ones
    (F1 on ETH3D in the paper).  value = Mpix/s of PatchMatch + PHI-MVS/M."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, scenes
    mvs.load()
    w = WORKLOAD
    sc = scenes.scene_highres(seed=rank, W=w["W"], H=w["H"], n_src=w["n_src"])
    H, W = sc.images[0].shape
    srcs = list(range(1, len(sc.images)))
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    params = make_params(mvs, seed=1 + rank)
    plane0 = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    cost0 = torch.empty((H, W), dtype=torch.float32, device=dev)
    plane = torch.empty_like(plane0)
    cost = torch.empty_like(cost0)
    gt = sc.gt_depth
    flat = ~sc.gt_textured
    phi = mvs.PhiParams()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def comp(d, ok=None):
        good = np.abs(d - gt) <= 0.01 * gt
        if ok is not None:
            good &= ok
        return float(good.mean()), float(good[flat].mean())

    rows = []
    with ClockSampler(local) as clk:
        pm_ms = timed(lambda: mvs.mvs_patchmatch(ctx.h, 0, srcs, params, plane0, cost0))
        d0 = plane0[..., 3].cpu().numpy()
        c, cf = comp(d0, cost0.cpu().numpy() < phi.hole_cost)
        rows.append({"pipeline": "PHI-MVS/P", "phi_ms": 0.0, "completeness": c, "completeness_textureless": cf})
        for name, sel in (("PHI-MVS/M", mvs.MVS_PHI_SELECT_MIN_COST), ("PHI-MVS", mvs.MVS_PHI_SELECT_MRF)):
            q = mvs.PhiParams(selection=sel)

            def step():
                plane.copy_(plane0)
                cost.copy_(cost0)
                mvs.mvs_plane_infer(ctx.h, 0, srcs, params, q, None, plane, cost)
            ms = timed(step)
            c, cf = comp(plane[..., 3].cpu().numpy())
            rows.append({"pipeline": name, "phi_ms": ms, "completeness": c, "completeness_textureless": cf})
    for r in rows:
        r["mpix_s"] = H * W / 1e3 / (pm_ms + r["phi_ms"])
    m = [r for r in rows if r["pipeline"] == "PHI-MVS/M"][0]
    line = {"metric": "depth-map Mpix/s (PatchMatch + PHI-MVS/M)", "value": m["mpix_s"], "unit": "Mpix/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": pm_ms + m["phi_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"table1 {W}x{H} uint8 ref + {len(srcs)} sources, 21x21 window dil 2, "
                                   "8 iterations, then no PHI / PHI without MRF / PHI with MRF",
                       "patchmatch_ms": pm_ms, "textureless_frac": float(flat.mean())},
            "rows": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


TABLE3 = [(5, 5), (5, 6), (6, 6), (5, 7), (7, 7), (5, 8), (8, 8), (5, 9), (9, 9), (5, 10), (10, 10)]
TABLE3_PAPER_S = {(5, 5): 9.79, (5, 6): 10.02, (6, 6): 12.58, (5, 7): 9.57, (7, 7): 16.41, (5, 8): 10.04,
                  (8, 8): 20.92, (5, 9): 10.51, (9, 9): 25.91, (5, 10): 10.86, (10, 10): 31.60}


def run_table3(args):
    """The paper's window-radius study (Sec. IV-B, Table III) on the
    high-resolution synthetic workload: for each (r_now, r_orig) the 8-
    iteration depth map (PatchMatch only, r_now samples per half side at
    spacing r_orig / r_now), its time and its completeness against the
    ground truth at 1 %, 2 % and 5 % relative depth error."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_06165_gb300 import mvs, scenes
    mvs.load()
    w = WORKLOAD
    sc = scenes.scene_highres(seed=rank, W=w["W"], H=w["H"], n_src=w["n_src"])
    H, W = sc.images[0].shape
    srcs = list(range(1, len(sc.images)))
    stream = torch.cuda.current_stream(dev)
    ctx = mvs.Context(sc.K, sc.R, sc.t, sc.images, stream=stream)
    plane = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    cost = torch.empty((H, W), dtype=torch.float32, device=dev)
    gt = sc.gt_depth
    rows = []
    with ClockSampler(local) as clk:
        for r_now, r_orig in TABLE3:
            p = mvs.PMParams(win_radius=float(r_orig), win_samples=2 * r_now + 1, sigma_s=w["sigma_s"],
                             sigma_c=w["sigma_c"], d_lo=2.0, d_hi=8.0, iters=w["iters"], seed=1 + rank)
            for _ in range(args.warmup):
                mvs.mvs_patchmatch(ctx.h, 0, srcs, p, plane, cost)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                mvs.mvs_patchmatch(ctx.h, 0, srcs, p, plane, cost)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            d = plane[..., 3].cpu().numpy()
            err = np.abs(d - gt) / np.where(gt > 0, gt, 1.0)
            rows.append({"r_now": r_now, "r_orig": r_orig, "ms": ms, "mpix_s": H * W / 1e3 / ms,
                         "completeness": {f"{t}%": float((err <= t / 100).mean()) for t in (1, 2, 5)},
                         "paper_time_s": TABLE3_PAPER_S[(r_now, r_orig)]})
    base = rows[0]["ms"]
    for r in rows:
        r["time_vs_5_5"] = r["ms"] / base
    line = {"metric": "depth-map Mpix/s per window configuration (Table III study)",
            "value": rows[3]["mpix_s"], "unit": "Mpix/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rows[3]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"table3 {W}x{H} uint8 ref + {len(srcs)} sources, 8 iterations, PatchMatch "
                                   "only; value = the paper's 5/7 setting",
                       "paper_hardware": "RTX 3070, ETH3D training scenes at 3024x2016 (context only)"},
            "rows": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per pixel group of the ZNCC kernels (0 = default)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"],
                    help="fp32 = FP32 ZNCC; mixed = half2 bilinear, FP32 moments, FP64 near-flat denominators")
    ap.add_argument("--workload", default="highres", choices=sorted(WORKLOADS),
                    help="highres = the measured workload; mid = 1536x1024 case for profiler captures; "
                         "batch24 = 24 views in one graph; learned = learned proposals vs plain 8 iterations; "
                         "table3 = the paper's window-radius study; sparse = sparse-feature initialisation "
                         "vs random by iteration count; table1 = PatchMatch alone vs PHI without / with the MRF; "
                         "pipeline = the whole Algorithm 1 on the 24-view scene")
    args = ap.parse_args()
    WORKLOAD.update(WORKLOADS[args.workload])
    studies = ("batch24", "learned", "table3", "sparse", "table1", "pipeline")
    if args.impl != "reference" and args.workload in studies and _env_rank()[0] != 0:
        return   # the single-GPU studies run on rank 0 only; the other ranks exit without work
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch24":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "combined":
        run_combined(args)
    elif args.workload == "table3":
        run_table3(args)
    elif args.workload == "sparse":
        run_sparse(args)
    elif args.workload == "table1":
        run_table1(args)
    elif args.workload == "pipeline":
        run_pipeline(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
