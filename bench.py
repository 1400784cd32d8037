#!/usr/bin/env python
"""End-to-end throughput of GMM superpixel EM (Ban, Liu, Cao, arXiv 1612.08792) on one GB300.

Headline line (default, `--workload learned481`): the learned initialiser
against plain EM at equal log-likelihood.  A step is Algorithm 1 on a batch
of 256 held-out synthetic 481x321 sRGB images (150 Voronoi regions, noise
sigma 8, seeds 1,000,000 + i) at spacing 15: CIELAB conversion, the trained
network's theta_0, 2 EM iterations (fused E-step + M-step partial sums, FP64
finalize with the eigenvalue floor), label pass -- one CUDA-graph launch of
the batch context.  The same images also run through plain EM (Sec. III-C
start, 10 iterations) for the ratio and the log-likelihood comparison.
`value` is device time with the images already in HBM and L2 flushed
(256 MiB memset) between timed steps; `e2e` adds the pinned host->device copy
of the images and the device->host copy of the labels.

Other lines: `--workload 481x321` (one image, K = 1000 -> v = 12, plain EM,
10 iterations), `batch256` (256 images of uneven sizes), `3840x2160`.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmmsp|reference] [--workload ...]

With N > 1 (torchrun) each rank runs an independent replica on its own images
(no collective on the data path: the images are independent problems);
`value` is all ranks' pixels over the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s end-to-end superpixels, learned-init vs plain EM at equal log-lik"
UNIT = "Mpixel/s"
W, H, K_REQ, ITERS, REGIONS, SIGMA = 481, 321, 1000, 10, 150, 8.0
FLUSH_BYTES = 256 << 20
# Algorithmic FP32 work of the fused E + M-partial pass, per (pixel, candidate):
#   E: d = z - mu (5), block quadratic form (9 products, 9 multiply-adds = 27 minus
#      the shared products folded: 23), log-normaliser add (1)              -> 28
#   log-sum-exp: max, subtract, add, normalise                              ->  4
#   M: W += R, R d (5), S1 += R d (5), 9 second-moment multiply-adds (18)   -> 29
# plus per pixel 1 (log-likelihood add); 1 MUFU ex2 per candidate, 2 per pixel.
FLOPS_PER_CAND = 61
FLOPS_PER_PIXEL = 1
# FP32 peak derived from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# The binding roofline of the E + M pass is the FP32 pipe's instruction rate (most of
# its operations are single adds and multiplies, so flops understate the work):
# algorithmic FP32-pipe lane-instructions per (pixel, candidate), from the formulas --
#   E: d = z - mu (5), the two quadratic forms (14), running max (1), exponent
#      shift (1), sum (1), normalisation (1)                                  -> 23
#   M: d = z - mu_old (5), W += R (1), R d (5), S1 += R d (5), the 9 block
#      second moments (9)                                                      -> 25
# plus 2 per pixel (log-likelihood adds); MUFU (ex2 per candidate, rcp and lg2 per
# pixel) runs on its own pipe.  Peak: 152 SMs x 128 FP32 lanes x 2.07 GHz.
INSTR_PER_CAND = 48
INSTR_PER_PIXEL = 2
FP32_PEAK_TINST = 152 * 128 * 2.070e9 / 1e12
# The same counts for the colour models (--colour, plain-EM lines):
#   split (Eq. BlockSigma1): no L-a, L-b terms -- E quadratic form 12 instead of 14,
#     M second moments 7 instead of 9                      -> 21 + 23 = 44 instructions
#     (flops: E 5 + 8 + 11 + 4, M 1 + 5 + 5 + 14            -> 53)
#   gray: z = (x, y, L) -- E d 3, quadratic forms 5 + 2, 4; M d 3, W 1, R d 3,
#     S1 3, second moments 4                                -> 14 + 14 = 28 instructions
#     (flops: E 3 + 8 + 3 + 4, M 1 + 3 + 3 + 8              -> 33)
INSTR_PER_CAND_MODEL = {"full": INSTR_PER_CAND, "split": 44, "gray": 28}
FLOPS_PER_CAND_MODEL = {"full": FLOPS_PER_CAND, "split": 53, "gray": 33}


# The E + M pass's other two rooflines, reported beside the binding FP32 one:
#   HBM: DRAM bytes per launch (ncu-measured where the launch variant was captured, else the
#        algorithmic 12 B of CIELAB per pixel plus the 544 B FP32 partial of every cell) over
#        the pass time, against the measured copy bandwidth of MEASURED_PEAKS.json;
#   MUFU (XU pipe): one ex2 per (pixel, candidate) and rcp + lg2 per pixel over the pass time,
#        against 152 SMs x 32 results per clock (the project probe's measured ex2 rate per SM)
#        x 2.07 GHz.
MUFU_PEAK_TOPS = 152 * 32 * 2.070e9 / 1e12
PARTIAL_BYTES_PER_CELL = 544


def side_rooflines(units, pixels, cells, em_ms, traffic):
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    algo = 12 * pixels + PARTIAL_BYTES_PER_CELL * cells
    nbytes = traffic if traffic else algo
    gbs = nbytes / (em_ms * 1e-3) / 1e9
    mufu = units + 2 * pixels
    tops = mufu / (em_ms * 1e-3) / 1e12
    return {"hbm": {"bytes_per_launch": int(nbytes), "bytes_source": "ncu dram bytes" if traffic else "algorithmic",
                    "algorithmic_bytes": int(algo), "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(gbs / hbm_peak, 4),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"},
            "mufu": {"ops_per_launch": int(mufu), "achieved": round(tops, 3), "peak": round(MUFU_PEAK_TOPS, 3),
                     "unit": "T MUFU results/s", "frac": round(tops / MUFU_PEAK_TOPS, 4),
                     "peak_source": "derived: 152 SMs x 32 ex2 per clock (measured per-SM rate) x 2.07 GHz"}}


def workload_config(v, nx, ny, K):
    return {
        "workload": f"{W}x{H} synthetic Voronoi sRGB ({REGIONS} regions, noise sigma {SIGMA:g}), "
                    f"K={K_REQ} requested -> v={v}, K={K}; {ITERS} plain-EM iterations (Sec. III-C init)",
        "W": W, "H": H, "K": K, "v": v, "nx": nx, "ny": ny, "iters": ITERS,
        "precision": "FP32 E-step and per-cell sums, FP64-accurate superpixel sums (FP32 TwoSum pairs), FP64 update / floor / inversion",
        "l2": "flushed between timed steps (256 MiB memset, outside the timed interval)",
        "init": "plain",
    }


def candidate_units(Wd, Hd, v, nx, ny):
    """sum over pixels of |K_i|: candidates along x times candidates along y."""
    def axis(extent, n):
        tot = 0
        for p in range(extent):
            c = min(p // v, n)  # cell index (remainder strip -> n)
            tot += sum(1 for kq in (c - 1, c, c + 1) if 0 <= kq < n)
        return tot
    return axis(Wd, nx) * axis(Hd, ny)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(", ") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over the ranks of the default process group (x itself when alone)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank: int, n: int):
    """Held-out image seeds of one replica: each rank its own n images."""
    return range(HELD_OUT0 + rank * n, HELD_OUT0 + (rank + 1) * n)


def whole_job_value(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput in millions of units per second: all ranks' units over the
    slowest rank's time (the ranks do equal, independent work)."""
    return world * units_per_rank / max_seconds / 1e6


def cpu_oracle_run(seconds: float, seed: int = 0):
    """The FP64 CPU oracle as it stands (RGB -> CIELAB -> EM -> labels), on all host
    threads, repeated for about `seconds`.  Returns (Mpixel/s, threads, reps)."""
    import oracle
    from synth import voronoi_image
    img = voronoi_image(W, H, REGIONS, SIGMA, seed)
    threads = oracle.max_threads()
    reps = 0
    t0 = time.perf_counter()
    while True:
        lab = oracle.rgb2lab(img)
        oracle.em(lab, W, H, K=K_REQ, T=ITERS)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return W * H * reps / el / 1e6, threads, reps, el


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    from synth import voronoi_image
    img = voronoi_image(W, H, REGIONS, SIGMA, 0)
    g = oracle.grid(W, H, K_REQ)
    for _ in range(args.warmup):
        oracle.em(oracle.rgb2lab(img), W, H, K=K_REQ, T=ITERS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.em(oracle.rgb2lab(img), W, H, K=K_REQ, T=ITERS)
    el = time.perf_counter() - t0
    value = W * H * args.steps / el / 1e6
    threads = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(g.v, g.nx, g.ny, g.K),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps of one {W}x{H} image, RGB->labels, FP64 C oracle "
                                   f"(OpenMP, {threads} threads)"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gmmsp(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    from synth import voronoi_image

    img_np = voronoi_image(W, H, REGIONS, SIGMA, seed=rank)
    img_host = torch.from_numpy(img_np).pin_memory()
    img_dev = img_host.to("cuda")
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
    sp = gm.Superpixels(img_dev, K=K_REQ, stream=stream)
    v, nx, ny, K = sp.grid.v, sp.grid.nx, sp.grid.ny, sp.grid.K
    N = W * H
    with torch.cuda.stream(stream):
        sp.em_iters(2)
        wpc, tune_ms = sp.autotune(reps=10)  # launch shape of the E + M pass

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            sp.segment(img_dev, ITERS, out=labels)
    stream.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(i & 0xff)
                starts[i].record(stream)
                sp.segment(img_dev, ITERS, out=labels)
                ends[i].record(stream)
        torch.cuda.synchronize()
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * N * args.steps / (total_ms / 1e3) / 1e6

    # log-likelihood of the timed configuration (for the equal-log-lik comparison)
    with torch.cuda.stream(stream):
        _, ll = sp.segment(img_dev, ITERS, out=labels, want_loglik=True)

    # end to end through the public API with host buffers
    labels_host = torch.empty((H, W), dtype=torch.int32).pin_memory()
    dev_img2 = torch.empty_like(img_dev)
    for _ in range(3):
        sp.segment_host(img_host, labels_host, ITERS, dev_image=dev_img2, dev_labels=labels)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sp.segment_host(img_host, labels_host, ITERS, dev_image=dev_img2, dev_labels=labels)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = world * N * args.steps / e2e_s / 1e6

    # roofline of the dominant kernel (fused E + M-partial pass), events on its stream;
    # the other kernels' launch times for the breakdown
    # In-pipeline breakdown: the same graph with event nodes between the kernels
    # (slightly slower than the timed graph; used for the per-kernel shares).
    with torch.cuda.stream(stream):
        sp.set_timing(True)
        pipe = []
        for i in range(20):
            flush.fill_(i & 0xff)
            sp.segment(img_dev, ITERS, out=labels)
            pipe.append(sp.get_timing())
        sp.set_timing(False)
        pipe = [sum(x) / len(x) for x in zip(*pipe)]
        em_pipe = sum(pipe[1:1 + 2 * ITERS:2]) / ITERS
        fin_pipe = sum(pipe[2:2 + 2 * ITERS:2]) / ITERS
        sp.segment(img_dev, ITERS, out=labels)
        em_ms = sp.profile_kernel(gm.GMMSP_KERNEL_EM_PASS, reps=50, flush=flush)
        fin_ms = sp.profile_kernel(gm.GMMSP_KERNEL_FINALIZE, reps=50, flush=flush)
        lab_ms = sp.profile_kernel(gm.GMMSP_KERNEL_LABELS, reps=50, labels=labels, flush=flush)
        em_warm = sp.profile_kernel(gm.GMMSP_KERNEL_EM_PASS, reps=50)
    units = candidate_units(W, H, v, nx, ny)
    flops = units * FLOPS_PER_CAND + N * FLOPS_PER_PIXEL
    achieved = flops / (em_pipe * 1e-3) / 1e12
    instr = units * INSTR_PER_CAND + N * INSTR_PER_PIXEL
    achieved_i = instr / (em_pipe * 1e-3) / 1e12
    sp.close()

    launches_per_step = 2 + 2 * ITERS + 1  # rgb2lab, init, (em_pass, finalize) x T, labels
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic", "config": dict(workload_config(v, nx, ny, K), parallelism=f"replicas x{world}",
                                            warps_per_cell=wpc),
        "loglik_final": float(ll[-1]), "loglik_per_pixel": float(ll[-1]) / N,
        "roofline": {"kernel": "k_em_pass (fused E-step + M-step partials)", "bound": "alu",
                     "achieved": round(achieved_i, 3), "peak": round(FP32_PEAK_TINST, 3),
                     "unit": "T FP32-lane-instr/s", "frac": round(achieved_i / FP32_PEAK_TINST, 4), "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (one FP32 instruction per "
                                    "lane per clock)",
                     "em_pass_ms": round(em_pipe, 5), "instr_per_launch": instr,
                     "flops": {"achieved_tflops": round(achieved, 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                               "frac": round(achieved / FP32_PEAK_TFLOPS, 4)},
                     "timing": "mean E+M pass duration inside the step (event nodes in the graph)"},
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": N * 3,
                "d2h_bytes_per_step": N * 4},
        "gpu_launches": launches_per_step * args.steps,
        "kernel_ms": {"in_step": {"prepare": round(pipe[0], 5), "em_pass": round(em_pipe, 5),
                                  "finalize": round(fin_pipe, 5), "labels": round(pipe[-1], 5),
                                  "sum": round(sum(pipe), 5)},
                      "cold_l2": {"em_pass": round(em_ms, 5), "finalize": round(fin_ms, 5),
                                  "labels": round(lab_ms, 5)},
                      "warm_repeat": {"em_pass": round(em_warm, 5)},
                      "em_pass_autotune": {str(k): round(v_, 5) for k, v_ in tune_ms.items()}},
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mpx, threads, reps, el = cpu_oracle_run(args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(mpx, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{reps} runs of the {W}x{H} workload (RGB->labels, T={ITERS}) "
                                          f"in {el:.1f} s, FP64 C oracle, OpenMP {threads} threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _timed_steps(step, stream, steps, flush, clk_index):
    """Per-step CUDA-event times (ms) with L2 flushed before every step, and the clock record."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    with ClockSampler(clk_index) as clk:
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.fill_(i & 0xff)
                starts[i].record(stream)
                step()
                ends[i].record(stream)
        torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)], clk.summary()


def run_other_workload(args):
    """Secondary workloads (not the headline line): `batch256` -- 256 images of
    uneven sizes in one batch context -- and `3840x2160` -- one 4K image."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    from synth import voronoi_image
    from synth.voronoi import batch_regions, batch_sizes
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    if args.workload == "batch256":
        sizes = batch_sizes(256)
        cache = {}
        imgs = []
        for i, (Wi, Hi) in enumerate(sizes):  # 4 distinct seeded images per size, reused
            key = (Wi, Hi, i % 4)
            if key not in cache:
                cache[key] = torch.from_numpy(voronoi_image(Wi, Hi, batch_regions(Wi, Hi), 8.0, seed=i % 4)).cuda()
            imgs.append(cache[key])
        with torch.cuda.stream(stream):
            bt = gm.SuperpixelsBatch([(h, w) for (w, h) in sizes], spacing=15, stream=stream, colour=args.colour)
            bps, tune = bt.autotune(imgs, reps=3)
        pix, K, cells = bt.info()
        cells_total = cells
        em_ms = tune[bps]
        units = sum(candidate_units(w, h, 15, w // 15, h // 15) for (w, h) in sizes)
        step = lambda: bt.segment(imgs, ITERS)
        for _ in range(max(args.warmup, 3)):
            with torch.cuda.stream(stream):
                step()
        step_ms, clocks = _timed_steps(step, stream, args.steps, flush, 0)
        with torch.cuda.stream(stream):
            _, ll = bt.segment(imgs, ITERS, want_loglik=True)
        config = {"workload": f"batch of 256 synthetic Voronoi sRGB images, sizes uniform over "
                              f"320x240/481x321/640x480/1280x720/1920x1080 (regions proportional to area, "
                              f"sigma 8), spacing 15, {ITERS} plain-EM iterations, one batch context, "
                              f"{args.colour} colour covariance",
                  "images": 256, "pixels": pix, "K": K, "cells": cells, "blocks_per_sm": bps,
                  "colour_model": args.colour,
                  "l2": "flushed between timed steps (256 MiB memset)"}
        launches = 2 + 2 * ITERS + 1
        extra = {"loglik_mean_per_pixel": float(np.sum(ll)) / pix, "em_pass_autotune_ms": tune}
        bt.close()
    else:
        Wd, Hd = 3840, 2160
        img = torch.from_numpy(voronoi_image(Wd, Hd, 2000, 6.0, seed=0)).cuda()
        labels = torch.empty((Hd, Wd), dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream):
            sp = gm.Superpixels(img, K=20000, stream=stream, colour=args.colour)
            sp.em_iters(2)
            wpc, _ = sp.autotune(reps=3)
        v, nx, ny, K = sp.grid.v, sp.grid.nx, sp.grid.ny, sp.grid.K
        pix = Wd * Hd
        cells_total = -(-Wd // v) * -(-Hd // v)
        step = lambda: sp.segment(img, ITERS, out=labels)
        for _ in range(max(args.warmup, 3)):
            with torch.cuda.stream(stream):
                step()
        step_ms, clocks = _timed_steps(step, stream, args.steps, flush, 0)
        with torch.cuda.stream(stream):
            _, ll = sp.segment(img, ITERS, out=labels, want_loglik=True)
            em_ms = sp.profile_kernel(gm.GMMSP_KERNEL_EM_PASS, reps=10)
            fin_ms = sp.profile_kernel(gm.GMMSP_KERNEL_FINALIZE, reps=10)
        units = candidate_units(Wd, Hd, v, nx, ny)
        config = {"workload": f"{Wd}x{Hd} synthetic Voronoi sRGB (2000 regions, sigma 6), K=20000 requested "
                              f"-> v={v}, K={K}; {ITERS} plain-EM iterations, {args.colour} colour covariance",
                  "W": Wd, "H": Hd, "K": K, "v": v, "colour_model": args.colour,
                  "warps_per_cell": wpc, "l2": "flushed between timed steps (256 MiB memset)"}
        launches = 2 + 2 * ITERS + 1
        extra = {"loglik_per_pixel": float(ll[-1]) / pix, "kernel_ms": {"em_pass": em_ms, "finalize": fin_ms}}
        sp.close()
    ms = sum(step_ms) / len(step_ms)
    flops = units * FLOPS_PER_CAND_MODEL[args.colour] + pix * FLOPS_PER_PIXEL
    achieved = flops / (em_ms * 1e-3) / 1e12
    instr = units * INSTR_PER_CAND_MODEL[args.colour] + pix * INSTR_PER_PIXEL
    achieved_i = instr / (em_ms * 1e-3) / 1e12
    line = {"metric": METRIC, "value": round(pix / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic", "config": config,
            "roofline": {"kernel": "E + M-partial pass", "bound": "alu", "achieved": round(achieved_i, 3),
                         "peak": round(FP32_PEAK_TINST, 3), "unit": "T FP32-lane-instr/s",
                         "frac": round(achieved_i / FP32_PEAK_TINST, 4), "traffic": None,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                         "em_pass_ms": round(em_ms, 4), "instr_per_launch": instr,
                         "flops": {"achieved_tflops": round(achieved, 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                                   "frac": round(achieved / FP32_PEAK_TFLOPS, 4)},
                         **side_rooflines(units, pix, cells_total, em_ms, None)},
            "gpu_launches": launches * args.steps, "clocks": clocks, **extra}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- learned start
LEARN_IMAGES, LEARN_V, LEARN_T, HELD_OUT0 = 256, 15, 2, 1_000_000
# Algorithmic tensor-core work of the network per 481 x 321 image at spacing 15
# (32 x 21 cells, 5 x 5 patches each): two 1 x 1 layers per patch (27 -> 32,
# 32 -> 32) and four 3 x 3 layers per cell (288 -> 32 three times, 288 -> 16).
E2E_CONTEXTS = 3  # batch contexts taking the end-to-end steps in turn
NET_FLOPS_PER_PATCH = 2 * (27 * 32 + 32 * 32)
NET_FLOPS_PER_CELL = 2 * (3 * 288 * 32 + 288 * 16)
# DRAM bytes per 481 x 321 image of one batched E + M pass, from an ncu capture on
# 96 such images (dram__bytes_read.sum + dram__bytes_write.sum), scaled per image
# (traffic grows with the image count), per launch variant (blocks per SM); a variant
# not captured with the current kernel reports null.
#   7: one-cell-per-warp k_em_pass_batch_flat capped at 72 registers: 182.06 MB + 29.63 MB.
EM_BATCH_TRAFFIC_PER_IMAGE = {7: int((182.059520e6 + 29.629184e6) / 96)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def learned_config(n, bps):
    return {
        "workload": f"{n} held-out synthetic {W}x{H} Voronoi sRGB images per step ({REGIONS} regions, noise "
                    f"sigma {SIGMA:g}, seeds {HELD_OUT0}+i), spacing {LEARN_V} (32x21 = 672 superpixels); "
                    f"learned theta_0 + {LEARN_T} EM iterations vs the Sec. III-C start + {ITERS} iterations",
        "images": n, "W": W, "H": H, "v": LEARN_V, "K": 672, "iters_learned": LEARN_T, "iters_plain": ITERS,
        "network": "6-layer conv initialiser, BF16 weights/activations, FP32 accumulation (tcgen05)",
        "precision": "FP32 E-step and per-cell sums, FP64-accurate superpixel sums (FP32 TwoSum pairs), FP64 update / floor / inversion",
        "l2": "flushed between timed steps (256 MiB memset, outside the timed interval); inputs > L2",
        "blocks_per_sm": bps,
    }


def oracle_learned_sample(weights, seconds, seed0=HELD_OUT0):
    """The oracle as it stands on the learned workload: FP64 CIELAB, the FP64
    network, its theta_0 and 2 EM iterations, image after image until about
    `seconds` of that work (image generation not counted).  Returns
    (Mpixel/s, threads, images, seconds)."""
    import oracle
    from oracle import cnn as ocnn
    from synth import voronoi_image
    threads = oracle.max_threads()
    n, el = 0, 0.0
    while True:
        img = voronoi_image(W, H, REGIONS, SIGMA, seed0 + n)
        t0 = time.perf_counter()
        lab = oracle.rgb2lab(img)
        planes = lab.transpose(2, 0, 1)
        out, _ = ocnn.forward(weights, planes[None], LEARN_V)
        mu, cs, cc = ocnn.theta0_from_outputs(out[0].reshape(-1, 16), planes, LEARN_V)
        oracle.em(lab, W, H, spacing=LEARN_V, T=LEARN_T, theta0=oracle.Theta(mu, cs, cc))
        el += time.perf_counter() - t0
        n += 1
        if el >= seconds:
            break
    return W * H * n / el / 1e6, threads, n, el


def run_learned(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    from paper_1612_08792_gb300.learned_init import load_pretrained, pretrained_path
    from synth.voronoi_torch import voronoi_batch

    n = args.images
    N = W * H
    seeds = replica_seeds(rank, n)
    regs = torch.empty((n, H, W), dtype=torch.int32, device="cuda")  # the generator's regions (ground truth)
    buf = voronoi_batch(W, H, REGIONS, SIGMA, seeds, regions_out=regs)
    imgs = [buf[i] for i in range(n)]
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        net = load_pretrained(LEARN_V, stream=stream)
        plain = gm.SuperpixelsBatch([(H, W)] * n, spacing=LEARN_V, stream=stream)
        bps, tune = plain.autotune(imgs, reps=3)
        learned = gm.SuperpixelsBatch([(H, W)] * n, spacing=LEARN_V, stream=stream)
        learned.autotune(imgs, reps=3)
        learned.set_launch(bps)
        learned.set_init_net(net)
        tuning = {"plain": plain.tuning(), "learned": learned.tuning(),
                  "em_pass_ms_by_blocks_per_sm": {str(k): round(v_, 5) for k, v_ in tune.items()}}
    step_l = lambda: learned.segment(imgs, LEARN_T)  # noqa: E731
    step_p = lambda: plain.segment(imgs, ITERS)  # noqa: E731
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step_l()
            step_p()
    stream.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    barrier()
    ms_l, clocks = _timed_steps(step_l, stream, args.steps, flush, local)
    barrier()
    ms_p, clocks_p = _timed_steps(step_p, stream, max(3, args.steps // 3), flush, local)
    barrier()
    t_l = max_over_ranks(sum(ms_l) / len(ms_l), world)
    t_p = max_over_ranks(sum(ms_p) / len(ms_p), world)
    value = whole_job_value(world, n * N, t_l * 1e-3)
    plain_value = whole_job_value(world, n * N, t_p * 1e-3)

    # log-likelihood (equal-log-lik check) and label agreement with plain EM
    with torch.cuda.stream(stream):
        lab_l, ll_l = learned.segment(imgs, LEARN_T, want_loglik=True)
        lab_l = [x.clone() for x in lab_l]
        lab_p, ll_p = plain.segment(imgs, ITERS, want_loglik=True)
        agree = float(sum(int((a == b).sum().item()) for a, b in zip(lab_l, lab_p))) / (n * N)
        _, ll_p2 = plain.segment(imgs, LEARN_T, want_loglik=True)
    llpp_l, llpp_p, llpp_p2 = (float(np.mean(x)) / N for x in (ll_l, ll_p, ll_p2))
    gap = abs(llpp_l - llpp_p) / abs(llpp_p)

    # Plain EM at every iteration count T = 2..10 and the learned start at T = 1..3 on the same
    # images: device time per step (L2 flushed), log-likelihood per pixel, and the accuracy of
    # Sec. IV (BR, UE, ASA) against the generator's regions.  The learned start's real gain is
    # its speed-up over the cheapest plain run within 0.5 % of plain EM's log-likelihood at T = 10.
    sweep = {}
    regions = [regs[i] for i in range(n)]
    for kind, ctx, Ts in (("plain", plain, range(2, ITERS + 1)), ("learned", learned, (1, 2, 3))):
        for T in Ts:
            step_t = lambda: ctx.segment(imgs, T)  # noqa: E731
            with torch.cuda.stream(stream):
                step_t()
            ms_t, _ = _timed_steps(step_t, stream, 3, flush, local)
            with torch.cuda.stream(stream):
                labels_t, ll_t = ctx.segment(imgs, T, want_loglik=True)
            mets = gm.gmmsp_segmentation_metrics_many(labels_t, regions, 672, REGIONS, stream=stream)
            sweep[f"{kind}_{T}"] = {"iters": T, "ms_per_step": round(float(np.median(ms_t)), 4),
                                    "loglik_per_pixel": float(np.mean(ll_t)) / N,
                                    **{k: round(float(np.mean([m[k] for m in mets])), 6) for k in ("br", "ue", "asa")}}
    ll10 = sweep[f"plain_{ITERS}"]["loglik_per_pixel"]
    within = [T for T in range(2, ITERS + 1)
              if abs(sweep[f"plain_{T}"]["loglik_per_pixel"] - ll10) / abs(ll10) <= 0.005]
    t_eq = min(within)
    same_time = max([T for T in range(2, ITERS + 1)
                     if sweep[f"plain_{T}"]["ms_per_step"] <= sweep[f"learned_{LEARN_T}"]["ms_per_step"]],
                    default=None)
    ll_learned = sweep[f"learned_{LEARN_T}"]["loglik_per_pixel"]
    t_match = min([T for T in range(2, ITERS + 1) if sweep[f"plain_{T}"]["loglik_per_pixel"] >= ll_learned],
                  default=None)
    plain_sweep = {
        "runs": sweep,
        "plain_iters_matching_learned_loglik": t_match,
        "learned_speedup_vs_plain_at_its_loglik": (round(sweep[f"plain_{t_match}"]["ms_per_step"] /
                                                         sweep[f"learned_{LEARN_T}"]["ms_per_step"], 3)
                                                   if t_match else None),
        "plain_iters_within_0.5pct_of_plain_10": t_eq,
        "learned_speedup_vs_that_plain": round(sweep[f"plain_{t_eq}"]["ms_per_step"] /
                                               sweep[f"learned_{LEARN_T}"]["ms_per_step"], 3),
        "plain_iters_at_learned_time": same_time,
        "how": "same images as the headline step; 3 timed steps per run (median), L2 flushed before each; "
               "BR (2 px), UE (eps 0.05), ASA against the generator's Voronoi regions",
    }

    # the network alone (events on its stream) and the E + M pass at the chosen launch shape
    lab_ptr = learned.lab_ptr()
    with torch.cuda.stream(stream):
        learned.segment(imgs, LEARN_T)
        out = net.forward(lab_ptr, n, W, H)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        e0.record(stream)
        reps = 20
        for _ in range(reps):
            gm.gmmsp_net_forward(net.n, lab_ptr, n, W, H, out)
        e1.record(stream)
    stream.synchronize()
    net_ms = e0.elapsed_time(e1) / reps
    net.check()
    net_flops = n * (672 * 25 * NET_FLOPS_PER_PATCH + 672 * NET_FLOPS_PER_CELL)
    em_ms = tune[bps]
    units = n * candidate_units(W, H, LEARN_V, W // LEARN_V, H // LEARN_V)
    flops = units * FLOPS_PER_CAND + n * N * FLOPS_PER_PIXEL
    achieved = flops / (em_ms * 1e-3) / 1e12
    instr = units * INSTR_PER_CAND + n * N * INSTR_PER_PIXEL
    achieved_i = instr / (em_ms * 1e-3) / 1e12

    # end to end through the public API: pinned host images in, host labels out.
    # E2E_CONTEXTS batch contexts (each with its network copy and stream) take steps in
    # turn, so that one step's host copies overlap the others' kernels; every step still copies its own
    # images in and its labels out, each as one copy (the images stacked in one tensor, the
    # labels in the context's one buffer).  The serial form (one context, copy - segment -
    # copy) is reported beside it.
    host_imgs = buf.cpu().pin_memory()
    t1 = learned.tuning()
    extra = []  # (stream, net, context) of the contexts beyond the first
    for _ in range(E2E_CONTEXTS - 1):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            net_x = load_pretrained(LEARN_V, stream=st)
            ctx_x = gm.SuperpixelsBatch([(H, W)] * n, spacing=LEARN_V, stream=st)
            gm.gmmsp_batch_set_tuning(ctx_x.b, t1["blocks_per_sm"], t1["finalize16"])
            ctx_x.set_init_net(net_x)
        extra.append((st, net_x, ctx_x))
    slots = []
    for ctx, st in [(learned, stream)] + [(c, st) for st, _, c in extra]:
        slots.append(dict(ctx=ctx, stream=st, dev_in=torch.empty_like(buf),
                          host_labels=torch.empty(n * H * W, dtype=torch.int32).pin_memory(),
                          done=torch.cuda.Event()))

    def e2e_issue(slot):
        # one copy in (the n images, stacked), the segment, one copy out (the labels buffer)
        with torch.cuda.stream(slot["stream"]):
            slot["dev_in"].copy_(host_imgs, non_blocking=True)
            slot["ctx"].segment_stacked(slot["dev_in"], LEARN_T)
            slot["host_labels"].copy_(slot["ctx"].labels_buffer, non_blocking=True)
            slot["done"].record(slot["stream"])

    def e2e_run(steps, pipelined):
        for k in range(steps):
            slot = slots[k % len(slots)] if pipelined else slots[0]
            slot["done"].synchronize()      # its previous step (labels on the host) is complete
            e2e_issue(slot)
        for slot in slots:
            slot["done"].synchronize()

    e2e_steps = max(4, args.steps // 4)
    e2e_run(4, True)
    barrier()
    with ClockSampler(local) as clk_e2e:
        t0 = time.perf_counter()
        e2e_run(e2e_steps, True)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = whole_job_value(world, n * N * e2e_steps, e2e_s)
    barrier()
    t0 = time.perf_counter()
    e2e_run(e2e_steps, False)
    e2e_serial = whole_job_value(world, n * N * e2e_steps, max_over_ranks(time.perf_counter() - t0, world))
    for _, net_x, ctx_x in extra:
        ctx_x.close()
        net_x.close()

    peaks = measured_peaks()
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    net_tflops = net_flops / (net_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(t_l, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 (EM), bf16 (net)",
        "data": "synthetic", "config": dict(learned_config(n, bps), parallelism=f"replicas x{world}"),
        "plain_em": {"value": round(plain_value, 3), "unit": UNIT, "ms_per_step": round(t_p, 5),
                     "iters": ITERS, "steps": len(ms_p)},
        "speedup_vs_plain": round(value / plain_value, 3),
        "loglik_per_pixel": {"learned": llpp_l, "plain": llpp_p, f"plain_{LEARN_T}_iters": llpp_p2,
                             "rel_gap": gap, "target": 0.005},
        "label_agreement_with_plain": round(agree, 5),
        "plain_sweep": plain_sweep,
        "roofline": {"kernel": "k_em_pass_batch (fused E-step + M-step partials)", "bound": "alu",
                     "achieved": round(achieved_i, 3), "peak": round(FP32_PEAK_TINST, 3),
                     "unit": "T FP32-lane-instr/s", "frac": round(achieved_i / FP32_PEAK_TINST, 4),
                     "traffic": EM_BATCH_TRAFFIC_PER_IMAGE[bps] * n if bps in EM_BATCH_TRAFFIC_PER_IMAGE else None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (one FP32 instruction per "
                                    "lane per clock)",
                     "em_pass_ms": round(em_ms, 5), "instr_per_launch": instr,
                     "flops": {"achieved_tflops": round(achieved, 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                               "frac": round(achieved / FP32_PEAK_TFLOPS, 4)},
                     "timing": "batch E+M pass alone, mean of repeated launches (autotuner)",
                     **side_rooflines(units, n * N, n * 726, em_ms,
                                      EM_BATCH_TRAFFIC_PER_IMAGE[bps] * n if bps in EM_BATCH_TRAFFIC_PER_IMAGE
                                      else None)},
        "tuning": tuning,
        "net_roofline": {"kernels": "k_pix + 4 x k_gemm (forward)", "bound": "tensor",
                         "achieved": round(net_tflops, 3), "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": round(net_tflops / bf16_peak, 5), "ms": round(net_ms, 5),
                         "flops_per_launch": net_flops,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" if peaks else "fallback"},
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": n * N * 3,
                "d2h_bytes_per_step": n * N * 4,
                "how": f"{E2E_CONTEXTS} batch contexts on as many streams take steps in turn (copies of one "
                       "step overlap the kernels of the others); each step copies its images in (one copy of the stacked "
                       "images) and its labels out (one copy of the context's label buffer)",
                "serial": round(e2e_serial, 3), "clocks": clk_e2e.summary()},
        "gpu_launches": (1 + 5 + 1 + 2 * LEARN_T + 1) * args.steps,
        "clocks": clocks, "clocks_plain": clocks_p,
        "weights": os.path.relpath(pretrained_path(LEARN_V), ROOT),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        w = np.load(pretrained_path(LEARN_V))["weights"]
        mpx, threads, imgs_done, el = oracle_learned_sample(w, args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(mpx, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{imgs_done} held-out images of the workload in {el:.1f} s (FP64 CIELAB, "
                                          f"FP64 network, theta_0, {LEARN_T} EM iterations, labels; C oracle "
                                          f"with OpenMP {threads} threads, numpy network)"}
    learned.close()
    plain.close()
    net.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_reference_learned(args):
    """The oracle on the learned workload, each step one held-out image."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_1612_08792_gb300.learned_init import pretrained_path
    w = np.load(pretrained_path(LEARN_V))["weights"]
    oracle_learned_sample(w, 0.0, HELD_OUT0 + 10_000)      # warm-up (one image)
    el = 0.0
    for i in range(args.steps):
        el += oracle_learned_sample(w, 0.0, HELD_OUT0 + i)[3]
    import oracle
    threads = oracle.max_threads()
    value = W * H * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": learned_config(1, None),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps of one held-out {W}x{H} image each (FP64 CIELAB, FP64 "
                                   f"network, theta_0, {LEARN_T} EM iterations, labels)"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """A short run for ncu captures: the bench workload, 4 EM iterations and the
    label pass, no timing (`--profile-case`)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    from synth import voronoi_image
    if args.workload == "learned481":
        # `--images` held-out images through the learned start + 2 iterations, twice
        from paper_1612_08792_gb300.learned_init import load_pretrained
        from synth.voronoi_torch import voronoi_batch
        buf = voronoi_batch(W, H, REGIONS, SIGMA, range(HELD_OUT0, HELD_OUT0 + args.images))
        imgs = [buf[i] for i in range(args.images)]
        net = load_pretrained(LEARN_V)
        bt = gm.SuperpixelsBatch([(H, W)] * args.images, spacing=LEARN_V)
        bt.autotune(imgs, reps=2)  # the launch choices of the timed step
        if args.blocks_per_sm:
            bt.set_launch(args.blocks_per_sm, first_pass=args.first_pass if args.first_pass else None)
        bt.set_init_net(net)
        for _ in range(2):
            bt.segment(imgs, LEARN_T)
        torch.cuda.synchronize()
        net.check()
        bt.close()
        net.close()
        print("profile case done", args.images)
        return 0
    if args.workload == "conn256":
        stream = torch.cuda.Stream()
        bt, _ = _conn_case(gm, torch, args.images, stream)
        st = bt.connectivity()
        bt.close()
        print("profile case done", st)
        return 0
    if args.workload == "3840x2160":
        img = torch.from_numpy(voronoi_image(3840, 2160, 2000, 6.0, seed=0)).cuda()
        sp = gm.Superpixels(img, K=20000, colour=args.colour)
    else:
        img = torch.from_numpy(voronoi_image(W, H, REGIONS, SIGMA, seed=0)).cuda()
        sp = gm.Superpixels(img, K=K_REQ)
    if args.warps_per_cell:
        sp.set_launch(args.warps_per_cell)
    sp.em_iters(4)
    labels = sp.labels()
    torch.cuda.synchronize()
    sp.close()
    print("profile case done", tuple(labels.shape))
    return 0

# Algorithmic DRAM bytes per pixel of the connectivity post-processing: the input
# labels (4 B) and CIELAB colour (12 B) read once, the output labels (4 B) written.
CONN_BYTES_PER_PIXEL = 20
CONN_LAUNCHES = 21  # kernels of one gmmsp_batch_connectivity call


def _conn_case(gm, torch, n, stream, keep_images=False, regions=None):
    """n held-out 481x321 images (v = 15) segmented by 10 plain-EM iterations in one batch
    context: the label maps the connectivity post-processing (and the accuracy metrics) work
    on.  regions: an (n, H, W) int32 tensor that receives the generator's region maps."""
    from synth.voronoi_torch import voronoi_batch
    buf = voronoi_batch(W, H, REGIONS, SIGMA, range(HELD_OUT0, HELD_OUT0 + n), regions_out=regions)
    imgs = [buf[i] for i in range(n)]
    with torch.cuda.stream(stream):
        bt = gm.SuperpixelsBatch([(H, W)] * n, spacing=LEARN_V, stream=stream)
        bt.segment(imgs, ITERS)
    stream.synchronize()
    before = [x.clone() for x in bt.labels]
    return (bt, before, buf) if keep_images else (bt, before)


def conn_oracle_sample(buf, labels, seconds):
    """The connectivity oracle, as it stands, on the case's images one at a time for about
    `seconds` (its CIELAB input from the FP64 conversion of the same sRGB image)."""
    import oracle
    from oracle.connectivity import enforce_connectivity
    K = (W // LEARN_V) * (H // LEARN_V)
    done, t0 = 0, time.perf_counter()
    while done < len(labels) and (done == 0 or time.perf_counter() - t0 < seconds):
        lab = oracle.rgb2lab(buf[done].cpu().numpy()).astype(np.float32)
        enforce_connectivity(labels[done].cpu().numpy(), lab, K)
        done += 1
    secs = time.perf_counter() - t0
    return done, secs


def run_conn_workload(args):
    """`conn256`: Algorithm 1, step 8 (connectivity post-processing) on the label maps of 256
    held-out 481x321 images after 10 plain-EM iterations, one call for the whole batch."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    n = 256
    bt, before, buf = _conn_case(gm, torch, n, stream, keep_images=True)

    def restore():
        with torch.cuda.stream(stream):
            for x, y in zip(bt.labels, before):
                x.copy_(y)

    for _ in range(max(args.warmup, 3)):
        restore()
        bt.connectivity()
    times = []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            restore()
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = bt.connectivity()        # synchronises the stream at its end
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    pix = n * W * H
    achieved = pix * CONN_BYTES_PER_PIXEL / (ms * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs")
    src = "MEASURED_PEAKS.json hbm_gbs"
    if not peak:
        peak, src = 6800.0, "fallback 6.8 TB/s"
    bt.close()
    cpu = None
    if not args.no_cpu_baseline:
        done, secs = conn_oracle_sample(buf, before, args.cpu_seconds)
        cpu = {"value": round(done * W * H / secs / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} of the {n} label maps in {secs:.1f} s (numpy, one thread; CIELAB conversion "
                         "included)"}
    line = {"metric": "Mpixel/s connectivity post-processing (Algorithm 1, step 8)",
            "value": round(pix / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32 (labels), int64 (fixed-point colour sums), f64",
            "data": "synthetic",
            "config": {"workload": f"{n} held-out synthetic 481x321 Voronoi images (150 regions, sigma 8), label maps "
                                   f"after {ITERS} plain-EM iterations at spacing {LEARN_V}; one "
                                   "gmmsp_batch_connectivity call per step", "images": n,
                       "l2": "flushed before every timed step (256 MiB memset); the label maps are restored "
                             "outside the timed interval"},
            "components": st["components"], "small": st["small"], "merged": st["merged"],
            "roofline": {"kernel": f"the whole post-processing call ({CONN_LAUNCHES} kernels)", "bound": "hbm",
                         "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_source": src,
                         "algorithmic_bytes_per_pixel": CONN_BYTES_PER_PIXEL},
            "gpu_launches": CONN_LAUNCHES * args.steps, "clocks": clk.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


# Algorithmic DRAM bytes per pixel of the accuracy metrics: the labels and the ground
# truth read once (4 + 4 B).
METRICS_BYTES_PER_PIXEL = 8
METRICS_LAUNCHES = 4  # kernels of one gmmsp_segmentation_metrics_many call


def run_metrics_workload(args):
    """`metrics256`: BR, UE (Eq. ue) and ASA of the label maps of 256 held-out 481x321
    images after 10 plain-EM iterations against the generator's regions, one
    gmmsp_segmentation_metrics_many call per step."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    n = 256
    regs = torch.empty((n, H, W), dtype=torch.int32, device="cuda")
    bt, labels, buf = _conn_case(gm, torch, n, stream, keep_images=True, regions=regs)
    K = (W // LEARN_V) * (H // LEARN_V)
    gts = [regs[i] for i in range(n)]

    def step():
        return gm.gmmsp_segmentation_metrics_many(labels, gts, K, REGIONS, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    times = []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step()                  # synchronises the stream at its end
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    bt.close()
    cpu = None
    if not args.no_cpu_baseline:
        done, secs = metrics_oracle_sample(labels, gts, K, args.cpu_seconds)
        cpu = {"value": round(done * W * H / secs / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} of the {n} label maps in {secs:.1f} s (numpy, one thread)"}
    ms = sum(times) / len(times)
    pix = n * W * H
    achieved = pix * METRICS_BYTES_PER_PIXEL / (ms * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs")
    src = "MEASURED_PEAKS.json hbm_gbs"
    if not peak:
        peak, src = 6800.0, "fallback 6.8 TB/s"
    line = {"metric": "Mpixel/s accuracy metrics (BR, Eq. ue, Eq. asa) against a ground truth",
            "value": round(pix / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32 counts (exact)", "data": "synthetic",
            "config": {"workload": f"{n} held-out synthetic 481x321 Voronoi images ({REGIONS} regions, sigma 8): "
                                   f"label maps after {ITERS} plain-EM iterations at spacing {LEARN_V} against the "
                                   "generator's region maps, BR radius 2, UE eps 0.05; one batched call per step",
                       "images": n, "K": K, "G": REGIONS,
                       "l2": "flushed before every timed step (256 MiB memset)"},
            "mean": {k: float(np.mean([r[k] for r in res])) for k in ("br", "ue", "asa")},
            "roofline": {"kernel": f"the whole metrics call ({METRICS_LAUNCHES} kernels)", "bound": "hbm",
                         "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_source": src,
                         "algorithmic_bytes_per_pixel": METRICS_BYTES_PER_PIXEL},
            "gpu_launches": METRICS_LAUNCHES * args.steps, "clocks": clk.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def metrics_oracle_sample(labels, gts, K, seconds):
    """The metrics oracle, as it stands, on the label maps one at a time for about `seconds`."""
    from oracle import metrics as om
    done, t0 = 0, time.perf_counter()
    while done < len(labels) and (done == 0 or time.perf_counter() - t0 < seconds):
        om.all_metrics(labels[done].cpu().numpy(), gts[done].cpu().numpy(), 2, 0.05)
        done += 1
    return done, time.perf_counter() - t0


def run_reference_metrics(args):
    """`--impl reference --workload metrics256`: the metrics oracle on the same label maps and
    region maps, one image per step."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n = max(args.steps + 1, 1)
    regs = torch.empty((n, H, W), dtype=torch.int32, device="cuda")
    bt, labels, _ = _conn_case(gm, torch, n, stream, keep_images=True, regions=regs)
    bt.close()
    K = (W // LEARN_V) * (H // LEARN_V)
    gts = [regs[i] for i in range(n)]
    metrics_oracle_sample(labels[:1], gts[:1], K, 0.0)   # untimed: the oracle's first call
    done, secs = metrics_oracle_sample(labels[1:], gts[1:], K, 1e9)
    v = round(done * W * H / secs / 1e6, 4)
    print(json.dumps({"impl": "reference", "metric": "Mpixel/s accuracy metrics (BR, Eq. ue, Eq. asa) against a "
                                                     "ground truth",
                      "value": v, "unit": UNIT, "n_gpus": 1, "steps": done, "warmup": 1,
                      "ms_per_step": round(secs / max(done, 1) * 1e3, 3), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                      "config": {"workload": "held-out synthetic 481x321 label maps after 10 plain-EM iterations "
                                             "against the generator's regions, one image per step"},
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"{done} images"},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)
    return 0


def run_reference_conn(args):
    """`--impl reference --workload conn256`: the connectivity oracle on the same label maps,
    one image per step (the label maps themselves come from the GPU EM)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    bt, before, buf = _conn_case(gm, torch, max(args.steps + args.warmup, 1), stream, keep_images=True)
    bt.close()
    conn_oracle_sample(buf[:1], before[:1], 0.0)   # untimed: the oracle's first call
    done, secs = conn_oracle_sample(buf[args.warmup:], before[args.warmup:], 1e9)
    v = round(done * W * H / secs / 1e6, 4)
    print(json.dumps({"impl": "reference", "metric": "Mpixel/s connectivity post-processing (Algorithm 1, step 8)",
                      "value": v, "unit": UNIT, "n_gpus": 1, "steps": done, "warmup": args.warmup,
                      "ms_per_step": round(secs / max(done, 1) * 1e3, 3), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64", "data": "synthetic",
                      "config": {"workload": "held-out synthetic 481x321 label maps after 10 plain-EM iterations, "
                                             "one image per step"},
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"{done} images"},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gmmsp", choices=["gmmsp", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a short untimed case for ncu captures and exit")
    ap.add_argument("--warps-per-cell", type=int, default=0, help="with --profile-case: launch shape")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="with --profile-case --workload learned481: E+M pass variant (after the autotuner)")
    ap.add_argument("--first-pass", type=int, default=0,
                    help="with --blocks-per-sm: the first E+M pass's variant (0: the autotuner's)")
    ap.add_argument("--workload", default="learned481",
                    choices=["learned481", "481x321", "3840x2160", "batch256", "conn256", "metrics256"],
                    help="learned481 (the headline line); 481x321, 3840x2160 or batch256 (other lines); "
                         "with --profile-case the case to profile")
    ap.add_argument("--images", type=int, default=LEARN_IMAGES, help="learned481: images per step")
    ap.add_argument("--colour", default="full", choices=["full", "split", "gray"],
                    help="colour covariance model of the plain-EM lines batch256 and 3840x2160 (the others "
                         "run the full model)")
    args = ap.parse_args()
    if args.colour != "full" and (args.workload not in ("batch256", "3840x2160") or
                                  (args.profile_case and args.workload != "3840x2160")):
        ap.error("--colour applies to the batch256 and 3840x2160 lines (and the 3840x2160 profile case) only")
    if args.profile_case:
        return run_profile_case(args)
    if args.workload == "learned481":
        return run_reference_learned(args) if args.impl == "reference" else run_learned(args)
    if args.workload == "conn256":
        return run_reference_conn(args) if args.impl == "reference" else run_conn_workload(args)
    if args.workload == "metrics256":
        return run_reference_metrics(args) if args.impl == "reference" else run_metrics_workload(args)
    if args.workload != "481x321" and args.impl == "gmmsp":
        return run_other_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gmmsp(args)


if __name__ == "__main__":
    sys.exit(main())
