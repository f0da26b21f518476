#!/usr/bin/env python
"""Benchmark of the clipped Gaussian-splat render on one GB300 per rank.

Workload: the general scene (1,000,000 Gaussians, SH degree 3, seeded synthetic stand-in
for a Mip-NeRF360 capture) at 1920x1080 with a sweep of 16 parallel clip-plane offsets
across the scene (the plane-sweep protocol of the paper's render-efficiency experiment).
One step = one sweep = 16 clipped frames through the C ABI (preprocess, bin, render).

Prints one JSON line: frames/s (device-resident inputs), per-frame p50/p99 latency, the
end-to-end figure with host buffers, the roofline of the dominant kernel, the CPU
oracle timed on this host, SM clocks sampled during the timed region, and the number of
kernel launches in the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it expects torchrun's environment; every rank renders its own sweep (weak
scaling, no data-path collective) and rank 0 reports the max-over-ranks time.
`--impl reference` times the FP64 CPU oracle on this host instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "clipped frames/sec at 1080p/1M Gaussians + p50/p99 latency, batched vs plain, same GB300"
UNIT = "frames/s"

# Algorithmic FP32 work of the render kernel per unit (see the design notes):
#   rectangle test   min of q over a warp's 8x4 pixel box (4 edges)  36 FLOP (one per warp and entry)
#   walked pair      dx, dy and the conic quadratic form q            9 FLOP
#   in-support pair  alpha = delta exp(-q/2), clamp, T update, RGB   12 FLOP + 1 MUFU (ex2)
#   cutoff pair      ray-traced decay weight (Eq. 4-8, 11)           60 FLOP + 3 MUFU
FLOP_TEST, FLOP_WALKED, FLOP_EVAL, FLOP_CUT = 36, 9, 12, 60
SMS, FP32_LANES = 152, 128  # GB300: 152 SMs x 128 FP32 lanes, FMA = 2 FLOP

TRAFFIC_FILE = os.path.join(ROOT, "profiles", "render_fwd_general_1080p.txt")
RENDER_SRC = os.path.join(ROOT, "paper_2506_20202_gb300", "csrc", "render.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--sweep", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload_config(args):
    return {
        "workload": f"general scene, {args.n:,} Gaussians, SH degree 3, {args.width}x{args.height}, "
                    f"{args.sweep}-offset clip-plane sweep, RaRa mode",
        "n_gaussians": args.n, "sh_degree": 3, "width": args.width, "height": args.height,
        "planes": args.sweep, "tile": "16x16", "step": f"one sweep = {args.sweep} frames",
        "l2": "inputs larger than L2 (236 MB scene re-read every frame), no flush",
    }


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, maxmhz, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                maxmhz = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": maxmhz, "reasons": sorted(reasons),
                "samples": len(mhz)}


def traffic_for_current_kernel():
    """DRAM bytes per render launch from the committed ncu summary, if it was taken on the
    current render.cu (matched by hash); otherwise None."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m = re.search(r"render_cu_sha256:\s*([0-9a-f]{64})", text)
    b = re.search(r"dram_bytes_per_launch_full_frame:\s*([0-9.eE+]+)", text)
    if not m or not b:
        return None
    cur = hashlib.sha256(open(RENDER_SRC, "rb").read()).hexdigest()
    return float(b.group(1)) if m.group(1) == cur else None


# --------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------

def oracle_frame_rate(scene, cam, planes, plane_ids, bands, band_rows, threads):
    """Time the FP64 oracle on a bounded sample: per plane the full preprocess + key sort,
    and `bands` row bands of `band_rows` rows spread over the image. Frame time is
    extrapolated as t_pre + t_keys + mean(t_band) * H / band_rows."""
    import oracle
    H = cam.height
    pre_t, band_t = [], []
    for pid in plane_ids:
        pl = planes[pid]
        t0 = time.perf_counter()
        pre = oracle.preprocess(scene, cam, pl)
        kvr = oracle.build_keys(pre)
        pre_t.append(time.perf_counter() - t0)
        for b in range(bands):
            y0 = int((b + 0.5) * H / bands) - band_rows // 2
            y0 = max(0, min(H - band_rows, y0))
            t0 = time.perf_counter()
            oracle.render(scene, pre, cam, pl, (0.0, 0.0, 0.0), kvr, threads=threads, rows=(y0, y0 + band_rows))
            band_t.append(time.perf_counter() - t0)
    frame_s = statistics.mean(pre_t) + statistics.mean(band_t) * H / band_rows
    sample = (f"{len(plane_ids)} sweep planes: full preprocess + key sort each, {bands} bands of {band_rows} rows "
              f"each ({len(plane_ids) * bands * band_rows} of {len(plane_ids) * H} rows rendered); frame time "
              f"extrapolated to all {H} rows")
    return 1.0 / frame_s, frame_s, sample, sum(pre_t) + sum(band_t)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2506_20202_gb300 import scenes
    oracle.build()
    scene, cam, planes = scenes.general_workload(args.n, args.width, args.height, seed=0, sweep=args.sweep)
    threads = os.cpu_count() or 1
    # each step: one row band of one plane (cycling), per-plane preprocess/keys measured once
    band_rows = 8
    pre_t, band_t = {}, []
    import oracle as orc
    cache = {}
    total_steps = args.warmup + args.steps
    for s in range(total_steps):
        pid = s % args.sweep
        if pid not in cache:
            t0 = time.perf_counter()
            pre = orc.preprocess(scene, cam, planes[pid])
            kvr = orc.build_keys(pre)
            pre_t[pid] = time.perf_counter() - t0
            cache[pid] = (pre, kvr)
        pre, kvr = cache[pid]
        y0 = (s * 97 * band_rows) % (cam.height - band_rows)
        t0 = time.perf_counter()
        orc.render(scene, pre, cam, planes[pid], (0.0, 0.0, 0.0), kvr, threads=threads, rows=(y0, y0 + band_rows))
        if s >= args.warmup:
            band_t.append(time.perf_counter() - t0)
    frame_s = statistics.mean(pre_t.values()) + statistics.mean(band_t) * cam.height / band_rows
    value = 1.0 / frame_s
    sample = (f"each step renders {band_rows} rows of one sweep frame (plane cycling over {args.sweep}); the full "
              f"per-plane preprocess + key sort is timed once per plane; frame time = mean(preprocess+sort) + "
              f"mean(band) x {cam.height}/{band_rows}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": frame_s * args.sweep * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------

def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = int(k), min(len(xs) - 1, int(k) + 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2506_20202_gb300 import build, rara, scenes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    build.build()

    scene, cam, planes = scenes.general_workload(args.n, args.width, args.height, seed=0, sweep=args.sweep)
    gs = rara.GaussianTensors.from_scene(scene, f"cuda:{local}")
    ctx = rara.rara_ctx_create(0)
    H, W = cam.height, cam.width
    image = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
    final_T = torch.empty((H, W), dtype=torch.float32, device="cuda")
    n_contrib = torch.empty((H, W), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    bg = (0.0, 0.0, 0.0)

    def frame(pl, evs=None):
        if evs is not None:
            evs[0].record(stream)
        rara.rara_preprocess(ctx, gs, cam, pl, stream)
        if evs is not None:
            evs[1].record(stream)
        rara.rara_bin(ctx, stream)
        if evs is not None:
            evs[2].record(stream)
        rara.rara_render(ctx, bg, image, final_T, n_contrib, stream)
        if evs is not None:
            evs[3].record(stream)

    # warm-up
    for _ in range(args.warmup):
        for pl in planes:
            frame(pl)
    stream.synchronize()

    # per-plane work counters (untimed pass)
    counts = []
    for pl in planes:
        frame(pl)
        counts.append(rara.rara_frame_info_get(ctx))
    stream.synchronize()

    nfr = args.steps * len(planes)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nfr)]
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = rara.rara_ctx_launches(ctx)
    t_begin.record(stream)
    k = 0
    for _ in range(args.steps):
        for pl in planes:
            frame(pl, evs[k])
            k += 1
    t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    launches = rara.rara_ctx_launches(ctx) - launches0
    sampler.stop()
    if dist:
        dist.barrier()
    elapsed_ms = t_begin.elapsed_time(t_end)
    if dist:
        t = torch.tensor([elapsed_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = world * nfr / (elapsed_ms / 1e3)

    lat = [e[0].elapsed_time(e[3]) for e in evs]
    t_pre = [e[0].elapsed_time(e[1]) for e in evs]
    t_bin = [e[1].elapsed_time(e[2]) for e in evs]
    t_ren = [e[2].elapsed_time(e[3]) for e in evs]
    clocks = sampler.summary()

    # roofline of the dominant kernel (the render: one launch per frame)
    peaks, peak_kind = measured_peaks()
    stage_ms = {"preprocess": statistics.mean(t_pre), "bin": statistics.mean(t_bin),
                "render": statistics.mean(t_ren)}
    flop = [FLOP_TEST * c["n_tested"] + FLOP_WALKED * c["n_walked"] + FLOP_EVAL * c["n_evaluated"]
            + FLOP_CUT * c["n_cut_evaluated"] for c in counts]
    ren_by_plane = [statistics.mean(t_ren[i::len(planes)]) for i in range(len(planes))]
    achieved = statistics.mean([f / (t * 1e-3) for f, t in zip(flop, ren_by_plane)]) / 1e12
    sm_max = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    peak = SMS * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": "k_render", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for_current_kernel(),
                "peak_basis": f"FP32 FMA: {SMS} SMs x {FP32_LANES} lanes x 2 FLOP x {sm_max:.0f} MHz "
                              f"(recipe unit counts, max SM clock)",
                "per_frame_units": {"tested": statistics.mean(c["n_tested"] for c in counts),
                                    "walked": statistics.mean(c["n_walked"] for c in counts),
                                    "evaluated": statistics.mean(c["n_evaluated"] for c in counts),
                                    "cut_evaluated": statistics.mean(c["n_cut_evaluated"] for c in counts)}}
    # HBM view of the other stages (context)
    n = scene.n
    pre_bytes = n * (12 + 12 + 16 + 4 + 4 * scene.sh.shape[0]) + \
        statistics.mean(c["n_rendered"] * (48 + 8 + 8) + n * 5 + c["n_cutoff"] * 64 for c in counts)
    stages = {k2: {"ms": v} for k2, v in stage_ms.items()}
    stages["preprocess"]["algorithmic_GBps"] = pre_bytes / (stage_ms["preprocess"] * 1e-3) / 1e9
    stages["preprocess"]["hbm_frac"] = stages["preprocess"]["algorithmic_GBps"] / peaks["hbm_gbs"]

    # end to end through the C ABI with host buffers: per step the scene is uploaded from
    # pinned host memory and each frame's image is read back into pinned host memory
    host = {k2: torch.from_numpy(np.ascontiguousarray(getattr(scene, k2), np.float32)).pin_memory()
            for k2 in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    dev = rara.GaussianTensors(*(torch.empty_like(host[k2], device="cuda") for k2 in
                                 ("means", "log_scales", "quats", "opacity_logits", "sh")), scene.sh_degree)
    img_host = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in planes]
    h2d = sum(t.numel() * 4 for t in host.values())
    d2h = len(planes) * 3 * H * W * 4
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            for k2, name in zip(("means", "log_scales", "quats", "opacity_logits", "sh"),
                                ("means", "log_scales", "quats", "opacity_logits", "sh")):
                getattr(dev, name).copy_(host[k2], non_blocking=True)
            for i, pl in enumerate(planes):
                rara.rara_render_frame(ctx, dev, cam, pl, bg, image, None, None, stream)
                img_host[i].copy_(image, non_blocking=True)
    stream.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * args.e2e_steps * len(planes) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "note": "per step: scene upload from pinned host memory + one C-ABI render per sweep frame + "
                   "image read-back into pinned host memory; host wall clock"}
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e["value"] = world * args.e2e_steps * len(planes) / float(t.item())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args),
        "latency_ms": {"plain_p50": percentile(lat, 50), "plain_p99": percentile(lat, 99),
                       "note": "per-frame preprocess+bin+render on one stream, one request per launch sequence"},
        "stages_ms": stages,
        "roofline": roofline, "peak_source": peak_kind,
        "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
        "frame_counts": {"cutoff_fraction_per_plane": [round(c["n_cutoff"] / max(1, c["n_rendered"]), 4)
                                                       for c in counts],
                         "pairs_mean": statistics.mean(c["n_pairs"] for c in counts)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fr, fs, sample, spent = oracle_frame_rate(scene, cam, planes, [4, 8, 12], 6, 16, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": fr, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": sample, "seconds": spent}
    rara.rara_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
