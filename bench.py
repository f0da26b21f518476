#!/usr/bin/env python
"""Benchmark of the clipped Gaussian-splat render on one GB300 per rank.

Workload: the general scene (1,000,000 Gaussians, SH degree 3, seeded synthetic stand-in
for a Mip-NeRF360 capture) at 1920x1080 with a sweep of 16 parallel clip-plane offsets
across the scene (the plane-sweep protocol of the paper's render-efficiency experiment).
One step = one sweep = 16 clipped frames through the C ABI (preprocess, bin, render).

Prints one JSON line. `value` is frames/s of the batched path (the 16 sweep frames as one
batch, one launch per stage, replayed as a CUDA graph, autotuned) with the scene resident;
`paths` also gives the plain one-frame-per-launch-sequence path, `latency_ms` the p50/p99 of
both, `e2e` the batched path end to end with host buffers, `roofline` the batched render
launch, `serving` a continuous-batching server against the plain path on Poisson arrivals,
`cpu_baseline` the FP64 oracle timed on this host, `clocks` the SM clocks sampled during the
timed region, and `gpu_launches` the kernel launches in it.

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

# Algorithmic FP32 work of the render per unit, the method's own arithmetic (the units the
# roofline is stated in): an evaluated (pixel, Gaussian) pair, alpha0 = delta exp(-q/2) >= 1/255
# inside the q <= 9 support (Eq. 2, Eq. 10, Algorithm 1 step 3: offset, q, alpha, clamp,
# transmittance and colour update) costs 15 FLOP + 1 exp; a cutoff pair adds the ray-traced
# decay weight (Eq. 4-8, Eq. 11: chord, front test, plane split) for 30 FLOP + sqrt + rcp.
FLOP_EVAL, FLOP_CUT = 15, 30
# The kernel's own work per unit, counted from its instructions (context: it includes the
# culling the method does not define):
#   rectangle test   min of q over a warp's 8x4 pixel box (4 edges)  36 FLOP (one per warp and entry)
#   walked pair      dx, dy and the conic quadratic form q            9 FLOP
#   blending pair    alpha0, clamp, T update, RGB                     12 FLOP + 1 MUFU (ex2)
#   cutoff pair      decay weight as the kernel evaluates it          60 FLOP + 3 MUFU
KFLOP_TEST, KFLOP_WALKED, KFLOP_EVAL, KFLOP_CUT = 36, 9, 12, 60
FP32_LANES = 128  # FP32 lanes per SM on GB300 (an FMA counts 2 FLOP)


def sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)

TRAFFIC_FILE = os.path.join(ROOT, "profiles", "render_fwd_general_1080p.txt")
RENDER_SRCS = [os.path.join(ROOT, "paper_2506_20202_gb300", "csrc", f) for f in ("render.cu", "render_common.cuh")]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--sweep", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--plain-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", default="", help="split thresholds 'a,b' instead of autotuning")
    ap.add_argument("--serve-s", type=float, default=30.0, help="serving window (0: skip)")
    ap.add_argument("--serve-fast-s", type=float, default=2.0, help="window of the 10x-rate serving leg")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-3m", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--train-steps", type=int, default=6, help="forward+backward steps of the multi-layer "
                    "differentiation workload (0: skip)")
    ap.add_argument("--train-per-shell", type=int, default=700_000)
    ap.add_argument("--train-multi", action="store_true", help="with several ranks, run the differentiation "
                    "leg data-parallel over all of them (views sharded, gradients all-reduced over NCCL)")
    ap.add_argument("--hair-steps", type=int, default=20, help="frames of the hair-strand workload per path "
                    "(0: skip)")
    ap.add_argument("--train-views", type=int, default=64)
    ap.add_argument("--volume-steps", type=int, default=20, help="batches of the clip-volume sweep (0: skip)")
    ap.add_argument("--mode-steps", type=int, default=20, help="batches per clipping mode of the Table 1 "
                    "comparison on the sweep and hair workloads (0: skip)")
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


def issue_slots_for_current_kernel():
    """The render kernel's issue-slot use from the committed ncu summary (issue active % of
    its active cycles), if it was taken on the current render sources; otherwise None."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m = re.search(r"issue active %\s+([0-9.]+)", text)
    if not m or not _profile_matches_sources(text):
        return None
    return {"issue_active_frac": float(m.group(1)) / 100.0, "source": os.path.relpath(TRAFFIC_FILE, ROOT),
            "note": "the kernel issues on this share of its SMs' active cycles (ncu, 4-view capture at 16x32 "
                    "tiles, 256-entry batches)"}


def _profile_matches_sources(text):
    for path in RENDER_SRCS:
        key = os.path.basename(path).replace(".", "_") + "_sha256"
        m = re.search(key + r":\s*([0-9a-f]{64})", text)
        if not m or m.group(1) != hashlib.sha256(open(path, "rb").read()).hexdigest():
            return False
    return True


def traffic_for_current_kernel(tuning):
    """DRAM bytes of the benchmark's render launch from the committed ncu summary, if it was
    taken on the current render sources (matched by hash) with the same tiling and split
    thresholds (tuning: tile_w, tile_h, depth, split2, split4); otherwise None."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    tag = ",".join(str(int(x)) for x in tuning)
    b = re.search(r"dram_bytes_per_bench_launch \(tuning " + re.escape(tag) + r"\):\s*([0-9.eE+]+)", text)
    if not b:
        return None
    for path in RENDER_SRCS:
        key = os.path.basename(path).replace(".", "_") + "_sha256"
        m = re.search(key + r":\s*([0-9a-f]{64})", text)
        if not m or m.group(1) != hashlib.sha256(open(path, "rb").read()).hexdigest():
            return None
    return float(b.group(1))


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
    if bands * band_rows >= H:
        sample = (f"{len(plane_ids)} of the {len(planes)} sweep frames (planes {list(plane_ids)}) rendered in full: "
                  f"preprocess, key sort and all {H} rows each")
    else:
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
    # each step: one eighth of a frame (a band of H/8 rows) of one plane, planes and bands
    # cycling; the per-plane preprocess/keys are timed once per plane. Bands this tall keep the
    # per-call set-up (argument conversion, output buffers) a small share of the band's time.
    band_rows = (cam.height + 7) // 8
    pre_t, band_t = {}, []
    import oracle as orc
    cache = {}
    total_steps = args.warmup + args.steps
    step_t = []
    for s in range(total_steps):
        pid = s % args.sweep
        t_step = time.perf_counter()
        if pid not in cache:
            t0 = time.perf_counter()
            pre = orc.preprocess(scene, cam, planes[pid])
            kvr = orc.build_keys(pre)
            pre_t[pid] = time.perf_counter() - t0
            cache[pid] = (pre, kvr)
        pre, kvr = cache[pid]
        y0 = min(((s // args.sweep + 3 * s) % 8) * band_rows, cam.height - band_rows)
        t0 = time.perf_counter()
        orc.render(scene, pre, cam, planes[pid], (0.0, 0.0, 0.0), kvr, threads=threads, rows=(y0, y0 + band_rows))
        if s >= args.warmup:
            band_t.append(time.perf_counter() - t0)
            step_t.append(time.perf_counter() - t_step)
    frame_s = statistics.mean(pre_t.values()) + statistics.mean(band_t) * cam.height / band_rows
    value = 1.0 / frame_s
    step_ms = 1e3 * (sum(step_t) / len(step_t))
    sample = (f"each step renders {band_rows} rows (one eighth) of one sweep frame (plane cycling over {args.sweep}); the full "
              f"per-plane preprocess + key sort is timed once per plane; frame time = mean(preprocess+sort) + "
              f"mean(band) x {cam.height}/{band_rows}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "frame_ms_extrapolated": frame_s * 1e3,
        "step_note": "ms_per_step is the measured mean of a timed step (one band, plus the plane's preprocess and "
                     "key sort on the step that first meets it); value extrapolates whole frames from those parts",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------

def max_over_ranks(value: float, dist) -> float:
    """The largest of a per-rank float over all ranks (the slowest rank's time), through the
    host process group; the value itself with one rank (dist None)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units per second of the whole job: every rank processed units_per_rank (weak scaling)
    and the job took the slowest rank's time."""
    return world * units_per_rank / seconds


def stage_hbm(kms, vinfo, scene, W, H, hbm_gbs, depth_keys=None, shared_pairs=0):
    """Algorithmic bytes of each preprocess and binning stage of an exact batched render, their
    GB/s over the stage's GPU time (rara_ctx_kernel_ms) and the fraction of the measured HBM
    copy bandwidth. Bytes per unit (the design notes list them):
      preprocess   the scene once (44 B of geometry + 12 (L+1)^2 B of SH per Gaussian), 5 B per
                   (view, Gaussian) slot (label, tiles), 84 B per rendered slot (emission
                   record, splat record, depth; with a shared listing the 32-byte emission
                   record only once per Gaussian some view renders), 64 B per cutoff slot
                   (ray-tracing record)
      compaction   8 B per slot read (tiles, depth), 8 B per rendered slot written
      depth sort   16 B per key per digit pass launched (4 depth + 1 view pass over the
                   rendered slots; for a one-camera batch 4 depth passes over the Gaussians some
                   view renders, plus the expansion into the views' slots: 4 B of sorted value
                   and 4 B of tile count read per (view, key), 4 B written per rendered slot)
      emission     36 B per rendered slot read (slot, its 32-byte emission record), 8 B per pair
      tile sort    16 B per pair per digit pass
      ranges       4 B per pair read, 8 B per tile written
    A one-camera batch of at most 32 views lists once (shared_pairs > 0): the depth sort has no
    expansion; the emission reads 40 B per Gaussian some view renders (its view mask too) and
    writes 8 B per shared pair; the tile sort sorts the shared pairs; the listing reads 20 B per
    shared pair (value and mask twice, key once) and writes 4 B per view pair and 8 B per tile."""
    views = len(vinfo)
    n = scene.n
    slots = views * n
    rendered = sum(v["n_rendered"] for v in vinfo)
    cutoff = sum(v["n_cutoff"] for v in vinfo)
    pairs = sum(v["n_pairs"] for v in vinfo)
    tiles = sum(v["tiles_x"] * v["tiles_y"] for v in vinfo)
    tile_bits = max(1, (max(v["tiles_x"] * v["tiles_y"] for v in vinfo) - 1).bit_length())
    tile_passes = (tile_bits + 7) // 8
    view_passes = 0 if views == 1 else (1 if views <= 256 else 2)
    bytes_ = {
        "preprocess": n * (44 + 4 * scene.sh.shape[0]) + 5 * slots + 64 * cutoff +
                      (52 * rendered + 32 * depth_keys if shared_pairs else 84 * rendered),
        "compaction": (8 * slots + 8 * rendered) if depth_keys is None else (4 * n + 8 * depth_keys),
        "depth_sort": 16 * rendered * (4 + view_passes) if depth_keys is None else
                      16 * depth_keys * 4 + (0 if shared_pairs else 8 * views * depth_keys + 4 * rendered),
        "emission": 40 * depth_keys + 8 * shared_pairs if shared_pairs else 36 * rendered + 8 * pairs,
        "tile_sort": 16 * (shared_pairs or pairs) * tile_passes,
        "ranges": (20 * shared_pairs + 4 * pairs + 8 * tiles) if shared_pairs else 4 * pairs + 8 * tiles,
    }
    out = {}
    for (name, b), ms in zip(bytes_.items(), kms):
        gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else None
        out[name] = {"ms": ms, "bytes": int(b), "GBps": gbs, "hbm_frac": gbs / hbm_gbs if gbs else None}
    return out


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

    from paper_2506_20202_gb300 import autotune, build, rara, scenes, serve

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        # host-side timing reductions over gloo; gradient all-reduces of CUDA tensors over NCCL
        dist.init_process_group("cpu:gloo,cuda:nccl")
    torch.cuda.set_device(local)
    build.build()

    scene, cam, planes = scenes.general_workload(args.n, args.width, args.height, seed=0, sweep=args.sweep)
    gs = rara.GaussianTensors.from_scene(scene, f"cuda:{local}")
    H, W = cam.height, cam.width
    stream = torch.cuda.Stream()
    bg = (0.0, 0.0, 0.0)
    nplanes = len(planes)

    # ---------------- plain path: one frame per launch sequence --------------------------
    plain, counts = None, None
    if args.plain_steps > 0:
        ctx = rara.rara_ctx_create(0)
        image = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
        final_T = torch.empty((H, W), dtype=torch.float32, device="cuda")
        n_contrib = torch.empty((H, W), dtype=torch.int32, device="cuda")

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

        for _ in range(args.warmup):
            for pl in planes:
                frame(pl)
        counts = []
        for pl in planes:
            frame(pl)
            counts.append(rara.rara_frame_info_get(ctx))
        stream.synchronize()
        plain_steps = max(3, min(args.steps, args.plain_steps))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(plain_steps * nplanes)]
        p_begin, p_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        p_begin.record(stream)
        k = 0
        for _ in range(plain_steps):
            for pl in planes:
                frame(pl, evs[k])
                k += 1
        p_end.record(stream)
        stream.synchronize()
        plain_ms = p_begin.elapsed_time(p_end)
        lat = [e[0].elapsed_time(e[3]) for e in evs]
        t_pre = [e[0].elapsed_time(e[1]) for e in evs]
        t_bin = [e[1].elapsed_time(e[2]) for e in evs]
        t_ren = [e[2].elapsed_time(e[3]) for e in evs]
        plain = {"frames_per_s": plain_steps * nplanes / (plain_ms / 1e3), "p50_ms": percentile(lat, 50),
                 "p99_ms": percentile(lat, 99), "stage_ms": {"preprocess": statistics.mean(t_pre),
                                                             "bin": statistics.mean(t_bin),
                                                             "render": statistics.mean(t_ren)},
                 "note": "per frame: preprocess, bin (one host wait), render on one stream"}
        rara.rara_ctx_destroy(ctx)

    # ---------------- batched path: the sweep as one batch, CUDA-graph replay ------------
    bctx = rara.rara_ctx_create(0)
    outs = [(torch.empty((3, H, W), dtype=torch.float32, device="cuda"),
             torch.empty((H, W), dtype=torch.float32, device="cuda"),
             torch.empty((H, W), dtype=torch.int32, device="cuda")) for _ in planes]
    views = [rara.View(0, cam, pl, o[0], o[1], o[2], bg) for pl, o in zip(planes, outs)]
    if args.tuning:
        best, tune_ms = autotune.parse(args.tuning), {}
        autotune.apply(bctx, best)
    else:
        best, tune_ms = autotune.autotune(bctx, [gs], views, stream, reps=3)
    # stage times and work counts of one exact batched render (for the roofline)
    rara.rara_ctx_count_work(bctx, True)
    rara.rara_render_batch(bctx, [gs], views, stream)
    rara.rara_ctx_count_work(bctx, False)
    stage = rara.rara_ctx_stage_ms(bctx)
    kms = rara.rara_ctx_kernel_ms(bctx)
    binfo = rara.rara_frame_info_get(bctx, 0)
    vinfo = [rara.rara_frame_info_get(bctx, v) for v in range(nplanes)]
    if counts is None:
        counts = [rara.rara_frame_info_get(bctx, v) for v in range(nplanes)]
    for _ in range(args.warmup):
        rara.rara_render_batch_graph(bctx, [gs], views, stream)
    rara.rara_ctx_sync(bctx, stream)

    sevs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = rara.rara_ctx_launches(bctx)
    t_begin.record(stream)
    for kk in range(args.steps):
        sevs[kk][0].record(stream)
        rara.rara_render_batch_graph(bctx, [gs], views, stream)
        sevs[kk][1].record(stream)
    t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    launches = rara.rara_ctx_launches(bctx) - launches0
    sampler.stop()
    rara.rara_ctx_sync(bctx, stream)   # raises if a replay overflowed its pair capacity
    if dist:
        dist.barrier()
    elapsed_ms = max_over_ranks(t_begin.elapsed_time(t_end), dist)
    value = whole_job_rate(args.steps * nplanes, world, elapsed_ms / 1e3)
    blat = [e[0].elapsed_time(e[1]) for e in sevs]
    batched = {"frames_per_s": value, "batch_p50_ms": percentile(blat, 50), "batch_p99_ms": percentile(blat, 99),
               "views_per_batch": nplanes, "tuning": list(best),
               "autotune_ms": {json.dumps(list(k2)): v for k2, v in tune_ms.items()},
               "stage_ms_exact_batch": {"preprocess": stage[0], "bin": stage[1], "render": stage[2]},
               "note": "the 16 sweep frames as one batch (one launch per stage), replayed as a CUDA graph; "
                       "a request's latency is its batch's"}
    clocks = sampler.summary()
    peaks, peak_kind = measured_peaks()

    # roofline of the dominant kernel: the render launch of the batch, timed by the events the
    # captured graph records around it (the replays the timed region ran); units from the
    # exact render of the same batch (the same work, counted on the device)
    replay_kms, replay_render = [], []
    for _ in range(10):
        rara.rara_render_batch_graph(bctx, [gs], views, stream)
        replay_render.append(rara.rara_ctx_stage_ms(bctx)[2])
        replay_kms.append(rara.rara_ctx_kernel_ms(bctx))
    t_render = statistics.mean(replay_render)
    sms = sm_count()
    flop = FLOP_EVAL * binfo["n_evaluated"] + FLOP_CUT * binfo["n_cut_evaluated"]
    kflop = (KFLOP_TEST * binfo["n_tested"] + KFLOP_WALKED * binfo["n_walked"] + KFLOP_EVAL * binfo["n_evaluated"]
             + KFLOP_CUT * binfo["n_cut_evaluated"])
    achieved = flop / (t_render * 1e-3) / 1e12
    sm_max = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    peak = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    issue = issue_slots_for_current_kernel()
    roofline = {"bound": "alu", "kernel": "k_render (one launch for the 16-view batch)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic_for_current_kernel(best),
                "launch_ms": t_render, "launch_ms_exact_render": stage[2],
                "flop_per_launch": flop,
                "units": "15 FLOP per evaluated (pixel, Gaussian) pair + 30 per cutoff pair (the method's arithmetic)",
                "peak_basis": f"FP32 FMA: {sms} SMs (device) x {FP32_LANES} lanes x 2 FLOP x {sm_max:.0f} MHz "
                              f"(max SM clock; of measured clocks)",
                "kernel_work": {"flop_per_launch": kflop, "achieved": kflop / (t_render * 1e-3) / 1e12,
                                "frac": kflop / (t_render * 1e-3) / 1e12 / peak,
                                "note": "the kernel's own arithmetic incl. its culling tests (36/9/12/60 FLOP per "
                                        "test/walked/blending/cutoff unit)"},
                "issue_slots": issue,
                "per_launch_units": {"tested": binfo["n_tested"], "walked": binfo["n_walked"],
                                     "evaluated": binfo["n_evaluated"], "cut_evaluated": binfo["n_cut_evaluated"]}}
    kms = [statistics.mean(k[j] for k in replay_kms) for j in range(6)]
    one_camera = binfo["n_depth_keys"] != sum(v["n_rendered"] for v in vinfo)
    batched["stage_hbm"] = stage_hbm(kms, vinfo, scene, W, H, peaks["hbm_gbs"],
                                     binfo["n_depth_keys"] if one_camera else None, binfo["n_shared_pairs"])
    batched["depth_keys"] = {"keys": binfo["n_depth_keys"], "one_camera_batch": one_camera,
                             "shared_pairs": binfo["n_shared_pairs"],
                             "view_pairs": sum(v["n_pairs"] for v in vinfo)}
    batched["stage_hbm_note"] = "stage times: mean of 10 graph replays (events recorded by the graph)"
    n = scene.n
    pre_bytes = n * (12 + 12 + 16 + 4 + 4 * scene.sh.shape[0]) + \
        statistics.mean(c["n_rendered"] * (48 + 8 + 8) + n * 9 + c["n_cutoff"] * 64 for c in counts)
    if plain:
        plain["preprocess_algorithmic_GBps"] = pre_bytes / (plain["stage_ms"]["preprocess"] * 1e-3) / 1e9
        plain["preprocess_hbm_frac"] = plain["preprocess_algorithmic_GBps"] / peaks["hbm_gbs"]

    e2e = None
    if args.e2e_steps > 0:
        # End to end through the C ABI with host buffers (graph path): every step uploads the
        # scene from pinned host memory and reads every image back into pinned host memory.
        # The steps are pipelined the way a serving loop runs them: the upload of step k and
        # the read-back of step k - 1 run on their own streams (the copy engines) while step
        # k - 1 renders, with the device scene and the images double-buffered. All copies of
        # every timed step are inside the timed region.
        keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
        host = {k2: torch.from_numpy(np.ascontiguousarray(getattr(scene, k2), np.float32)).pin_memory()
                for k2 in keys}
        devs = [rara.GaussianTensors(*(torch.empty_like(host[k2], device="cuda") for k2 in keys), scene.sh_degree)
                for _ in range(2)]
        e_outs = [outs] + [[(torch.empty((3, H, W), dtype=torch.float32, device="cuda"),
                             torch.empty((H, W), dtype=torch.float32, device="cuda"),
                             torch.empty((H, W), dtype=torch.int32, device="cuda")) for _ in planes]]
        e_views = [[rara.View(0, cam, pl, o[0], o[1], o[2], bg) for pl, o in zip(planes, oo)] for oo in e_outs]
        img_host = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in planes]
        h2d = sum(t.numel() * 4 for t in host.values())
        d2h = nplanes * 3 * H * W * 4
        ectx = rara.rara_ctx_create(0)
        autotune.apply(ectx, best)
        up_stream, down_stream = torch.cuda.Stream(), torch.cuda.Stream()
        ev_up = [torch.cuda.Event() for _ in range(2)]
        ev_ren = [torch.cuda.Event() for _ in range(2)]
        ev_down = [torch.cuda.Event() for _ in range(2)]
        for b in range(2):
            ev_ren[b].record(stream)
            ev_down[b].record(stream)
        step_no = [0]

        def e2e_step():
            b = step_no[0] & 1
            step_no[0] += 1
            up_stream.wait_event(ev_ren[b])           # the render that read devs[b] is done
            with torch.cuda.stream(up_stream):
                for k2 in keys:
                    getattr(devs[b], k2).copy_(host[k2], non_blocking=True)
            ev_up[b].record(up_stream)
            stream.wait_event(ev_up[b])
            stream.wait_event(ev_down[b])             # the read-back of e_outs[b] is done
            rara.rara_render_batch_graph(ectx, [devs[b]], e_views[b], stream)
            ev_ren[b].record(stream)
            down_stream.wait_event(ev_ren[b])
            with torch.cuda.stream(down_stream):
                for i in range(nplanes):
                    img_host[i].copy_(e_outs[b][i][0], non_blocking=True)
            ev_down[b].record(down_stream)

        def e2e_sync():
            rara.rara_ctx_sync(ectx, stream)
            up_stream.synchronize()
            down_stream.synchronize()

        for _ in range(3):
            e2e_step()
        e2e_sync()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        e2e_sync()
        e2e_s = time.perf_counter() - t0
        rara.rara_ctx_destroy(ectx)
        e2e_s = max_over_ranks(e2e_s, dist)
        e2e = {"value": whole_job_rate(args.e2e_steps * nplanes, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "per step: scene upload from pinned host memory + one C-ABI batched render of the 16 sweep "
                       "frames (graph replay) + read-back of every image into pinned host memory; steps pipelined "
                       "(upload and read-back on their own streams, scene and images double-buffered); host wall "
                       "clock from the first step's upload to the last step's read-back"}
    rara.rara_ctx_destroy(bctx)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args),
        "paths": {"batched_graph": batched, "plain": plain},
        "latency_ms": {"plain_p50": plain and plain["p50_ms"], "plain_p99": plain and plain["p99_ms"],
                       "batched_p50": batched["batch_p50_ms"], "batched_p99": batched["batch_p99_ms"]},
        "roofline": roofline, "peak_source": peak_kind,
        "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
        "frame_counts": {"cutoff_fraction_per_plane": [round(c["n_cutoff"] / max(1, c["n_rendered"]), 4)
                                                       for c in counts],
                         "pairs_mean": statistics.mean(c["n_pairs"] for c in counts)},
    }
    if rank == 0 and world == 1 and args.mode_steps > 0:
        line["paths"]["modes"] = {"general_sweep": run_modes(args, gs, cam, planes, best),
                                  "paper_table1_rtx4090": PAPER_TABLE1}
    if rank == 0 and world == 1 and args.volume_steps > 0:
        line["volume"] = run_volume(args, gs, cam, planes)
    if rank == 0 and world == 1 and args.hair_steps > 0:
        line["hair"] = run_hair(args)
        if "modes" in line["hair"] and "modes" in line["paths"]:
            line["paths"]["modes"]["hair"] = line["hair"]["modes"]
    if args.train_steps > 0 and (world == 1 or args.train_multi):
        tr = run_training(args, rank, world)
        if rank == 0:
            line["training"] = tr
    if rank == 0 and world == 1 and args.serve_s > 0:
        line["serving"] = run_serving(args, gs, scene)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # every sweep frame in full (about 15 s of oracle work on a 16-core host)
        pids = list(range(len(planes)))
        fr, fs, sample, spent = oracle_frame_rate(scene, cam, planes, pids, 1, cam.height, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": fr, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": sample, "seconds": spent}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# Algorithmic FP32 work of the render backward per unit, counted from the kernel's
# arithmetic (the forward's pair counts of the same batch serve as unit counts):
#   walked pair      dx, dy and q                                           10 FLOP
#   in-support pair  alpha recomputed, T / (1 - alpha), colour and alpha
#                    gradients, running colour, q -> conic and mean grads  50 FLOP + 2 MUFU
#   cutoff pair      decay weight recomputed and its gradient             135 FLOP + 5 MUFU
FLOP_BWD_WALKED, FLOP_BWD_EVAL, FLOP_BWD_CUT = 10, 50, 135


def run_training(args, rank=0, world=1):
    """Multi-layer differentiation workload: 3 nested shells (3 x 700k Gaussians, SH degree
    2), 64 views at 512^2 / 1024^2 / 1920x1080 with 64 planes cutting the shells. One step =
    batched forward (CUDA-graph replay, autotuned) + L2 loss to target renders of a perturbed
    copy of the scene + rara_render_backward + an Adam update of the Gaussians, as a
    data-parallel step (dp.data_parallel_gradients): with several ranks each renders and
    differentiates every world-th view and one all-reduce sums the parameter gradients."""
    import torch

    from paper_2506_20202_gb300 import autotune, dp, rara, scenes
    t_setup = time.perf_counter()
    scene, target, vp = scenes.shells_training_workload(args.train_per_shell, args.train_views, seed=3)
    gs = rara.GaussianTensors.from_scene(scene)
    tg = rara.GaussianTensors.from_scene(target)
    stream = torch.cuda.Stream()
    ctx = rara.rara_ctx_create(0)
    mine = dp.shard_views(len(vp), rank, world)

    def make_views(idx):
        out = []
        for k in idx:
            cam, pl = vp[k]
            H, W = cam.height, cam.width
            out.append(rara.View(0, cam, pl, torch.empty((3, H, W), device="cuda"),
                                 torch.empty((H, W), device="cuda"),
                                 torch.empty((H, W), dtype=torch.int32, device="cuda"), (0.0, 0.0, 0.0)))
        return out

    tviews = make_views(mine)
    rara.rara_render_batch(ctx, [tg], tviews, stream)
    rara.rara_ctx_sync(ctx, stream)
    targets = {k: v.image for k, v in zip(mine, tviews)}
    del tg
    local = dp.GpuViews(ctx, gs, vp, targets, stream)
    views = local._views(mine)[0]
    if args.tuning:
        best, tune_ms = autotune.parse(args.tuning), {}
        autotune.apply(ctx, best)
    else:
        # the tiling serves the backward too: tune on the forward + loss + backward of the views
        def step_ms(reps):
            local(mine)                                   # capture the forward's graph
            torch.cuda.synchronize()
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(torch.cuda.current_stream())
                local(mine)
                e1.record(torch.cuda.current_stream())
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            return statistics.median(times)
        best, tune_ms = autotune.autotune(ctx, [gs], views, stream, reps=2, timer=step_ms)
    grads = local.grads
    # Adam on the Gaussians' own storage (nn.Parameter shares it), gradients from the backward
    params = [torch.nn.Parameter(t) for t in (gs.means, gs.log_scales, gs.quats, gs.opacity_logits, gs.sh)]
    for p_, g_ in zip(params, (grads.means, grads.log_scales, grads.quats, grads.opacity_logits, grads.sh)):
        p_.grad = g_
    opt = torch.optim.Adam(params, lr=1e-3, foreach=True)
    losses = []

    def step(evs):
        cur = torch.cuda.current_stream()
        evs[0].record(stream)
        res = dp.data_parallel_gradients(lambda idx: local(idx, evs[1:4]), len(vp), rank, world)
        opt.step()
        evs[4].record(cur)
        return res.loss

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    # the forward's work counts (the backward's roofline units) from an exact render: graph
    # replays run the render without its counters
    rara.rara_ctx_count_work(ctx, True)
    rara.rara_render_batch(ctx, [gs], views, stream)
    rara.rara_ctx_count_work(ctx, False)
    info = rara.rara_frame_info_get(ctx, 0)
    for _ in range(2):
        step(mk())
    rara.rara_ctx_sync(ctx, stream)
    setup_s = time.perf_counter() - t_setup
    evs = [mk() for _ in range(args.train_steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(args.train_steps):
        losses.append(step(evs[k]))
    t1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    rara.rara_ctx_sync(ctx, stream)
    total_ms = t0.elapsed_time(t1)
    bwd_ms = rara.rara_ctx_backward_ms(ctx)
    med = lambda a, b: statistics.median(e[a].elapsed_time(e[b]) for e in evs)
    pixels = sum(vp[k][0].width * vp[k][0].height for k in mine)
    flop = (FLOP_BWD_WALKED * info["n_walked"] + FLOP_BWD_EVAL * info["n_evaluated"]
            + FLOP_BWD_CUT * info["n_cut_evaluated"])
    peak = sm_count() * FP32_LANES * 2 * 2070.0 * 1e6 / 1e12
    achieved = flop / (bwd_ms[0] * 1e-3) / 1e12
    out = {"workload": f"3 nested shells x {args.train_per_shell} Gaussians (SH 2), {len(vp)} views "
                       f"(512^2 / 1024^2 / 1920x1080), 64 planes cutting the shells, L2 loss to renders of a "
                       f"perturbed copy", "gaussians": scene.n, "views": len(vp), "views_this_rank": len(mine),
           "ranks": world, "pixels_per_step": pixels,
           "steps": args.train_steps, "ms_per_step": total_ms / args.train_steps,
           "views_per_s": args.train_steps * len(mine) / (total_ms * 1e-3),
           "stage_ms_median": {"forward_graph": med(0, 1), "loss_grad": med(1, 2), "backward": med(2, 3),
                               "allreduce_and_adam": med(3, 4)},
           "backward_kernels_ms_last": {"render_backward": bwd_ms[0], "preprocess_backward": bwd_ms[1]},
           "tuning": list(best), "loss_per_step": [float(x) for x in losses],
           "render_backward_roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                        "frac": achieved / peak,
                                        "units": {"walked": info["n_walked"], "evaluated": info["n_evaluated"],
                                                  "cut_evaluated": info["n_cut_evaluated"]}},
           "pairs": sum(rara.rara_frame_info_get(ctx, v)["n_pairs"] for v in range(len(views))),
           "setup_s": setup_s,
           "note": "a data-parallel step (views dealt round-robin over ranks, one all-reduce of the parameter "
                   "gradients; at one rank the all-reduce is skipped)"}
    rara.rara_ctx_destroy(ctx)
    del gs, grads, targets, tviews, views, local
    torch.cuda.empty_cache()
    return out


# The paper's render-efficiency comparison (Section 4.2, Table 1, RTX 4090, real captures at
# an unstated resolution; context only): frames/s without clipping, with hard clipping and
# with RaRa clipping over a plane sweep.
PAPER_TABLE1 = {"360garden (~4M Gaussians)": {"original": 77.82, "hard": 81.49, "rara": 81.47},
                "Hair (~3M Gaussians)": {"original": 128.02, "hard": 146.88, "rara": 145.46}}


def time_modes(gs, views_for_mode, steps, tuning, stream):
    """frames/s of one batched, graph-replayed batch per clipping mode (no clipping, hard
    clipping, RaRa), each on its own context (the pair capacity depends on the mode)."""
    import torch

    from paper_2506_20202_gb300 import autotune, rara, scenes
    out = {}
    for name, mode in (("original", scenes.MODE_NONE), ("hard", scenes.MODE_HARD), ("rara", scenes.MODE_RARA)):
        views = views_for_mode(mode)
        ctx = rara.rara_ctx_create(0)
        autotune.apply(ctx, tuning)
        for _ in range(3):
            rara.rara_render_batch_graph(ctx, [gs], views, stream)
        rara.rara_ctx_sync(ctx, stream)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            rara.rara_render_batch_graph(ctx, [gs], views, stream)
        t1.record(stream)
        stream.synchronize()
        rara.rara_ctx_sync(ctx, stream)
        render_ms = rara.rara_ctx_stage_ms(ctx)[2]
        rara.rara_ctx_destroy(ctx)
        out[name] = {"frames_per_s": steps * len(views) / (t0.elapsed_time(t1) / 1e3),
                     "render_ms_last_batch": render_ms}
    out["rara_over_hard"] = out["rara"]["frames_per_s"] / out["hard"]["frames_per_s"]
    out["rara_over_original"] = out["rara"]["frames_per_s"] / out["original"]["frames_per_s"]
    return out


def run_modes(args, gs, cam, planes, tuning):
    """Table 1's protocol on the general-scene sweep: the 16 sweep planes rendered without
    clipping, with hard clipping and with RaRa, each as one graph-replayed batch."""
    import torch

    from paper_2506_20202_gb300 import rara, scenes
    H, W = cam.height, cam.width
    stream = torch.cuda.Stream()
    outs = [(torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
             torch.empty((H, W), dtype=torch.int32, device="cuda")) for _ in planes]

    def views_for(mode):
        return [rara.View(0, cam, scenes.Plane(p.n, p.d, p.k_sigma, mode), o[0], o[1], o[2]) for p, o in zip(planes, outs)]

    res = time_modes(gs, views_for, args.mode_steps, tuning, stream)
    del outs
    torch.cuda.empty_cache()
    res["workload"] = "general scene 1M SH3, 1920x1080, the 16-offset plane sweep as one batch per mode"
    return res


def run_volume(args, gs, cam, planes):
    """Clip-volume sweep: the general scene's 16 sweep planes, each joined by a second fixed
    plane through the scene centre (normal n x (0, 1, 0), so the two planes meet along a line
    through the image) into a wedge, rendered as one batch of 16 frames, graph-replayed and
    autotuned like the single-plane sweep."""
    import numpy as np
    import torch

    from paper_2506_20202_gb300 import autotune, rara, scenes
    H, W = cam.height, cam.width
    stream = torch.cuda.Stream()
    m = np.cross(np.asarray(planes[0].n, np.float64), [0.0, 1.0, 0.0])
    m = np.float32(m / np.linalg.norm(m))
    extra = ((float(m[0]), float(m[1]), float(m[2]), 0.05),)
    vols = [scenes.Plane(p.n, p.d, p.k_sigma, p.mode, extra) for p in planes]
    ctx = rara.rara_ctx_create(0)
    views = [rara.View(0, cam, v, torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
                       torch.empty((H, W), dtype=torch.int32, device="cuda"), (0.0, 0.0, 0.0)) for v in vols]
    if args.tuning:
        best = autotune.parse(args.tuning)
        autotune.apply(ctx, best)
    else:
        best, _ = autotune.autotune(ctx, [gs], views, stream, reps=2)
    rara.rara_render_batch(ctx, [gs], views, stream)
    stage = rara.rara_ctx_stage_ms(ctx)
    info = [rara.rara_frame_info_get(ctx, v) for v in range(len(views))]
    for _ in range(3):
        rara.rara_render_batch_graph(ctx, [gs], views, stream)
    rara.rara_ctx_sync(ctx, stream)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.volume_steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for e in ev:
        e[0].record(stream)
        rara.rara_render_batch_graph(ctx, [gs], views, stream)
        e[1].record(stream)
    t1.record(stream)
    stream.synchronize()
    rara.rara_ctx_sync(ctx, stream)
    lat = [e[0].elapsed_time(e[1]) for e in ev]
    rara.rara_ctx_destroy(ctx)
    del views
    torch.cuda.empty_cache()
    n = gs.n
    return {"workload": "general scene 1M SH3, 1920x1080, 16-offset sweep, each plane joined by a second plane "
                        "(a wedge)",
            "frames_per_s": len(vols) * args.volume_steps / (t0.elapsed_time(t1) / 1e3),
            "batch_p50_ms": percentile(lat, 50), "batch_p99_ms": percentile(lat, 99), "tuning": list(best),
            "stage_ms_exact_batch": {"preprocess": stage[0], "bin": stage[1], "render": stage[2]},
            "cutoff_fraction_per_frame": [round(i["n_cutoff"] / n, 4) for i in info]}


def run_hair(args):
    """Hair-strand workload: 500k strand Gaussians (10,000 cubic curves x 50 segments, axis
    scales 1:1:40 along the tangent, SH 1) at 1024x1024 with an oblique plane cutting 30-50%
    of them. The plain path renders one frame per launch sequence from a fixed camera; the
    batched path renders 16 views on an orbit around the head as one graph replay."""
    import math

    import numpy as np
    import torch

    from paper_2506_20202_gb300 import autotune, rara, scenes
    scene, nrm, d = scenes.hair_scene(curves=10_000, segments=50, seed=0)
    gs = rara.GaussianTensors.from_scene(scene)
    pl = scenes.Plane(np.asarray(nrm, np.float32), float(d), 3.0, scenes.MODE_RARA)
    W = H = 1024
    cam = scenes.look_at_camera((0.2, -0.3, -3.2), (0.0, 0.3, 0.0), W, H, 60.0)
    stream = torch.cuda.Stream()
    out = {"workload": "hair strands: 500,000 Gaussians (10,000 curves x 50 segments, scales 1:1:40, SH 1), "
                       "1024x1024, one oblique plane"}
    ctx = rara.rara_ctx_create(0)
    img = torch.empty((3, H, W), device="cuda")
    T = torch.empty((H, W), device="cuda")
    nc = torch.empty((H, W), dtype=torch.int32, device="cuda")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.hair_steps)]

    def frame(e=None):
        if e is not None:
            e[0].record(stream)
        rara.rara_preprocess(ctx, gs, cam, pl, stream)
        rara.rara_bin(ctx, stream)
        rara.rara_render(ctx, (0.0, 0.0, 0.0), img, T, nc, stream)
        if e is not None:
            e[1].record(stream)

    for _ in range(3):
        frame()
    info = rara.rara_frame_info_get(ctx)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for e in ev:
        frame(e)
    t1.record(stream)
    stream.synchronize()
    lat = [e[0].elapsed_time(e[1]) for e in ev]
    out["plain"] = {"frames_per_s": args.hair_steps / (t0.elapsed_time(t1) / 1e3), "p50_ms": percentile(lat, 50),
                    "p99_ms": percentile(lat, 99)}
    out["cutoff_fraction_of_rendered"] = info["n_cutoff"] / max(1, info["n_rendered"])
    out["cutoff_fraction_of_all"] = info["n_cutoff"] / scene.n
    out["pairs"] = info["n_pairs"]
    rara.rara_ctx_destroy(ctx)
    # batched: 16 views on an orbit of radius 3.2 around the head, one graph replay per step
    bctx = rara.rara_ctx_create(0)
    views = []
    for k in range(16):
        a = 2.0 * math.pi * k / 16
        c = scenes.look_at_camera((3.2 * math.sin(a), -0.3, -3.2 * math.cos(a)), (0.0, 0.3, 0.0), W, H, 60.0)
        views.append(rara.View(0, c, pl, torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
                               torch.empty((H, W), dtype=torch.int32, device="cuda"), (0.0, 0.0, 0.0)))
    if args.tuning:
        best = autotune.parse(args.tuning)
        autotune.apply(bctx, best)
    else:
        best, _ = autotune.autotune(bctx, [gs], views, stream, reps=2)
    rara.rara_render_batch(bctx, [gs], views, stream)
    stage = rara.rara_ctx_stage_ms(bctx)
    for _ in range(3):
        rara.rara_render_batch_graph(bctx, [gs], views, stream)
    rara.rara_ctx_sync(bctx, stream)
    bev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.hair_steps)]
    torch.cuda.synchronize()
    t0.record(stream)
    for e in bev:
        e[0].record(stream)
        rara.rara_render_batch_graph(bctx, [gs], views, stream)
        e[1].record(stream)
    t1.record(stream)
    stream.synchronize()
    rara.rara_ctx_sync(bctx, stream)
    blat = [e[0].elapsed_time(e[1]) for e in bev]
    out["batched_graph"] = {"frames_per_s": 16 * args.hair_steps / (t0.elapsed_time(t1) / 1e3),
                            "batch_p50_ms": percentile(blat, 50), "batch_p99_ms": percentile(blat, 99),
                            "views_per_batch": 16, "tuning": list(best),
                            "stage_ms_exact_batch": {"preprocess": stage[0], "bin": stage[1], "render": stage[2]}}
    rara.rara_ctx_destroy(bctx)
    if args.mode_steps > 0:
        def views_for(mode):
            return [rara.View(0, v.camera, scenes.Plane(pl.n, pl.d, pl.k_sigma, mode), v.image, v.final_T, v.n_contrib)
                    for v in views]
        out["modes"] = time_modes(gs, views_for, args.mode_steps, best, stream)
        out["modes"]["workload"] = "hair strands, the 16 orbit views as one batch per mode"
    del gs, views
    torch.cuda.empty_cache()
    return out


def run_serving(args, gs_1m, scene_1m):
    """Continuous-batching server vs the plain one-request-per-launch path on the same
    seeded Poisson arrivals: resident scenes of 100k, 1M and 3M Gaussians, random scene,
    camera, resolution (512^2, 1280x720, 1920x1080) and plane per request, 60 GB budget.
    Both paths start warm: every scene x resolution rendered beforehand on their own
    contexts (kernels loaded, buffers grown / reserved) and pinned image pools filled."""
    import torch

    from paper_2506_20202_gb300 import rara, scenes, serve
    sc = {"100k": rara.GaussianTensors.from_scene(scenes.general_scene(100_000, seed=11)), "1M": gs_1m}
    if args.serve_3m:
        sc["3M"] = rara.GaussianTensors.from_scene(scenes.general_scene(3_000_000, seed=12))
    names = list(sc)
    out = {"scenes": names, "budget_gb": 60, "rate_hz": args.serve_rate, "window_s": args.serve_s}
    reqs = serve.poisson_requests(names, serve.orbit_camera, args.serve_rate, args.serve_s, seed=21)
    srv = serve.Server(sc, budget_bytes=60 << 30, slots=2, max_batch=64, keep_images=False)
    try:
        srv.warm(serve.orbit_camera, seed=22)
        out["reserved"] = srv.reserved
        res = srv.run(reqs)
        out["served"] = serve.summarize(res, args.serve_s)
        out["served"]["batches"] = srv.batches
        out["served"]["rejected"] = srv.rejected
        # the same arrivals 10x faster (a shorter window), where the GPU is the bottleneck
        fast = serve.poisson_requests(names, serve.orbit_camera, args.serve_rate * 10, args.serve_fast_s, seed=23)
        srv.batches = srv.rejected = 0
        res = srv.run(fast)
        out["served_10x_rate"] = serve.summarize(res)
        out["served_10x_rate"]["batches"] = srv.batches
    finally:
        srv.close()
    torch.cuda.synchronize()
    ctx, pool = serve.warm_plain(sc, serve.orbit_camera, seed=22)
    try:
        out["plain"] = serve.summarize(serve.serve_plain(sc, reqs, keep_images=False, ctx=ctx, pool=pool),
                                       args.serve_s)
        out["plain_10x_rate"] = serve.summarize(serve.serve_plain(sc, fast, keep_images=False, ctx=ctx, pool=pool))
    finally:
        rara.rara_ctx_destroy(ctx)
    out["p99_served_over_plain"] = out["served"]["p99_ms"] / out["plain"]["p99_ms"]
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
