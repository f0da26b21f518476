"""Autotuner for the render's tile shape, blend batch depth and work granularity.

Three knobs set how the render maps onto the GPU, none of which changes the image beyond
float rounding order (with one lane per pixel, not even that):
  - the screen tile (rara_ctx_set_tiling): 8x8, 16x16, 32x8, 8x32, 32x16 or 16x32 pixels;
    smaller tiles give shorter lists and more (Gaussian, tile) pairs to sort;
  - the blend batch depth: list entries staged in shared memory at a time (128, 256, 512
    by the whole block; deeper batches mean fewer block barriers and more staged entries a
    saturated pixel never reads), or 32 per warp, each warp walking the list on its own;
  - the split thresholds (rara_ctx_set_tuning): a tile with a long list is split into work
    items with 2 or 4 lanes per pixel.
Where each pays depends on the workload (list lengths, share of cutoff Gaussians,
resolution mix), so the tuner times candidates on the actual batch, through the captured-
graph path, by coordinate descent: split thresholds (16x16 tiles, depth 256), then tile
shapes, then depths, then the split thresholds again for the chosen tile and depth,
keeping the fastest of each. Results can be cached in a JSON
file keyed by the device name and the batch shape.
"""
from __future__ import annotations

import json
import os
import statistics

from . import rara

TILES = [(16, 16), (32, 8), (8, 32), (8, 8), (32, 16), (16, 32)]
DEPTHS = [256, 32, 128, 512]
# (split2_bits, split4_bits): a tile with >= 2^(bits-1) list entries is split
CANDIDATES = [(33, 33), (13, 14), (12, 13), (11, 12), (10, 11), (11, 13), (10, 12), (9, 11)]
DEFAULT = (16, 16, 256, 11, 12)


def apply(ctx, setting):
    """Set a (tile_w, tile_h, depth, split2_bits, split4_bits) setting on ctx."""
    tw, th, depth, s2, s4 = setting
    rara.rara_ctx_set_tiling(ctx, tw, th, depth)
    rara.rara_ctx_set_tuning(ctx, s2, s4)


def parse(text: str):
    """A setting from 'split2,split4' (16x16 tiles, depth 256) or 'tw,th,depth,split2,split4'."""
    v = tuple(int(x) for x in text.split(","))
    if len(v) == 2:
        return DEFAULT[:3] + v
    if len(v) == 5:
        return v
    raise ValueError(f"tuning '{text}': give split2,split4 or tile_w,tile_h,depth,split2,split4")


def _shape_key(scenes, views) -> str:
    import torch
    dev = torch.cuda.get_device_name()
    parts = [dev] + [f"s{g.n}:{g.sh_degree}" for g in scenes]
    parts += [f"v{v.scene}:{v.camera.width}x{v.camera.height}" for v in views]
    return "|".join(parts)


def time_batch(ctx, scenes, views, stream, reps: int = 5) -> float:
    """Median GPU milliseconds of a graph replay of the batch on `stream`."""
    import torch
    rara.rara_render_batch_graph(ctx, scenes, views, stream)   # exact render + capture
    rara.rara_ctx_sync(ctx, stream)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rara.rara_render_batch_graph(ctx, scenes, views, stream)
        e1.record(stream)
        rara.rara_ctx_sync(ctx, stream)
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def autotune(ctx, scenes, views, stream=None, reps: int = 5, tiles=None, depths=None, candidates=None,
             cache_path: str | None = None, timer=None):
    """Pick the fastest (tile_w, tile_h, depth, split2_bits, split4_bits) for this batch and
    set it on ctx.

    Returns (best, {setting: ms}). With cache_path, a stored choice for the same device and
    batch shape is reused without timing, and a new choice is stored. timer(reps), if given,
    times the candidate instead of the batch's graph replay (milliseconds): for example a
    whole differentiation step, whose backward runs on the forward's tiles too."""
    import torch
    stream = stream or torch.cuda.current_stream()
    key = _shape_key(scenes, views)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if key in cache:
            best = tuple(cache[key]["best"])
            apply(ctx, best)
            return best, {tuple(json.loads(k)): v for k, v in cache[key]["ms"].items()}
    results = {}

    def trial(setting):
        if setting not in results:
            apply(ctx, setting)
            results[setting] = timer(reps) if timer else time_batch(ctx, scenes, views, stream, reps)
        return results[setting]

    best = DEFAULT

    def splits():
        nonlocal best
        for s2, s4 in candidates or CANDIDATES:
            cand = best[:3] + (s2, s4)
            if trial(cand) < trial(best):
                best = cand

    splits()                          # at the default tile, so tiles are compared at a good split
    first = best
    for tw, th in tiles or TILES:
        cand = (tw, th) + best[2:]
        if trial(cand) < trial(best):
            best = cand
    for depth in depths or DEPTHS:
        cand = best[:2] + (depth,) + best[3:]
        if trial(cand) < trial(best):
            best = cand
    if best[:3] != first[:3]:
        splits()                      # the split that suits the chosen tile and depth
    apply(ctx, best)
    if cache_path:
        cache[key] = {"best": list(best), "ms": {json.dumps(list(k)): v for k, v in results.items()}}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best, results
