"""Autotuner for the render's work granularity.

The render splits a tile with a long list into 2 or 4 work items with 2 or 4 lanes per
pixel (rara_ctx_set_tuning). Where the split pays depends on the workload (list lengths,
share of cutoff Gaussians, resolution mix), so the tuner times candidate thresholds on the
actual batch, through the captured-graph path, and keeps the fastest. Images do not depend
on the choice beyond float rounding order. Results can be cached in a JSON file keyed by
the device name and the batch shape.
"""
from __future__ import annotations

import json
import os
import statistics

from . import rara

# (split2_bits, split4_bits): a tile with >= 2^(bits-1) list entries is split
CANDIDATES = [(33, 33), (13, 14), (12, 13), (11, 12), (10, 11), (11, 13), (10, 12), (9, 11)]


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


def autotune(ctx, scenes, views, stream=None, reps: int = 5, candidates=None, cache_path: str | None = None):
    """Pick the fastest split thresholds for this batch and set them on ctx.

    Returns (best, {candidate: ms}). With cache_path, a stored choice for the same device
    and batch shape is reused without timing, and a new choice is stored."""
    import torch
    stream = stream or torch.cuda.current_stream()
    key = _shape_key(scenes, views)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if key in cache:
            best = tuple(cache[key]["best"])
            rara.rara_ctx_set_tuning(ctx, *best)
            return best, {tuple(json.loads(k)): v for k, v in cache[key]["ms"].items()}
    results = {}
    for cand in candidates or CANDIDATES:
        rara.rara_ctx_set_tuning(ctx, *cand)
        results[tuple(cand)] = time_batch(ctx, scenes, views, stream, reps)
    best = min(results, key=results.get)
    rara.rara_ctx_set_tuning(ctx, *best)
    if cache_path:
        cache[key] = {"best": list(best), "ms": {json.dumps(list(k)): v for k, v in results.items()}}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best, results
