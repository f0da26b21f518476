"""Serving loop for clipped renders: continuous batching over resident scenes.

Requests (scene, camera, resolution, clip plane) arrive over time. The server keeps the
scenes resident on the device and runs up to `slots` batches at once, each on its own
CUDA stream and render context (scratch stays allocated across batches). Whenever a slot
is free, every queued request that fits the device-memory budget is admitted into one
batch and launched with rara_render_batch (one launch per stage for the whole batch), so
requests that arrive while other batches are on the GPU join the next batch and their work
overlaps on the device with the batches already running. Each result's image is copied
back to pinned host memory on the batch's stream; a request's latency runs from its
arrival to the moment its batch's copy has finished.

The plain baseline serves the same arrivals one request per launch sequence
(rara_render_frame on one stream, in arrival order).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import rara


@dataclasses.dataclass
class Request:
    rid: int
    scene: str
    camera: object
    plane: object
    bg: tuple = (0.0, 0.0, 0.0)
    arrival: float = 0.0      # seconds since the start of the run


@dataclasses.dataclass
class Result:
    rid: int
    image: "torch.Tensor"     # pinned host [3, H, W]
    arrival: float
    done: float

    @property
    def latency_ms(self) -> float:
        return (self.done - self.arrival) * 1e3


# Device bytes one view of a scene of n Gaussians at W x H needs inside a render context:
# per-(view, Gaussian) slot ~145 B (label, tiles, rectangle, 48 B record, 64 B ray-tracing
# record, depth, two sort buffers) plus pairs (assume 8 tiles per Gaussian, 16 B per pair)
# and the outputs (image, transmittance, n_contrib).
def request_bytes(n: int, width: int, height: int) -> int:
    return n * 145 + n * 8 * 16 + width * height * 20


class _PinnedPool:
    """Reusable pinned host images, one free list per resolution."""

    def __init__(self):
        self.free = {}

    def get(self, H, W):
        import torch
        lst = self.free.get((H, W))
        if lst:
            return lst.pop()
        return torch.empty((3, H, W), dtype=torch.float32, pin_memory=True)

    def put(self, t):
        self.free.setdefault((t.shape[1], t.shape[2]), []).append(t)


class _Slot:
    def __init__(self, budget):
        import torch
        self.stream = torch.cuda.Stream()
        self.ctx = rara.rara_ctx_create(budget)
        self.event = torch.cuda.Event()
        self.batch = None      # list of (request, outputs, host image)
        self.bytes = 0

    def close(self):
        rara.rara_ctx_destroy(self.ctx)


class Server:
    def __init__(self, scenes: dict, budget_bytes: int = 60 << 30, slots: int = 2, max_batch: int = 64,
                 keep_images: bool = True):
        import torch
        self.keep_images = keep_images
        self.pool = _PinnedPool()
        self.scenes = {k: v for k, v in scenes.items()}          # name -> GaussianTensors (resident)
        self.names = list(self.scenes)
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        resident = sum(sum(t.numel() * 4 for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh))
                       for g in self.scenes.values())
        self.free_bytes = self.budget - resident
        if self.free_bytes <= 0:
            raise ValueError("the resident scenes exceed the memory budget")
        self.slots = [_Slot(self.free_bytes) for _ in range(slots)]  # cap per slot; admission shares the budget
        self.queue: list[Request] = []
        self.results: dict[int, Result] = {}
        self.batches = 0
        self.rejected = 0
        self.t0 = None
        self._torch = torch

    def close(self):
        for s in self.slots:
            s.close()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        n = self.scenes[req.scene].n
        if request_bytes(n, req.camera.width, req.camera.height) > self.free_bytes // len(self.slots):
            self.rejected += 1       # can never fit one slot's share of the budget
            return
        self.queue.append(req)

    def _collect(self, block: bool = False):
        for s in self.slots:
            if s.batch is None:
                continue
            if block:
                s.event.synchronize()
            elif not s.event.query():
                continue
            t = self.now()
            rara.rara_ctx_sync(s.ctx, s.stream)
            for req, _, host in s.batch:
                self.results[req.rid] = Result(req.rid, host if self.keep_images else None, req.arrival, t)
                if not self.keep_images:
                    self.pool.put(host)
            s.batch = None
            s.bytes = 0

    def _launch(self, s: _Slot):
        torch = self._torch
        share = self.free_bytes // len(self.slots)
        take, used = [], 0
        while self.queue and len(take) < self.max_batch:
            req = self.queue[0]
            b = request_bytes(self.scenes[req.scene].n, req.camera.width, req.camera.height)
            if take and used + b > share:
                break
            take.append(self.queue.pop(0))
            used += b
        if not take:
            return
        names = sorted({r.scene for r in take}, key=self.names.index)
        scene_idx = {nm: i for i, nm in enumerate(names)}
        batch, views = [], []
        with torch.cuda.stream(s.stream):
            for req in take:
                H, W = req.camera.height, req.camera.width
                img = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
                host = self.pool.get(H, W)
                views.append(rara.View(scene_idx[req.scene], req.camera, req.plane, img, None, None, req.bg))
                batch.append((req, img, host))
        rara.rara_render_batch(s.ctx, [self.scenes[nm] for nm in names], views, s.stream)
        with torch.cuda.stream(s.stream):
            for _, img, host in batch:
                host.copy_(img, non_blocking=True)
        s.event.record(s.stream)
        s.batch = batch
        s.bytes = used
        self.batches += 1

    def step(self):
        self._collect()
        for s in self.slots:
            if s.batch is None and self.queue:
                self._launch(s)

    def run(self, requests: list[Request]) -> list[Result]:
        """Serve `requests` (sorted by arrival time) in real time; return their results."""
        self.t0 = time.perf_counter()
        pending = list(requests)
        k = 0
        while k < len(pending) or self.queue or any(s.batch is not None for s in self.slots):
            t = self.now()
            while k < len(pending) and pending[k].arrival <= t:
                self.submit(pending[k])
                k += 1
            self.step()
            if k < len(pending) and not self.queue and all(s.batch is None for s in self.slots):
                time.sleep(max(0.0, min(pending[k].arrival - self.now(), 0.002)))
        self._collect(block=True)
        return [self.results[r.rid] for r in requests if r.rid in self.results]


def serve_plain(scenes: dict, requests: list[Request], keep_images: bool = True) -> list[Result]:
    """Baseline: one request per launch sequence, on one stream, in arrival order."""
    import torch
    stream = torch.cuda.Stream()
    ctx = rara.rara_ctx_create(0)
    pool = _PinnedPool()
    results = []
    t0 = time.perf_counter()
    try:
        for req in requests:
            now = time.perf_counter() - t0
            if req.arrival > now:
                time.sleep(req.arrival - now)
            H, W = req.camera.height, req.camera.width
            with torch.cuda.stream(stream):
                img = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
                host = pool.get(H, W) if not keep_images else \
                    torch.empty((3, H, W), dtype=torch.float32, pin_memory=True)
            rara.rara_render_frame(ctx, scenes[req.scene], req.camera, req.plane, req.bg, img, None, None, stream)
            with torch.cuda.stream(stream):
                host.copy_(img, non_blocking=True)
            stream.synchronize()
            results.append(Result(req.rid, host if keep_images else None, req.arrival, time.perf_counter() - t0))
            if not keep_images:
                pool.put(host)
    finally:
        rara.rara_ctx_destroy(ctx)
    return results


def poisson_requests(scene_names, cameras_for, rate_hz: float, duration_s: float, seed: int = 0,
                     resolutions=((512, 512), (1280, 720), (1920, 1080))) -> list[Request]:
    """Seeded Poisson arrivals with a random scene, camera, resolution and clip plane each.
    cameras_for(rng, width, height) returns a camera; planes cut through the scene."""
    from . import scenes as sc
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        plane = sc.Plane(np.float32(nrm), float(rng.uniform(-0.5, 0.5)), 3.0, sc.MODE_RARA)
        reqs.append(Request(len(reqs), scene_names[int(rng.integers(len(scene_names)))], cameras_for(rng, w, h),
                            plane, (0.0, 0.0, 0.0), t))
    return reqs


def orbit_camera(rng, width, height, distance: float = 3.0):
    from . import scenes as sc
    v = rng.standard_normal(3)
    v = distance * v / np.linalg.norm(v)
    return sc.look_at_camera(v, (0.0, 0.0, 0.0), width, height, 60.0)


def summarize(results: list[Result], wall_s: float | None = None) -> dict:
    lat = np.array([r.latency_ms for r in results])
    if wall_s is None:
        wall_s = max(r.done for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "frames_per_s": len(results) / wall_s if wall_s > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
