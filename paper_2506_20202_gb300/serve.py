"""Serving loop for clipped renders: continuous batching over resident scenes.

Requests (scene, camera, resolution, clip plane) arrive over time. The server keeps the
scenes resident on the device and runs up to `slots` batches at once. Each slot has its own
CUDA stream, render context and host thread: the admission loop never waits for the GPU,
and a slot's thread alone waits for its batch (the pair-count read of rara_render_batch and
the image read-back). Whenever a slot is free, the queued requests (oldest first) that fit
the slot's reserved scratch are admitted into one batch and handed to the slot's thread,
which renders them with rara_render_batch (one launch per stage for the whole batch) and
copies the images back to pinned host memory on the slot's stream. Requests that arrive
while batches are on the GPU wait for the next free slot and run alongside the batches
already in flight. A request's latency runs from its arrival to the moment its image is in
host memory.

Memory: the byte budget (default 60 GB) minus the resident scenes is split evenly over the
slots; each slot's context is created with its share as its cap, so the contexts together
never hold more than the budget, and its scratch is reserved up front (rara_ctx_reserve)
for `reserve_batch` requests of the largest scene at the largest resolution, from pair
counts measured while warming up, so no allocation (and no device-wide synchronisation of
cudaFree / cudaMalloc) happens inside the serving window. A request whose estimated bytes
exceed a slot's share is refused at admission; a batch the context still refuses
(RARA_ERR_BUDGET) is split in halves and retried.

The plain baseline serves the same arrivals one request per launch sequence
(rara_render_frame on one stream, in arrival order).
"""
from __future__ import annotations

import dataclasses
import threading
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


# Device bytes of one (view, Gaussian) slot inside a render context: label 1, tiles 4,
# rectangle 8, splat record 48, ray-tracing record 64, depth 4, four compaction/sort words 16
# (plus look-back words); of one listed pair: four sort words 16 (+ sort scratch); of one
# output pixel: image 12, final transmittance 4, last index 4.
SLOT_BYTES, PAIR_BYTES, PIXEL_BYTES = 150, 20, 20


def request_bytes(n: int, width: int, height: int, pairs: int | None = None) -> int:
    """Device bytes one request needs; `pairs` defaults to 8 rectangle tiles per Gaussian."""
    pairs = 8 * n if pairs is None else pairs
    return n * SLOT_BYTES + pairs * PAIR_BYTES + width * height * PIXEL_BYTES


class _PinnedPool:
    """Reusable pinned host images, one free list per resolution (thread-safe)."""

    def __init__(self):
        self.free = {}
        self.lock = threading.Lock()

    def get(self, H, W):
        import torch
        with self.lock:
            lst = self.free.get((H, W))
            if lst:
                return lst.pop()
        return torch.empty((3, H, W), dtype=torch.float32, pin_memory=True)

    def put(self, t):
        with self.lock:
            self.free.setdefault((t.shape[1], t.shape[2]), []).append(t)

    def fill(self, H, W, count):
        got = [self.get(H, W) for _ in range(count)]
        for t in got:
            self.put(t)


class _Slot:
    def __init__(self, server: "Server", share: int):
        import torch
        self.server = server
        self.device = torch.cuda.current_device()
        self.stream = torch.cuda.Stream()
        self.share = share
        self.ctx = rara.rara_ctx_create(share)   # the slot's share of the budget caps its context
        self.job = None
        self.busy = False
        self.go = threading.Event()
        self.stop = False
        self.error = None
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def _loop(self):
        import torch
        torch.cuda.set_device(self.device)
        while True:
            self.go.wait()
            self.go.clear()
            if self.stop:
                return
            take = self.job
            try:
                self._serve(take)
            except Exception as e:  # surfaced by Server.run
                self.error = e
            finally:
                self.job = None
                self.server._slot_done(self)

    def _render(self, take):
        """rara_render_batch of `take`; a batch the context refuses for its budget is split."""
        import torch
        srv = self.server
        names = sorted({r.scene for r in take}, key=srv.names.index)
        scene_idx = {nm: i for i, nm in enumerate(names)}
        views, imgs = [], []
        with torch.cuda.stream(self.stream):
            for req in take:
                img = torch.empty((3, req.camera.height, req.camera.width), dtype=torch.float32, device="cuda")
                views.append(rara.View(scene_idx[req.scene], req.camera, req.plane, img, None, None, req.bg))
                imgs.append(img)
        try:
            rara.rara_render_batch(self.ctx, [srv.scenes[nm] for nm in names], views, self.stream)
        except rara.RaraError as e:
            if e.code != rara.RARA_ERR_BUDGET:
                raise
            if len(take) == 1:
                return [(take[0], None)]
            h = len(take) // 2
            return self._render(take[:h]) + self._render(take[h:])
        out = []
        with torch.cuda.stream(self.stream):
            for req, img in zip(take, imgs):
                host = srv.pool.get(req.camera.height, req.camera.width)
                host.copy_(img, non_blocking=True)
                out.append((req, host))
        return out

    def _serve(self, take):
        srv = self.server
        done = self._render(take)
        self.stream.synchronize()
        t = srv.now()
        with srv.lock:
            for req, host in done:
                if host is None:
                    srv.rejected += 1
                    continue
                srv.results[req.rid] = Result(req.rid, host if srv.keep_images else None, req.arrival, t)
                if not srv.keep_images:
                    srv.pool.put(host)

    def close(self):
        self.stop = True
        self.go.set()
        self.thread.join(timeout=30)
        rara.rara_ctx_destroy(self.ctx)


class Server:
    """Continuous-batching server over resident scenes (see the module docstring).

    scenes: name -> GaussianTensors (resident); resolutions: the (W, H) sizes requests use
    (warmed and reserved for); reserve_batch: how many requests of the largest scene at the
    largest resolution each slot's reserved scratch holds; max_batch: requests per batch.
    """

    def __init__(self, scenes: dict, budget_bytes: int = 60 << 30, slots: int = 2, max_batch: int = 64,
                 keep_images: bool = True, resolutions=((512, 512), (1280, 720), (1920, 1080)),
                 reserve_batch: int = 4):
        import torch
        self.keep_images = keep_images
        self.pool = _PinnedPool()
        self.scenes = {k: v for k, v in scenes.items()}          # name -> GaussianTensors (resident)
        self.names = list(self.scenes)
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.resolutions = [tuple(r) for r in resolutions]
        self.reserve_batch = reserve_batch
        resident = sum(sum(t.numel() * 4 for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh))
                       for g in self.scenes.values())
        self.free_bytes = self.budget - resident
        if self.free_bytes <= 0:
            raise ValueError("the resident scenes exceed the memory budget")
        self.share = self.free_bytes // slots
        self.pairs = {}          # (scene, W, H) -> candidate pairs per request (measured, with margin)
        self.queue: list[Request] = []
        self.results: dict[int, Result] = {}
        self.batches = 0
        self.rejected = 0
        self.t0 = time.perf_counter()
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.slots = [_Slot(self, self.share) for _ in range(slots)]
        self.reserved = None
        self._torch = torch

    def close(self):
        for s in self.slots:
            s.close()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ---------------------------------------------------------------- sizes and warm-up
    def _pairs(self, name, W, H) -> int:
        p = self.pairs.get((name, W, H))
        return p if p is not None else 8 * self.scenes[name].n

    def _bytes(self, req) -> int:
        W, H = req.camera.width, req.camera.height
        return request_bytes(self.scenes[req.scene].n, W, H, self._pairs(req.scene, W, H))

    def warm(self, cameras_for, seed: int = 0, per_shape: int = 2, pinned_per_res: int = 8):
        """Render every scene at every resolution on every slot (kernels loaded, pair counts
        measured), reserve each slot's scratch, and fill the pinned image pool."""
        import torch
        rng = np.random.default_rng(seed)
        from . import scenes as sc
        for s in self.slots:
            for name in self.names:
                for (W, H) in self.resolutions:
                    for _ in range(per_shape):
                        cam = cameras_for(rng, W, H)
                        nrm = rng.standard_normal(3)
                        nrm /= np.linalg.norm(nrm)
                        pl = sc.Plane(np.float32(nrm), float(rng.uniform(-0.5, 0.5)), 3.0, sc.MODE_RARA)
                        img = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
                        v = rara.View(0, cam, pl, img)
                        rara.rara_render_batch(s.ctx, [self.scenes[name]], [v], s.stream)
                        cand = rara.rara_frame_info_get(s.ctx, 0)["n_pair_candidates"]
                        key = (name, W, H)
                        self.pairs[key] = max(self.pairs.get(key, 0), int(1.5 * cand) + 4096)
            s.stream.synchronize()
        big = max(self.names, key=lambda nm: self.scenes[nm].n)
        Wb, Hb = max(self.resolutions, key=lambda r: r[0] * r[1])
        nres = self.reserve_batch
        slots_res = nres * self.scenes[big].n
        pairs_res = max(nres * max(self.pairs.values()), 1)
        tiles = max(((W + 15) // 16) * ((H + 15) // 16) for W, H in self.resolutions)
        for s in self.slots:
            # as much of the reservation as the slot's share holds (the rest grows on demand)
            for frac in (1.0, 0.5, 0.25):
                try:
                    rara.rara_ctx_reserve(s.ctx, int(slots_res * frac), int(pairs_res * frac), self.max_batch, tiles)
                    break
                except rara.RaraError as e:
                    if e.code != rara.RARA_ERR_BUDGET:
                        raise
        self.reserved = {"requests": nres, "slots": slots_res, "pairs": pairs_res,
                         "bytes_per_slot_context": [rara.rara_ctx_bytes(s.ctx) for s in self.slots]}
        for (W, H) in self.resolutions:
            self.pool.fill(H, W, pinned_per_res)
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- request loop
    def submit(self, req: Request):
        if self._bytes(req) > self.share:
            self.rejected += 1       # can never fit one slot's share of the budget
            return
        self.queue.append(req)

    def _slot_done(self, s: _Slot):
        with self.lock:
            s.busy = False
        self.wake.set()

    def _launch(self, s: _Slot):
        cap_slots = (self.reserved or {}).get("slots")
        cap_pairs = (self.reserved or {}).get("pairs")
        take, used, n_used, p_used = [], 0, 0, 0
        while self.queue and len(take) < self.max_batch:
            req = self.queue[0]
            W, H = req.camera.width, req.camera.height
            b, n, p = self._bytes(req), self.scenes[req.scene].n, self._pairs(req.scene, W, H)
            if take and (used + b > self.share or (cap_slots and n_used + n > cap_slots)
                         or (cap_pairs and p_used + p > cap_pairs)):
                break
            take.append(self.queue.pop(0))
            used, n_used, p_used = used + b, n_used + n, p_used + p
        if not take:
            return
        with self.lock:
            s.busy = True
        s.job = take
        self.batches += 1
        s.go.set()

    def run(self, requests: list[Request]) -> list[Result]:
        """Serve `requests` (sorted by arrival time) in real time; return their results."""
        self.t0 = time.perf_counter()
        self.results = {}
        pending = list(requests)
        k = 0
        while True:
            self.wake.clear()
            t = self.now()
            while k < len(pending) and pending[k].arrival <= t:
                self.submit(pending[k])
                k += 1
            for s in self.slots:
                if not self.queue:
                    break
                if not s.busy:
                    self._launch(s)
            for s in self.slots:
                if s.error is not None:
                    raise s.error
            with self.lock:
                idle = not any(s.busy for s in self.slots)
            if k >= len(pending) and not self.queue and idle:
                break
            wait = pending[k].arrival - self.now() if k < len(pending) else 0.01
            if self.queue:
                wait = 0.01      # a slot will free up and wake the loop
            if wait > 0:
                self.wake.wait(timeout=min(wait, 0.01))
        with self.lock:
            return [self.results[r.rid] for r in requests if r.rid in self.results]


def serve_plain(scenes: dict, requests: list[Request], keep_images: bool = True, ctx=None,
                pool: _PinnedPool | None = None) -> list[Result]:
    """Baseline: one request per launch sequence, on one stream, in arrival order. A context
    and pinned pool warmed by warm_plain can be passed in."""
    import torch
    stream = torch.cuda.Stream()
    own = ctx is None
    ctx = rara.rara_ctx_create(0) if own else ctx
    pool = pool or _PinnedPool()
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
        if own:
            rara.rara_ctx_destroy(ctx)
    return results


def warm_plain(scenes: dict, cameras_for, resolutions=((512, 512), (1280, 720), (1920, 1080)), seed: int = 0,
               per_shape: int = 2, pinned_per_res: int = 4):
    """A context and pinned pool for serve_plain with every scene x resolution rendered once
    (buffers grown to the largest shape, kernels loaded): the same warm start the server gets."""
    reqs = []
    rng = np.random.default_rng(seed)
    from . import scenes as sc
    for name in scenes:
        for (W, H) in resolutions:
            for _ in range(per_shape):
                nrm = rng.standard_normal(3)
                nrm /= np.linalg.norm(nrm)
                pl = sc.Plane(np.float32(nrm), float(rng.uniform(-0.5, 0.5)), 3.0, sc.MODE_RARA)
                reqs.append(Request(len(reqs), name, cameras_for(rng, W, H), pl))
    ctx = rara.rara_ctx_create(0)
    pool = _PinnedPool()
    for (W, H) in resolutions:
        pool.fill(H, W, pinned_per_res)
    serve_plain(scenes, reqs, keep_images=False, ctx=ctx, pool=pool)
    return ctx, pool


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
