"""Data-parallel differentiation and view-parallel rendering over ranks (one GPU per rank).

The clipped render shards by view: every rank renders its own views of a replicated scene
with no exchange, and a data-parallel differentiation step has exactly one: the sum over
ranks of the Gaussians' parameter gradients (about (59 + 1) floats per Gaussian at SH
degree 3), done here as one all-reduce of one flat buffer (NCCL between GPUs, gloo on CPU).
Each view's clip-plane gradient belongs to that view and stays on the rank that rendered it.
After the all-reduce every rank holds the same gradients, so identical optimiser steps keep
the replicas identical with no parameter broadcast.

Views are dealt round-robin (view v on rank v mod world), which spreads a batch's mixed
resolutions evenly over the ranks.
"""
from __future__ import annotations

import dataclasses

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def shard_views(num_views: int, rank: int, world: int) -> list[int]:
    """The views rank `rank` of `world` renders."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} of {world}")
    return list(range(rank, num_views, world))


def allreduce_sum(tensors, group=None):
    """Sum the tensors over the ranks of the process group, in place, with one collective on
    one contiguous buffer (no-op without an initialised group of more than one rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1 or not tensors:
        return tensors
    flat = torch.cat([t.reshape(-1) for t in tensors])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for t in tensors:
        n = t.numel()
        t.copy_(flat[off:off + n].view_as(t))
        off += n
    return tensors


@dataclasses.dataclass
class StepResult:
    loss: "torch.Tensor"        # [1], summed over all ranks' views (left on the device: no host wait)
    grads: dict                 # parameter name -> gradient, summed over all ranks (identical on every rank)
    plane_grads: dict           # view index -> dL/d(n, d) of this rank's views
    views: list                 # the view indices this rank rendered


def data_parallel_gradients(local_fn, num_views: int, rank: int, world: int, group=None) -> StepResult:
    """One data-parallel differentiation step. local_fn(view_indices) renders and
    differentiates this rank's views and returns (loss tensor, {name: gradient tensor},
    {view: plane gradient}); the losses and parameter gradients are then summed over ranks."""
    import torch
    mine = shard_views(num_views, rank, world)
    loss, grads, plane_grads = local_fn(mine)
    loss_t = torch.as_tensor(loss, dtype=grads[PARAMS[0]].dtype, device=grads[PARAMS[0]].device).reshape(1).clone()
    allreduce_sum([loss_t] + [grads[k] for k in PARAMS], group)
    return StepResult(loss_t, grads, plane_grads, mine)


class GpuViews:
    """This rank's share of a differentiation workload on its GPU: the L2 loss of rendered
    views against target images and its gradient through rara_render_backward, as the
    local_fn of data_parallel_gradients. The rank's views are rendered as one batch
    (replayed as a CUDA graph once captured); scene: GaussianTensors (replicated)."""

    def __init__(self, ctx, scene, cameras_planes, targets, stream=None, bg=(0.0, 0.0, 0.0)):
        import torch

        from . import rara
        self.rara = rara
        self.ctx = ctx
        self.scene = scene
        self.all = list(cameras_planes)
        self.targets = targets
        self.stream = stream or torch.cuda.current_stream()
        self.bg = bg
        self.views = {}
        self.grads = scene.empty_like()

    def _views(self, idx):
        import torch
        key = tuple(idx)
        if key not in self.views:
            vv = []
            for v in idx:
                cam, pl = self.all[v]
                H, W = cam.height, cam.width
                vv.append(self.rara.View(0, cam, pl, torch.empty((3, H, W), device="cuda"),
                                         torch.empty((H, W), device="cuda"),
                                         torch.empty((H, W), dtype=torch.int32, device="cuda"), self.bg))
            self.views[key] = (vv, [torch.empty_like(x.image) for x in vv],
                               torch.empty((len(vv), 4), device="cuda"),
                               torch.empty(len(vv), dtype=torch.float64, device="cuda"))
        return self.views[key]

    def __call__(self, idx, events=None):
        """Loss and gradients of views idx; events (3 CUDA events or None) are recorded
        after the forward, the loss gradient and the backward. The work waits for the caller's
        current stream first (the previous optimiser step ran there), and the caller's stream
        is made to wait for it (the all-reduce and the optimiser run there)."""
        import torch
        rara = self.rara
        views, dimgs, pg, lv = self._views(idx)
        # the render reads the parameters the caller's stream last updated (the optimiser step)
        self.stream.wait_stream(torch.cuda.current_stream())
        if not views:
            return torch.zeros((), device="cuda"), {k: getattr(self.grads, k).zero_() for k in PARAMS}, {}
        rara.rara_render_batch_graph(self.ctx, [self.scene], views, self.stream)
        if events:
            events[0].record(self.stream)
        # per-view mean squared error and its gradient, one launch for the batch
        rara.rara_loss_l2(self.ctx, [self.targets[k] for k in idx], dimgs, [1.0 / d.numel() for d in dimgs], lv,
                          self.stream)
        with torch.cuda.stream(self.stream):
            loss = lv.sum().float()
        if events:
            events[1].record(self.stream)
        rara.rara_render_backward(self.ctx, dimgs, [self.grads], pg, self.stream)
        if events:
            events[2].record(self.stream)
        torch.cuda.current_stream().wait_stream(self.stream)
        grads = {k: getattr(self.grads, k) for k in PARAMS}
        return loss, grads, {k: pg[i] for i, k in enumerate(idx)}
