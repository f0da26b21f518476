"""Differentiable clipped render: a torch.autograd.Function over the C ABI.

render_views() renders every camera's view of one scene as one batch (rara_render_batch,
or its captured CUDA graph) and returns the images; their backward is
rara_render_backward, which gives the gradients of the means, log-scales, quaternions,
opacity logits and SH coefficients, and of each view's clip plane (n, d). Both directions
run in the CUDA library; this module only marshals tensors.

The backward reads the render context's state of the forward (tile lists, per-pixel final
transmittance and last contributor), so a Renderer serves one differentiable forward at a
time: running another forward on it before the backward raises in the backward.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rara
from . import scenes as sc


class _RenderViews(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, sh_degree, cameras, k_sigmas, modes, bgs, graph, means, log_scales, quats,
                opacity_logits, sh, planes):
        dev = means.device
        g = rara.GaussianTensors(means.detach().contiguous(), log_scales.detach().contiguous(),
                                 quats.detach().contiguous(), opacity_logits.detach().contiguous(),
                                 sh.detach().contiguous(), int(sh_degree))
        pl = planes.detach().to("cpu", torch.float32).numpy()
        views = []
        for v, cam in enumerate(cameras):
            H, W = int(cam.height), int(cam.width)
            plane = sc.Plane(np.ascontiguousarray(pl[v, :3]), float(pl[v, 3]), float(k_sigmas[v]), int(modes[v]))
            views.append(rara.View(0, cam, plane, torch.empty((3, H, W), dtype=torch.float32, device=dev),
                                   torch.empty((H, W), dtype=torch.float32, device=dev),
                                   torch.empty((H, W), dtype=torch.int32, device=dev), tuple(bgs[v])))
        fn = rara.rara_render_batch_graph if graph else rara.rara_render_batch
        fn(renderer.ctx, [g], views)
        renderer.generation += 1
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        ctx.views = views
        ctx.gaussians = g
        return tuple(v.image for v in views)

    @staticmethod
    def backward(ctx, *grad_images):
        r = ctx.renderer
        if r.generation != ctx.generation:
            raise RuntimeError("the Renderer ran another forward after this one; its backward needs the "
                               "forward's state (use one Renderer per pending backward)")
        dimgs = [(gi if gi is not None else torch.zeros_like(v.image)).to(torch.float32).contiguous()
                 for gi, v in zip(grad_images, ctx.views)]
        grads = ctx.gaussians.empty_like()
        pg = torch.empty((len(ctx.views), 4), dtype=torch.float32, device=dimgs[0].device)
        rara.rara_render_backward(r.ctx, dimgs, [grads], pg)
        return (None,) * 7 + (grads.means, grads.log_scales, grads.quats, grads.opacity_logits, grads.sh, pg)


def render_views(renderer: "rara.Renderer", means, log_scales, quats, opacity_logits, sh, sh_degree: int,
                 cameras, planes, k_sigma=3.0, modes=sc.MODE_RARA, bgs=(0.0, 0.0, 0.0), graph: bool = False):
    """Render len(cameras) views of one scene; differentiable in the Gaussian tensors and in
    planes ([V, 4] tensor of (n.x, n.y, n.z, d) per view).

    Tensors use the planar layouts of rara_gaussians (means [3, n], log_scales [3, n],
    quats [4, n], opacity_logits [n], sh [(L+1)^2 * 3, n]) on the CUDA device. k_sigma,
    modes and bgs are one value for all views or one per view. Returns a tuple of [3, H, W]
    images."""
    V = len(cameras)
    ks = list(k_sigma) if np.ndim(k_sigma) else [k_sigma] * V
    ms = list(modes) if np.ndim(modes) else [modes] * V
    bg = list(bgs) if np.ndim(bgs) == 2 else [tuple(bgs)] * V
    if planes.shape != (V, 4):
        raise ValueError(f"planes must be [{V}, 4], got {tuple(planes.shape)}")
    return _RenderViews.apply(renderer, sh_degree, list(cameras), ks, ms, bg, graph, means, log_scales, quats,
                              opacity_logits, sh, planes)
