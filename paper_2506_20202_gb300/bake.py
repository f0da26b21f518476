"""Baking a clip into the Gaussians: re-fit the cut Gaussians so that a renderer without
clipping reproduces the RaRa-clipped images.

The paper leaves re-optimising Gaussians after clipping to future work (Discussion,
Limitations) and gives no method, so the objective is defined here. Given a scene,
a clip plane and a set of cameras, the target is the RaRa render of the whole scene
(Algorithm 1) from each camera. The baked scene drops the invisible Gaussians (Section 3.2:
they never contribute) and keeps the visible ones unchanged (their decay weight is 1, so they
render the same with or without the plane); the cutoff Gaussians, whose clipped appearance
depends on each ray's chord (Eq. 11), are free parameters (means, log-scales, quaternions,
opacity logits, SH). They start from the mass and mean of their visible part (the truncated
normal along the plane normal) and are fitted with Adam so that the unclipped render (mode
NONE) of the baked scene matches the targets in L2, with gradients from the render backward. The result
is a plain Gaussian scene that any unclipped splat renderer can draw.

The optimisation loop is independent of where gradients come from: loss_and_grad(params)
returns the summed loss over the cameras and the gradient of every parameter array of the
kept Gaussians. GpuBake provides it through the CUDA library; the tests also drive the loop
with the oracle's FP64 gradient.
"""
from __future__ import annotations

import dataclasses

import numpy as np

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")
INVISIBLE, VISIBLE, CUTOFF = 0, 1, 2


def split_by_label(labels: np.ndarray):
    """Indices of the Gaussians the baked scene keeps (visible or cutoff, in order) and, over
    those, which ones are free (cutoff)."""
    labels = np.asarray(labels)
    keep = np.nonzero(labels != INVISIBLE)[0]
    return keep, labels[keep] == CUTOFF


def subset(scene, idx):
    """The Gaussians idx of a scene (planar arrays, last axis = Gaussian)."""
    return dataclasses.replace(scene, **{k: np.ascontiguousarray(getattr(scene, k)[..., idx]) for k in PARAMS})


def truncated_moments(scene, plane, free):
    """Starting point of the fit: each free (cutoff) Gaussian replaced by the mass and mean of
    its part on the visible side of the plane. Along the plane normal n the Gaussian has
    standard deviation s_n = sqrt(n^T R S^2 R^T n) and its centre sits at d_ep = n.mu + d; with
    a = d_ep / s_n the visible share of its mass is Phi(a) and the visible part's mean lies
    s_n phi(a) / Phi(a) further along n (the standard truncated normal). Opacity is scaled by
    Phi(a) (kept within [1e-3, 0.99]); scales and rotation are kept. Returns a new Scene."""
    from math import erfc, exp, log, pi, sqrt
    n = np.asarray(plane.n, np.float64)
    means = np.asarray(scene.means, np.float64).copy()
    logits = np.asarray(scene.opacity_logits, np.float64).copy()
    sig = np.exp(np.asarray(scene.log_scales, np.float64))
    q = np.asarray(scene.quats, np.float64)
    for i in np.nonzero(np.asarray(free))[0]:
        w, x, y, z = q[:, i] / np.linalg.norm(q[:, i])
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        sn = float(np.linalg.norm(sig[:, i] * (R.T @ n)))
        a = (float(n @ means[:, i]) + float(plane.d)) / sn
        Phi = 0.5 * erfc(-a / sqrt(2.0))
        phi = exp(-0.5 * a * a) / sqrt(2.0 * pi)
        if Phi > 1e-12:
            means[:, i] += n * sn * phi / Phi
        op = 1.0 / (1.0 + exp(-logits[i]))
        op = min(0.99, max(1e-3, op * Phi))
        logits[i] = log(op / (1.0 - op))
    return dataclasses.replace(scene, means=means.astype(np.float32), opacity_logits=logits.astype(np.float32))


def fit(params: dict, free: np.ndarray, loss_and_grad, steps: int, lr: float = 2e-3, lr_means: float | None = None):
    """Adam on the free Gaussians' parameters (columns where free is True) of params
    (name -> torch tensor [..., n], updated in place). loss_and_grad(params) returns
    (loss, {name: gradient}). Returns the loss before every step and after the last."""
    import torch
    dev = params[PARAMS[0]].device
    mask = torch.as_tensor(np.asarray(free), device=dev)
    groups = []
    for k in PARAMS:
        p = torch.nn.Parameter(params[k])
        groups.append({"params": [p], "lr": lr_means if (k == "means" and lr_means) else lr})
    opt = torch.optim.Adam(groups)
    ps = [g["params"][0] for g in groups]
    losses = []
    for _ in range(steps):
        loss, grads = loss_and_grad(params)
        losses.append(float(loss))
        for p, k in zip(ps, PARAMS):
            p.grad = grads[k] * mask.to(grads[k].dtype)   # fixed Gaussians keep their values
        opt.step()
    losses.append(float(loss_and_grad(params)[0]))
    return losses


class GpuBake:
    """Bake on the GPU through the C ABI: labels from the preprocess, targets rendered with
    RaRa clipping, the kept Gaussians fitted against them with rara_render_backward.

    scene: a host Scene (numpy arrays); plane: the clip plane (RaRa mode); cameras: the
    cameras the targets are rendered from."""

    def __init__(self, scene, plane, cameras, bg=(0.0, 0.0, 0.0)):
        import torch

        from . import rara, scenes
        self.rara, self.torch = rara, torch
        self.scene, self.plane, self.bg = scene, plane, bg
        self.cameras = list(cameras)
        self.none = scenes.Plane(np.float32([0.0, 0.0, 1.0]), 0.0, 3.0, scenes.MODE_NONE)
        self.hard = scenes.Plane(plane.n, plane.d, plane.k_sigma, scenes.MODE_HARD)
        self.ctx = rara.rara_ctx_create(0)
        full = rara.GaussianTensors.from_scene(scene)
        self.labels = self._labels(full, plane)
        self.keep, self.free = split_by_label(self.labels)
        self.kept = subset(scene, self.keep)
        self.hard_kept = subset(scene, np.nonzero(self._labels(full, self.hard) != INVISIBLE)[0])
        self.targets = self.render(full, plane, self.cameras)
        self.start = truncated_moments(self.kept, plane, self.free)
        self.params = {k: getattr(rara.GaussianTensors.from_scene(self.start), k) for k in PARAMS}
        self.sh_degree = int(scene.sh_degree)
        self._views = None

    def _labels(self, gs, plane):
        # labels depend on the plane only: one preprocess from any camera
        rara, torch = self.rara, self.torch
        rara.rara_preprocess(self.ctx, gs, self.cameras[0], plane)
        lab = torch.zeros(gs.n, dtype=torch.uint8, device="cuda")
        rara.rara_frame_gaussians(self.ctx, 0, labels=lab)
        return lab.cpu().numpy()

    def render(self, gs, plane, cameras):
        rara, torch = self.rara, self.torch
        views = [rara.View(0, c, plane, torch.empty((3, c.height, c.width), device="cuda"), None, None, self.bg)
                 for c in cameras]
        rara.rara_render_batch(self.ctx, [gs], views)
        torch.cuda.synchronize()
        return [v.image for v in views]

    def gaussians(self):
        return self.rara.GaussianTensors(*(self.params[k] for k in PARAMS), self.sh_degree)

    def loss_and_grad(self, params):
        """L = sum over the cameras of |unclipped render - RaRa target|^2 and its gradient."""
        rara, torch = self.rara, self.torch
        gs = self.gaussians()
        if self._views is None:
            self._views = [rara.View(0, c, self.none, torch.empty((3, c.height, c.width), device="cuda"),
                                     torch.empty((c.height, c.width), device="cuda"),
                                     torch.empty((c.height, c.width), dtype=torch.int32, device="cuda"), self.bg)
                           for c in self.cameras]
            self._dimg = [torch.empty_like(v.image) for v in self._views]
            self._loss = torch.empty(len(self._views), dtype=torch.float64, device="cuda")
            self._grads = gs.empty_like()
        rara.rara_render_batch(self.ctx, [gs], self._views)
        rara.rara_loss_l2(self.ctx, self.targets, self._dimg, [1.0] * len(self._views), self._loss)
        rara.rara_render_backward(self.ctx, self._dimg, [self._grads], None)
        return float(self._loss.sum()), {k: getattr(self._grads, k) for k in PARAMS}

    def errors(self, cameras=None):
        """Mean squared error against the RaRa render of the original scene, on the fitting
        cameras (default) or others, of: the baked scene drawn without clipping, the kept
        Gaussians before fitting, and hard clipping (centres behind the plane dropped, the
        rest unchanged) drawn without clipping; also of the fit's starting point (truncated
        moments) and of the kept Gaussians unchanged."""
        rara = self.rara
        cams = self.cameras if cameras is None else list(cameras)
        targets = self.targets if cameras is None else \
            self.render(rara.GaussianTensors.from_scene(self.scene), self.plane, cams)

        def mse(imgs):
            return float(sum(((a - b) ** 2).sum() for a, b in zip(imgs, targets)) /
                         sum(t.numel() for t in targets))
        return {"baked": mse(self.render(self.gaussians(), self.none, cams)),
                "start": mse(self.render(rara.GaussianTensors.from_scene(self.start), self.none, cams)),
                "kept_unclipped": mse(self.render(rara.GaussianTensors.from_scene(self.kept), self.none, cams)),
                "hard_clip": mse(self.render(rara.GaussianTensors.from_scene(self.hard_kept), self.none, cams))}

    def baked_scene(self):
        """The baked Gaussians as a host Scene."""
        return dataclasses.replace(self.kept, **{k: self.params[k].detach().cpu().numpy().astype(np.float32)
                                                 for k in PARAMS})

    def close(self):
        self.rara.rara_ctx_destroy(self.ctx)


def bake_on_gpu(scene, plane, cameras, steps: int = 100, lr: float = 2e-3, lr_means: float = 2e-4,
                held_out=()):
    """Bake `plane` into `scene` from `cameras`; returns (baked Scene, report)."""
    b = GpuBake(scene, plane, cameras)
    try:
        before = b.errors()
        losses = fit(b.params, b.free, b.loss_and_grad, steps, lr, lr_means)
        report = {"kept": int(b.keep.size), "free": int(b.free.sum()), "dropped": int(scene.n - b.keep.size),
                  "losses": losses, "mse_before": before, "mse_after": b.errors()}
        if held_out:
            report["held_out"] = b.errors(held_out)
        return b.baked_scene(), report
    finally:
        b.close()
