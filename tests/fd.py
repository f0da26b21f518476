"""Finite-difference gradients of the FP64 oracle render (test infrastructure).

The loss is linear in the images, L = sum_v sum(weights_v * image_v), so dL/dimage_v is
weights_v. Central differences with step h on float64 copies of the parameters, which the
oracle takes unrounded (float32 inputs widen exactly, so the unperturbed point is the same
one the GPU renders). Pixels whose oracle pixel sequence passes near a discontinuity of
the render (the q = 9 support edge, alpha = 1/255, T = 1e-4, a grazing ray on the clipped
side, a depth near-tie, a Gaussian near a class threshold) get weight 0, so the loss is
smooth within the steps taken.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")
# event tolerances for the mask: q, alpha, T (relative), 1 - b^2, Gaussian threshold margin
# (world units), position (pixels), depth ulps
MASK_TOL = (2e-3, 2e-3, 2e-3, 2e-3, 1e-3, 2e-3, 256)
CLASS_MARGIN = 1e-3


@dataclasses.dataclass
class ExactPlane:
    """A clip plane the oracle uses unrounded (float64 n and d)."""
    n: np.ndarray
    d: float
    k_sigma: float = 3.0
    mode: int = 2
    exact: bool = True

    @staticmethod
    def of(plane) -> "ExactPlane":
        return ExactPlane(np.asarray(plane.n, np.float32).astype(np.float64), float(np.float32(plane.d)),
                          float(plane.k_sigma), int(plane.mode))


def scene64(scene):
    return dataclasses.replace(scene, **{k: np.asarray(getattr(scene, k), np.float32).astype(np.float64)
                                         for k in PARAMS})


def render(scene, cam, plane, bg, tol=oracle.DEFAULT_TOL):
    pre = oracle.preprocess(scene, cam, plane)
    kvr = oracle.build_keys(pre)
    return pre, oracle.render(scene, pre, cam, plane, bg, kvr, tol=tol, threads=1)


def loss(scene, views, weights) -> float:
    total = 0.0
    for (cam, plane, bg), w in zip(views, weights):
        total += float(np.sum(w * render(scene, cam, plane, bg)[1]["image"]))
    return total


def smooth_mask(scene, cam, plane, bg) -> np.ndarray:
    """True where the pixel is away from every discontinuity (safe for finite differences)."""
    pre, out = render(scene, cam, plane, bg, tol=MASK_TOL)
    bad = out["events"] != 0
    near = np.nonzero((pre["margin_class"] < CLASS_MARGIN) & (pre["culled"] == 0))[0]
    if near.size:
        bad |= oracle.support_mask(pre, near, cam.height, cam.width)
    return ~bad


def fd_gradients(scene, views, weights, h: float = 1e-6, params=PARAMS, planes: bool = True) -> dict:
    """Central-difference dL/dparam for every Gaussian parameter (arrays shaped like the
    scene's) and, with planes=True, dL/d(n.x, n.y, n.z, d) per view ([V, 4])."""
    base = scene64(scene)
    views = [(cam, ExactPlane.of(pl), bg) for cam, pl, bg in views]
    out = {}
    for name in params:
        arr = getattr(base, name)
        g = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            x0 = arr[idx]
            arr[idx] = x0 + h
            lp = loss(base, views, weights)
            arr[idx] = x0 - h
            lm = loss(base, views, weights)
            arr[idx] = x0
            g[idx] = (lp - lm) / (2 * h)
        out[name] = g
    if planes:
        pg = np.zeros((len(views), 4))
        for v, (cam, pl, bg) in enumerate(views):
            for j in range(4):
                vals = []
                for s in (+h, -h):
                    n = pl.n.copy()
                    d = pl.d
                    if j < 3:
                        n[j] += s
                    else:
                        d += s
                    p2 = ExactPlane(n, d, pl.k_sigma, pl.mode)
                    vals.append(float(np.sum(weights[v] * render(base, cam, p2, bg)[1]["image"])))
                pg[v, j] = (vals[0] - vals[1]) / (2 * h)
        out["planes"] = pg
    return out


def directional_fd(scene, views, weights, direction: dict, h: float = 1e-6) -> float:
    """Central difference of L along `direction` (arrays shaped like the scene's)."""
    base = scene64(scene)
    views = [(cam, ExactPlane.of(pl), bg) for cam, pl, bg in views]
    vals = []
    for s in (+h, -h):
        moved = dataclasses.replace(base, **{k: getattr(base, k) + s * direction[k] for k in direction})
        vals.append(loss(moved, views, weights))
    return (vals[0] - vals[1]) / (2 * h)


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
