"""Hand-built tiny scenes for the oracle pins (inputs only)."""
import math

import numpy as np

from paper_2506_20202_gb300 import scenes

Y00 = 0.5 / math.sqrt(math.pi)


def axis_camera(width=64, height=64, f=None):
    """Camera at the origin looking down +z (identity rotation), square pixels."""
    w2c = np.zeros((3, 4), np.float32)
    w2c[:, :3] = np.eye(3)
    f = float(f if f is not None else width)
    return scenes.Camera(w2c, f, f, width / 2, height / 2, width, height)


def make_scene(means, sigmas, quats=None, opacity=None, rgb=None, sh=None, sh_degree=0):
    """Scene from per-Gaussian lists; sigmas are per-axis standard deviations."""
    means = np.asarray(means, np.float64).reshape(-1, 3).T
    n = means.shape[1]
    sig = np.asarray(sigmas, np.float64).reshape(n, 3).T
    if quats is None:
        quats = np.tile(np.array([[1.0], [0.0], [0.0], [0.0]]), (1, n))
    else:
        quats = np.asarray(quats, np.float64).reshape(n, 4).T
    if opacity is None:
        opacity = np.full(n, 0.5)
    opacity = np.asarray(opacity, np.float64)
    logits = np.log(opacity / (1.0 - opacity))
    if sh is None:
        rgb = np.full((n, 3), 0.5) if rgb is None else np.asarray(rgb, np.float64).reshape(n, 3)
        sh = ((rgb.T - 0.5) / Y00)
        sh_degree = 0
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    return scenes.Scene(f(means), f(np.log(sig)), f(quats), f(logits), f(sh), sh_degree)


def plane(n, d, mode=scenes.MODE_RARA, k=3.0):
    n = np.asarray(n, np.float64)
    return scenes.Plane(np.asarray(n, np.float32), float(d), float(k), mode)
