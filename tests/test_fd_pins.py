"""Pins of the finite-difference gradients of the oracle (the reference the GPU backward is
checked against), on cases with closed-form derivatives."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_20202_gb300 import scenes
from tests import fd

Y00 = 0.5 / math.sqrt(math.pi)


def _one_gaussian(sigma=0.1, logit=0.3, rgb=(0.8, 0.4, 0.2)):
    g = scenes.Scene(np.zeros((3, 1), np.float32), np.full((3, 1), np.log(sigma), np.float32),
                     np.array([[1.0], [0.0], [0.0], [0.0]], np.float32), np.array([logit], np.float32),
                     ((np.array(rgb, np.float32) - 0.5) / np.float32(Y00)).reshape(3, 1).astype(np.float32), 0)
    # 33 x 33 with the principal point at 16.5: pixel (16, 16) looks straight at the origin
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 33, 33, 60.0)
    return g, cam


def _centre_weight(channel=0):
    w = np.zeros((3, 33, 33))
    w[channel, 16, 16] = 1.0
    return w


def test_opacity_and_colour_gradients_at_the_centre():
    """C = rgb * sigmoid(logit) at the centre pixel (q = 0, black background):
    dC/dlogit = rgb op (1 - op), dC/dsh0 = Y00 op, dC/dmean = 0 (q is minimal there)."""
    g, cam = _one_gaussian()
    pl = scenes.Plane(np.float32([0, 0, 1]), 0.0, 3.0, scenes.MODE_NONE)
    op = 1.0 / (1.0 + math.exp(-float(np.float32(0.3))))
    rgb0 = float(g.sh[0, 0]) * Y00 + 0.5
    got = fd.fd_gradients(g, [(cam, pl, (0, 0, 0))], [_centre_weight(0)], planes=False,
                          params=("opacity_logits", "sh", "means"))
    assert got["opacity_logits"][0] == pytest.approx(rgb0 * op * (1 - op), rel=1e-6)
    assert got["sh"][0, 0] == pytest.approx(Y00 * op, rel=1e-6)
    assert np.all(got["sh"][1:, 0] == 0.0)                       # other channels: no effect on C_r
    assert np.max(np.abs(got["means"])) < 1e-6


def test_plane_gradients_of_a_split_chord():
    """Central ray through a sphere of radius R = 3 sigma, plane z = s (n = (0,0,1), d = -s):
    w = (R - s) / (2R), so dC/dd = rgb op / (2R), dC/dn_z = rgb op s / (2R), and tilting the
    plane about the ray (n_x, n_y) leaves the hit point and w unchanged."""
    sigma = 0.1
    R = 3.0 * sigma
    s = 0.09
    g, cam = _one_gaussian(sigma)
    pl = scenes.Plane(np.float32([0, 0, 1]), float(np.float32(-s)), 3.0, scenes.MODE_RARA)
    s = -float(np.float32(-s))
    op = 1.0 / (1.0 + math.exp(-float(np.float32(0.3))))
    rgb0 = float(g.sh[0, 0]) * Y00 + 0.5
    pre = oracle.preprocess(g, cam, pl)
    assert pre["label"][0] == oracle.CUTOFF
    got = fd.fd_gradients(g, [(cam, pl, (0, 0, 0))], [_centre_weight(0)], params=(), planes=True)
    pg = got["planes"][0]
    R32 = 3.0 * float(np.exp(np.float32(np.log(sigma))))
    assert pg[3] == pytest.approx(rgb0 * op / (2 * R32), rel=1e-6)
    assert pg[2] == pytest.approx(rgb0 * op * s / (2 * R32), rel=1e-6)
    assert abs(pg[0]) < 1e-7 and abs(pg[1]) < 1e-7


def test_masked_loss_is_smooth():
    """With the discontinuity mask applied, steps h and h/2 agree (no jump inside +-h)."""
    sc = scenes.gradient_scene(10, seed=3, sh_degree=0)
    cam = scenes.look_at_camera((0.3, -0.2, -3.0), (0.0, 0.0, 0.0), 48, 40, 60.0)
    pl = scenes.Plane(np.float32(scenes.random_unit_normal(5)), 0.05, 3.0, scenes.MODE_RARA)
    rng = np.random.default_rng(0)
    w = rng.standard_normal((3, 40, 48)) * fd.smooth_mask(sc, cam, pl, (0.1, 0.2, 0.3))
    views = [(cam, pl, (0.1, 0.2, 0.3))]
    a = fd.fd_gradients(sc, views, [w], h=1e-6)
    b = fd.fd_gradients(sc, views, [w], h=5e-7)
    for k in a:
        assert fd.rel_l2(b[k], a[k]) < 1e-5, k
    # the scene exercises the clipped weight: some Gaussians are cutoff and the plane matters
    pre = oracle.preprocess(sc, cam, pl)
    assert np.sum(pre["label"] == oracle.CUTOFF) >= 3
    assert np.linalg.norm(a["planes"]) > 1e-3
