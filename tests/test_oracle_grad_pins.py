"""Pins of the oracle's analytic FP64 gradient (oracle/grad.py).

Its forward is an independent float64 restatement (PyTorch CPU) and must reproduce the C
oracle's images; its gradient must match central differences of the C oracle's render and
closed forms on single Gaussians. None of these calls the CUDA library.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import grad as ograd
from paper_2506_20202_gb300 import scenes
from tests import fd

Y00 = 0.5 / math.sqrt(math.pi)


def _forward_cases():
    sc, cam, pl = scenes.small_uniform_workload(n=1500, width=72, height=56, seed=3)
    yield "uniform SH0", sc, cam, pl
    g = scenes.general_scene(3000, seed=4, sh_degree=3)
    cam2 = scenes.look_at_camera((0.3, -0.5, -2.6), (0.0, 0.0, 0.0), 80, 48, 60.0)
    pl2 = scenes.Plane(np.float32(scenes.random_unit_normal(2)), 0.1, 3.0, scenes.MODE_RARA)
    yield "general SH3", g, cam2, pl2
    yield "ablation mode", g, cam2, scenes.Plane(pl2.n, pl2.d, 3.0, scenes.MODE_RARA_ALL)
    yield "k_sigma 1", g, cam2, scenes.Plane(pl2.n, pl2.d, 1.0, scenes.MODE_RARA)
    yield "hard", g, cam2, scenes.Plane(pl2.n, pl2.d, 3.0, scenes.MODE_HARD)
    gs = scenes.gradient_scene(200, seed=6, sh_degree=2)
    cam3 = scenes.look_at_camera((0.2, 0.3, -2.8), (0.0, 0.0, 0.0), 64, 64, 60.0)
    yield "gradient scene SH2", gs, cam3, scenes.Plane(np.float32(scenes.random_unit_normal(7)), 0.02, 3.0,
                                                       scenes.MODE_RARA)


@pytest.mark.parametrize("case", list(range(6)))
def test_forward_equals_the_c_oracle(orc, case):
    name, sc, cam, pl = list(_forward_cases())[case]
    bg = (0.1, 0.2, 0.3)
    pre, kvr, ref = orc.render_frame(sc, cam, pl, bg, threads=2)
    got = ograd.render_and_grad(sc, cam, pl, bg, grad=False)
    ok = ref["events"] == 0
    assert ok.mean() > 0.9
    assert np.abs(got["image"] - ref["image"])[:, ok].max() <= 1e-10, name
    assert np.abs(got["T"] - ref["T"])[ok].max() <= 1e-10, name
    if pl.mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL):
        assert (pre["label"] == orc.CUTOFF).sum() > 10, name      # the weight is exercised


def _views(sc_seed=5, sh=1):
    sc = scenes.gradient_scene(24, seed=sc_seed, sh_degree=sh)
    views = [(scenes.look_at_camera((0.4, -0.3, -2.9), (0.0, 0.0, 0.0), 48, 40, 60.0),
              scenes.Plane(np.float32(scenes.random_unit_normal(9)), 0.05, 3.0, scenes.MODE_RARA), (0, 0, 0)),
             (scenes.look_at_camera((-1.2, 0.8, -2.5), (0.0, 0.0, 0.0), 40, 48, 60.0),
              scenes.Plane(np.float32(scenes.random_unit_normal(4)), -0.03, 3.0, scenes.MODE_RARA), (0.2, 0.1, 0.0))]
    return sc, views


@pytest.mark.parametrize("sh", [0, 1, 3])
def test_gradient_matches_central_differences(orc, sh):
    sc, views = _views(5, sh)
    rng = np.random.default_rng(sh)
    weights = [rng.standard_normal((3, cam.height, cam.width)) * fd.smooth_mask(sc, cam, pl, bg)
               for cam, pl, bg in views]
    ref = fd.fd_gradients(sc, views, weights)
    tot = {k: 0.0 for k in ograd.PARAMS}
    planes = []
    for (cam, pl, bg), w in zip(views, weights):
        g = ograd.render_and_grad(sc, cam, fd.ExactPlane.of(pl), bg, w)
        for k in ograd.PARAMS:
            tot[k] = tot[k] + g[k]
        planes.append(g["plane"])
    for k in ograd.PARAMS:
        assert fd.rel_l2(tot[k], ref[k]) <= 1e-6, (k, fd.rel_l2(tot[k], ref[k]))
    assert fd.rel_l2(np.array(planes), ref["planes"]) <= 1e-6
    assert np.linalg.norm(ref["planes"]) > 0 and np.linalg.norm(ref["means"]) > 0


def _one_gaussian(sigma=0.1, logit=0.3, rgb=(0.8, 0.4, 0.2)):
    g = scenes.Scene(np.zeros((3, 1), np.float32), np.full((3, 1), np.log(sigma), np.float32),
                     np.array([[1.0], [0.0], [0.0], [0.0]], np.float32), np.array([logit], np.float32),
                     ((np.array(rgb, np.float32) - 0.5) / np.float32(Y00)).reshape(3, 1).astype(np.float32), 0)
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 33, 33, 60.0)
    return g, cam


def test_closed_forms_at_the_centre_pixel(orc):
    """C = rgb sigmoid(logit) at the centre pixel (q = 0): dC/dlogit = rgb op (1 - op),
    dC/dsh0 = Y00 op, dC/dmean = 0; and for the central ray through a sphere of radius
    R = 3 sigma split by the plane z = s: w = (R - s)/(2R), dC/dd = rgb op / (2R),
    dC/dn_z = rgb op s / (2R), dC/dn_x = dC/dn_y = 0."""
    g, cam = _one_gaussian()
    w = np.zeros((3, 33, 33))
    w[0, 16, 16] = 1.0
    op = 1.0 / (1.0 + math.exp(-float(np.float32(0.3))))
    rgb0 = float(g.sh[0, 0]) * Y00 + 0.5
    got = ograd.render_and_grad(g, cam, scenes.Plane(np.float32([0, 0, 1]), 0.0, 3.0, scenes.MODE_NONE), (0, 0, 0), w)
    assert got["opacity_logits"][0] == pytest.approx(rgb0 * op * (1 - op), rel=1e-12)
    assert got["sh"][0, 0] == pytest.approx(Y00 * op, rel=1e-12)
    assert np.all(got["sh"][1:, 0] == 0.0)
    assert np.abs(got["means"]).max() < 1e-12
    s = -float(np.float32(-0.09))
    R = 3.0 * math.exp(float(np.float32(math.log(0.1))))
    pl = scenes.Plane(np.float32([0, 0, 1]), float(np.float32(-0.09)), 3.0, scenes.MODE_RARA)
    got = ograd.render_and_grad(g, cam, pl, (0, 0, 0), w)
    assert got["plane"][3] == pytest.approx(rgb0 * op / (2 * R), rel=1e-9)
    assert got["plane"][2] == pytest.approx(rgb0 * op * s / (2 * R), rel=1e-9)
    assert abs(got["plane"][0]) < 1e-12 and abs(got["plane"][1]) < 1e-12
    assert got["image"][0, 16, 16] == pytest.approx(rgb0 * op * (R - s) / (2 * R), rel=1e-12)


def test_sh_basis_matches_the_c_oracle(orc):
    rng = np.random.default_rng(0)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    b = ograd.sh_basis(torch.as_tensor(d), 3).numpy()
    for i in range(40):
        for l in range(4):
            for m in range(-l, l + 1):
                assert b[i, l * l + l + m] == pytest.approx(orc.real_sh(l, m, d[i]), abs=1e-13)
