"""Baking a clip into the Gaussians (an extension: the paper leaves re-fitting after clipping
to future work). The fitting loop, driven by the oracle's FP64 gradient on a small scene:
only the cutoff Gaussians move, the unclipped render of the baked scene approaches the RaRa
render of the original, and it ends closer than hard clipping."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import grad as ograd
from paper_2506_20202_gb300 import bake, scenes


def _setup():
    # 120 Gaussians about 0.05 wide in [-0.6, 0.6]^3 and a plane through the centre: about a
    # fifth invisible, a quarter visible, the rest cutoff
    sc = scenes.gradient_scene(120, seed=21, sh_degree=1)
    sc = dataclasses.replace(sc, log_scales=(sc.log_scales - 0.8).astype(np.float32))
    pl = scenes.Plane(np.float32(scenes.random_unit_normal(3)), 0.0, 3.0, scenes.MODE_RARA)
    cams = [scenes.look_at_camera((2.8 * np.sin(a), -0.5, -2.8 * np.cos(a)), (0.0, 0.0, 0.0), 64, 48, 60.0)
            for a in (0.0, 0.9, -0.8)]
    return sc, pl, cams


def test_split_and_subset():
    keep, free = bake.split_by_label(np.array([0, 1, 2, 2, 0, 1], np.uint8))
    assert keep.tolist() == [1, 2, 3, 5] and free.tolist() == [False, True, True, False]
    sc = scenes.gradient_scene(6, seed=1, sh_degree=2)
    sub = bake.subset(sc, keep)
    assert sub.n == 4 and np.array_equal(sub.sh, sc.sh[:, keep]) and np.array_equal(sub.means, sc.means[:, keep])


def test_fit_with_the_oracle_gradient(orc):
    sc, pl, cams = _setup()
    labels = orc.preprocess(sc, cams[0], pl)["label"]
    keep, free = bake.split_by_label(labels)
    assert free.sum() >= 10 and (~free).sum() >= 10 and keep.size < sc.n
    targets = [orc.render_frame(sc, c, pl, threads=2)[2]["image"] for c in cams]
    kept = bake.subset(sc, keep)
    none = scenes.Plane(np.float32([0, 0, 1]), 0.0, 3.0, scenes.MODE_NONE)
    start_scene = bake.truncated_moments(kept, pl, free)
    params = {k: torch.tensor(np.asarray(getattr(start_scene, k), np.float64)) for k in bake.PARAMS}
    start = {k: v.clone() for k, v in params.items()}

    def scene_of(p):
        return dataclasses.replace(kept, **{k: p[k].numpy().copy() for k in bake.PARAMS})

    def loss_and_grad(p):
        s = scene_of(p)
        loss, grads = 0.0, {k: torch.zeros_like(v) for k, v in p.items()}
        for c, t in zip(cams, targets):
            img = ograd.render_and_grad(s, c, none, (0, 0, 0), grad=False)["image"]
            g = ograd.render_and_grad(s, c, none, (0, 0, 0), weights=2.0 * (img - t))
            loss += float(((img - t) ** 2).sum())
            for k in bake.PARAMS:
                grads[k] += torch.from_numpy(g[k])
        return loss, grads

    losses = bake.fit(params, free, loss_and_grad, steps=25, lr=2e-2, lr_means=2e-3)
    assert losses[-1] < 0.8 * losses[0], losses
    for k in bake.PARAMS:                      # the visible Gaussians did not move
        assert torch.equal(params[k][..., ~free], torch.tensor(np.asarray(getattr(kept, k), np.float64))[..., ~free])
        assert not torch.equal(params[k][..., free], start[k][..., free]) or k == "quats"
    # hard clipping (centres behind the plane dropped) drawn unclipped, against the same targets
    hard = scenes.Plane(pl.n, pl.d, 3.0, scenes.MODE_HARD)
    hkeep = np.nonzero(orc.preprocess(sc, cams[0], hard)["label"] != orc.INVISIBLE)[0]
    hs = bake.subset(sc, hkeep)
    hard_loss = sum(float(((orc.render_frame(hs, c, none, threads=2)[2]["image"] - t) ** 2).sum())
                    for c, t in zip(cams, targets))
    assert losses[-1] < hard_loss, (losses[-1], hard_loss)


def test_truncated_moments_of_one_gaussian():
    """An isotropic Gaussian of sigma s at d_ep = a s: opacity times Phi(a), centre moved by
    s phi(a) / Phi(a) along n; a Gaussian far on the visible side is unchanged."""
    from math import erfc, exp, pi, sqrt
    s, a = 0.1, 0.7
    sc = scenes.Scene(np.zeros((3, 2), np.float32), np.full((3, 2), np.log(s), np.float32),
                      np.array([[1, 1], [0, 0], [0, 0], [0, 0]], np.float32), np.zeros(2, np.float32),
                      np.zeros((3, 2), np.float32), 0)
    sc.means[2, 1] = 10.0
    pl = scenes.Plane(np.float32([0, 0, 1]), float(np.float32(a * s)), 3.0, scenes.MODE_RARA)   # d_ep = a s
    out = bake.truncated_moments(sc, pl, np.array([True, True]))
    d = float(np.float32(a * s)) / s             # the a of the float32 plane offset
    Phi, phi = 0.5 * erfc(-d / sqrt(2)), exp(-0.5 * d * d) / sqrt(2 * pi)
    assert out.means[2, 0] == pytest.approx(s * phi / Phi, rel=1e-5)
    assert 1 / (1 + np.exp(-out.opacity_logits[0])) == pytest.approx(0.5 * Phi, rel=1e-5)
    assert out.means[2, 1] == pytest.approx(10.0) and out.opacity_logits[1] == pytest.approx(0.0, abs=1e-6)
