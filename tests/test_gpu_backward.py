"""Backward of the clipped render (rara_render_backward) against central differences of the
FP64 oracle, plus its consistency across batching, graph replay and the autograd wrapper.

Gradients are compared per parameter group by relative L2 error (<= 1e-3) on tiny scenes
whose loss weights are zero at pixels near a discontinuity of the render (tests/fd.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2506_20202_gb300 import rara, scenes
from tests import fd

pytestmark = pytest.mark.gpu

REL_L2 = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()
    oracle.build()


def _views(seed, mode, sizes=((64, 48), (56, 64))):
    rng = np.random.default_rng(seed)
    out = []
    for k, (w, h) in enumerate(sizes):
        eye = rng.normal(0, 1, 3)
        eye = 3.0 * eye / np.linalg.norm(eye)
        cam = scenes.look_at_camera(eye, (0.0, 0.0, 0.0), w, h, 60.0)
        pl = scenes.Plane(np.float32(scenes.random_unit_normal(seed * 10 + k)), float(rng.uniform(-0.15, 0.15)),
                          3.0, mode)
        out.append((cam, pl, tuple(float(x) for x in rng.uniform(0.0, 0.4, 3))))
    return out


def _weights(sc, views, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((3, cam.height, cam.width)) * fd.smooth_mask(sc, cam, pl, bg)
            for cam, pl, bg in views]


def gpu_gradients(sc, views, weights, graph=False, renderer=None):
    """Forward (batch) + rara_render_backward; returns numpy gradients like fd_gradients."""
    r = renderer or rara.Renderer()
    g = rara.GaussianTensors.from_scene(sc)
    vs = []
    for cam, pl, bg in views:
        H, W = cam.height, cam.width
        vs.append(rara.View(0, cam, pl, torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
                            torch.empty((H, W), dtype=torch.int32, device="cuda"), bg))
    (rara.rara_render_batch_graph if graph else rara.rara_render_batch)(r.ctx, [g], vs)
    grads = g.empty_like()
    pg = torch.empty((len(views), 4), device="cuda")
    dimg = [torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda() for w in weights]
    rara.rara_render_backward(r.ctx, dimg, [grads], pg)
    torch.cuda.synchronize()
    out = {k: getattr(grads, k).cpu().numpy().astype(np.float64) for k in fd.PARAMS}
    out["planes"] = pg.cpu().numpy().astype(np.float64)
    out["images"] = [v.image.cpu().numpy() for v in vs]
    if renderer is None:
        r.close()
    return out


@pytest.mark.parametrize("deg,mode,seed", [(1, scenes.MODE_RARA, 0), (3, scenes.MODE_RARA, 1),
                                           (0, scenes.MODE_RARA_ALL, 2), (2, scenes.MODE_HARD, 3),
                                           (1, scenes.MODE_NONE, 4)])
def test_gradients_match_finite_differences(deg, mode, seed):
    sc = scenes.gradient_scene(24, seed=seed, sh_degree=deg)
    views = _views(seed, mode)
    weights = _weights(sc, views, seed + 100)
    ref = fd.fd_gradients(sc, views, weights)
    got = gpu_gradients(sc, views, weights)
    for k in fd.PARAMS:
        assert np.linalg.norm(ref[k]) > 0, k
        assert fd.rel_l2(got[k], ref[k]) <= REL_L2, (k, fd.rel_l2(got[k], ref[k]))
    if mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL):
        assert np.linalg.norm(ref["planes"]) > 1e-3
        assert fd.rel_l2(got["planes"], ref["planes"]) <= REL_L2, fd.rel_l2(got["planes"], ref["planes"])
    else:   # hard clipping and no clipping: the image does not vary smoothly with the plane
        assert np.all(got["planes"] == 0.0)


def test_gradients_with_cutoff_dominated_scene():
    """Most Gaussians straddle the plane; their chord-split weights carry the gradient."""
    sc = scenes.gradient_scene(32, seed=7, sh_degree=1)
    sc.log_scales = np.ascontiguousarray(sc.log_scales + np.float32(0.3))
    views = _views(7, scenes.MODE_RARA, sizes=((64, 64),))
    pre = oracle.preprocess(sc, views[0][0], views[0][1])
    assert np.mean(pre["label"] == oracle.CUTOFF) > 0.5
    weights = _weights(sc, views, 8)
    ref = fd.fd_gradients(sc, views, weights)
    got = gpu_gradients(sc, views, weights)
    for k in list(fd.PARAMS) + ["planes"]:
        assert fd.rel_l2(got[k], ref[k]) <= REL_L2, (k, fd.rel_l2(got[k], ref[k]))


def test_directional_derivative_on_a_larger_batch():
    """4000 Gaussians, three views: the gradient's projection on a random direction equals
    the oracle's central difference along it."""
    sc = scenes.general_scene(4000, seed=11, sh_degree=2)
    views = _views(11, scenes.MODE_RARA, sizes=((160, 120), (128, 128), (96, 144)))
    weights = _weights(sc, views, 12)
    got = gpu_gradients(sc, views, weights)
    rng = np.random.default_rng(13)
    scale = {"means": 1e-2, "log_scales": 1e-1, "quats": 1e-1, "opacity_logits": 1.0, "sh": 1.0}
    for trial in range(3):
        direction = {k: scale[k] * rng.standard_normal(getattr(sc, k).shape) for k in fd.PARAMS}
        ref = fd.directional_fd(sc, views, weights, direction)
        dot = sum(float(np.sum(got[k] * direction[k])) for k in fd.PARAMS)
        assert abs(dot - ref) <= 1e-3 * max(abs(ref), 1e-6) + 1e-6, (trial, dot, ref)


def test_batch_gradient_is_the_sum_of_single_view_gradients():
    sc = scenes.gradient_scene(200, seed=21, sh_degree=1)
    sc.means = np.ascontiguousarray(sc.means * np.float32(1.5))
    views = _views(21, scenes.MODE_RARA, sizes=((96, 64), (64, 80), (80, 80)))
    weights = _weights(sc, views, 22)
    whole = gpu_gradients(sc, views, weights)
    parts = [gpu_gradients(sc, [v], [w]) for v, w in zip(views, weights)]
    for k in fd.PARAMS:
        s = sum(p[k] for p in parts)
        assert fd.rel_l2(whole[k], s) <= 1e-5, k
    for v, p in enumerate(parts):
        assert np.allclose(whole["planes"][v], p["planes"][0], rtol=1e-5, atol=1e-7)


def test_batch_gradient_over_more_views_than_a_chunk():
    """35 views, more than the preprocess backward's chunk of 32 views (each lane takes the
    chunk's views that render its Gaussian in rounds): the batch's parameter and plane
    gradients equal the sums of the single-view backwards."""
    sc = scenes.gradient_scene(300, seed=71, sh_degree=2)
    sc.means = np.ascontiguousarray(sc.means * np.float32(1.4))
    views = _views(71, scenes.MODE_RARA, sizes=tuple((32 + 4 * (k % 3), 28 + 4 * (k % 4)) for k in range(35)))
    weights = _weights(sc, views, 72)
    whole = gpu_gradients(sc, views, weights)
    r = rara.Renderer()
    parts = [gpu_gradients(sc, [v], [w], renderer=r) for v, w in zip(views, weights)]
    r.close()
    for k in fd.PARAMS:
        s_ = sum(p[k] for p in parts)
        assert np.linalg.norm(s_) > 0, k
        assert fd.rel_l2(whole[k], s_) <= 1e-5, (k, fd.rel_l2(whole[k], s_))
    for v, p in enumerate(parts):   # float sums in another order: relative to the vector's norm
        d = np.linalg.norm(whole["planes"][v] - p["planes"][0])
        assert d <= 1e-5 * np.linalg.norm(p["planes"][0]) + 1e-7, (v, d)


def test_backward_after_graph_capture_and_replay():
    """The first graph call captures (and replays once); a backward after it, and after a
    later replay with new cameras, equals the backward of the exact batch render."""
    sc = scenes.gradient_scene(300, seed=31, sh_degree=2)
    r = rara.Renderer()
    for seed in (31, 32):
        views = _views(seed, scenes.MODE_RARA, sizes=((64, 64), (80, 48)))
        weights = _weights(sc, views, seed)
        got = gpu_gradients(sc, views, weights, graph=True, renderer=r)
        ref = gpu_gradients(sc, views, weights)
        for k in list(fd.PARAMS) + ["planes"]:
            assert fd.rel_l2(got[k], ref[k]) <= 1e-5, (seed, k)
        for a, b in zip(got["images"], ref["images"]):
            assert np.array_equal(a, b)
    r.close()


def test_repeated_backwards_on_one_context_start_from_zero_records():
    """The per-slot gradient records are zeroed by the backward that read them, not by a
    clear of the whole buffer: backwards of different batches (view counts, sizes, a
    one-camera sweep) in turn on one context, each twice, equal those of fresh contexts."""
    sc = scenes.gradient_scene(300, seed=41, sh_degree=1)
    sweep_cam = _views(44, scenes.MODE_RARA, sizes=((72, 56),))[0][0]
    batches = [_views(41, scenes.MODE_RARA, sizes=((64, 64), (80, 48), (48, 72))),
               _views(42, scenes.MODE_RARA_ALL, sizes=((96, 80),)),
               [(sweep_cam, scenes.Plane(np.float32(scenes.random_unit_normal(45)), float(o), 3.0, scenes.MODE_RARA),
                 (0.1, 0.2, 0.3)) for o in (-0.1, 0.0, 0.1)],
               _views(43, scenes.MODE_RARA, sizes=((64, 64), (80, 48), (48, 72), (56, 56)))]
    r = rara.Renderer()
    for k, views in enumerate(batches):
        weights = _weights(sc, views, 50 + k)
        ref = gpu_gradients(sc, views, weights)
        for rep in range(2):
            got = gpu_gradients(sc, views, weights, renderer=r)
            for name in list(fd.PARAMS) + ["planes"]:
                assert np.linalg.norm(ref[name]) > 0, (k, name)
                assert fd.rel_l2(got[name], ref[name]) <= 1e-5, (k, rep, name, fd.rel_l2(got[name], ref[name]))
    r.close()


def test_l2_loss_entry_point_against_a_plain_reference():
    """rara_loss_l2 on a batch of views of mixed sizes (whole and ragged blocks, an element
    count that is not a multiple of 4): the per-view loss and gradient equal the plain
    float64 expressions; an output may be its target; invalid calls are refused."""
    sc = scenes.gradient_scene(400, seed=61, sh_degree=1)
    views = _views(61, scenes.MODE_RARA, sizes=((64, 64), (37, 29), (96, 80)))
    g = rara.GaussianTensors.from_scene(sc)
    r = rara.Renderer()
    try:
        with pytest.raises(rara.RaraError):   # nothing rendered on the context yet
            rara.rara_loss_l2(r.ctx, [], [], [], torch.empty(1, dtype=torch.float64, device="cuda"))
        vs = [rara.View(0, cam, pl, torch.empty((3, cam.height, cam.width), device="cuda"), None, None, bg)
              for cam, pl, bg in views]
        rara.rara_render_batch(r.ctx, [g], vs)
        gen = torch.Generator(device="cuda").manual_seed(5)
        targets = [torch.rand(v.image.shape, generator=gen, device="cuda") for v in vs]
        scale = [1.0 / v.image.numel() for v in vs[:2]] + [0.25]
        for alias in (False, True):
            tg = [t.clone() for t in targets]
            out = tg if alias else [torch.empty_like(t) for t in tg]
            loss = torch.full((len(vs),), float("nan"), dtype=torch.float64, device="cuda")
            rara.rara_loss_l2(r.ctx, tg, out, scale, loss)
            torch.cuda.synchronize()
            for k, v in enumerate(vs):
                d = v.image.double() - targets[k].double()
                ref_loss = float(scale[k] * (d * d).sum())
                assert abs(float(loss[k]) - ref_loss) <= 1e-5 * abs(ref_loss), (alias, k)
                ref_grad = (v.image - targets[k]) * float(np.float32(2.0) * np.float32(scale[k]))
                assert torch.allclose(out[k], ref_grad, rtol=1e-6, atol=1e-12), (alias, k)
        with pytest.raises(rara.RaraError):   # the gradient output is the rendered image
            rara.rara_loss_l2(r.ctx, targets, [v.image for v in vs], scale, loss)
        with pytest.raises(rara.RaraError):   # a non-finite scale
            rara.rara_loss_l2(r.ctx, targets, [torch.empty_like(t) for t in targets], [1.0, float("inf"), 1.0], loss)
    finally:
        r.close()


def test_autograd_function_matches_the_c_entry_point():
    from paper_2506_20202_gb300 import autograd
    sc = scenes.gradient_scene(64, seed=41, sh_degree=1)
    views = _views(41, scenes.MODE_RARA)
    weights = _weights(sc, views, 42)
    ref = gpu_gradients(sc, views, weights)
    g = rara.GaussianTensors.from_scene(sc)
    params = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)]
    planes = torch.tensor([list(pl.n) + [pl.d] for _, pl, _ in views], dtype=torch.float32, device="cuda",
                          requires_grad=True)
    r = rara.Renderer()
    imgs = autograd.render_views(r, *params, 1, [c for c, _, _ in views], planes, bgs=[bg for _, _, bg in views])
    loss = sum((img * torch.from_numpy(np.float32(w)).cuda()).sum() for img, w in zip(imgs, weights))
    loss.backward()
    for t, k in zip(params, fd.PARAMS):
        assert fd.rel_l2(t.grad.cpu().numpy(), ref[k]) <= 1e-5, k
    assert fd.rel_l2(planes.grad.cpu().numpy(), ref["planes"]) <= 1e-5
    # a second forward on the same renderer invalidates the first one's backward
    imgs1 = autograd.render_views(r, *params, 1, [c for c, _, _ in views], planes)
    autograd.render_views(r, *params, 1, [c for c, _, _ in views], planes)
    with pytest.raises(RuntimeError):
        sum(i.sum() for i in imgs1).backward()
    r.close()


def test_gradient_descent_reduces_an_l2_loss():
    """A few plain gradient steps on an L2 loss to target images lower the loss."""
    from paper_2506_20202_gb300 import autograd
    sc = scenes.gradient_scene(400, seed=51, sh_degree=2)
    rng = np.random.default_rng(52)
    target_sc = scenes.gradient_scene(400, seed=51, sh_degree=2)     # same layout, other colours and opacities
    target_sc.sh = np.ascontiguousarray(target_sc.sh + rng.normal(0, 0.4, target_sc.sh.shape).astype(np.float32))
    target_sc.opacity_logits = np.ascontiguousarray(target_sc.opacity_logits + np.float32(0.7))
    views = _views(51, scenes.MODE_RARA, sizes=((96, 96), (96, 96)))
    cams = [c for c, _, _ in views]
    planes0 = torch.tensor([list(pl.n) + [pl.d] for _, pl, _ in views], dtype=torch.float32, device="cuda")
    r = rara.Renderer()
    tg = rara.GaussianTensors.from_scene(target_sc)
    with torch.no_grad():
        targets = [t.clone() for t in autograd.render_views(r, tg.means, tg.log_scales, tg.quats, tg.opacity_logits,
                                                            tg.sh, 2, cams, planes0)]
    g = rara.GaussianTensors.from_scene(sc)
    params = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)]
    opt = torch.optim.Adam(params, lr=0.01)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        imgs = autograd.render_views(r, *params, 2, cams, planes0)
        loss = sum(((a - b) ** 2).mean() for a, b in zip(imgs, targets))
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.7 * losses[0], losses
    r.close()


def test_backward_reports_missing_state():
    sc = scenes.gradient_scene(50, seed=61, sh_degree=0)
    g = rara.GaussianTensors.from_scene(sc)
    r = rara.Renderer()
    dimg = [torch.zeros((3, 32, 32), device="cuda")]
    with pytest.raises(rara.RaraError) as e:                    # nothing rendered yet
        rara.rara_render_backward(r.ctx, dimg, [g.empty_like()])
    assert e.value.code == rara.RARA_ERR_INVALID_ARG
    cam = scenes.look_at_camera((0, 0, -3.0), (0, 0, 0), 32, 32)
    pl = scenes.Plane(np.float32([0, 0, 1]), 0.0)
    view = rara.View(0, cam, pl, torch.empty((3, 32, 32), device="cuda"))   # no final_T / n_contrib
    rara.rara_render_batch(r.ctx, [g], [view])
    with pytest.raises(rara.RaraError) as e:
        rara.rara_render_backward(r.ctx, dimg, [g.empty_like()])
    assert e.value.code == rara.RARA_ERR_INVALID_ARG
    r.close()
