"""Batched multi-view render and its CUDA-graph replay, through the C ABI.

A batch renders many views (cameras, planes, resolutions) of one or more scenes with one
launch per stage; every view must equal the same view rendered alone (bit for bit: the
per-view arithmetic and list order are the same), and the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2506_20202_gb300 import rara, scenes
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()
    oracle.build()


def _outputs(cam):
    H, W = cam.height, cam.width
    return (torch.full((3, H, W), -1.0, dtype=torch.float32, device="cuda"),
            torch.full((H, W), -1.0, dtype=torch.float32, device="cuda"),
            torch.zeros((H, W), dtype=torch.int32, device="cuda"))


def _batch_case(seed=0):
    rng = np.random.default_rng(seed)
    sc = [scenes.uniform_scene(6000, seed=seed, sh_degree=1), scenes.general_scene(8000, seed=seed + 1, sh_degree=3)]
    sizes = [(160, 120), (96, 200), (256, 144), (64, 64), (200, 136), (33, 47)]
    views = []
    for k, (w, h) in enumerate(sizes):
        eye = rng.normal(0, 1, 3)
        eye = 3.0 * eye / np.linalg.norm(eye)
        cam = scenes.look_at_camera(eye, (0.0, 0.0, 0.0), w, h, 60.0)
        nrm = np.float32(scenes.random_unit_normal(seed * 100 + k))
        mode = [scenes.MODE_RARA, scenes.MODE_RARA, scenes.MODE_HARD, scenes.MODE_RARA_ALL, scenes.MODE_NONE,
                scenes.MODE_RARA][k]
        pl = scenes.Plane(nrm, float(rng.uniform(-0.2, 0.2)), 3.0, mode)
        views.append((k % 2, cam, pl, tuple(rng.uniform(0, 0.3, 3))))
    return sc, views


def _pairs(ctx, view):
    """The view's exported tile lists: 64-bit keys, Gaussian indices, per-tile ranges."""
    info = rara.rara_frame_info_get(ctx, view)
    p, nt = int(info["n_pairs"]), info["tiles_x"] * info["tiles_y"]
    keys = torch.zeros(max(p, 1), dtype=torch.int64, device="cuda")
    vals = torch.zeros(max(p, 1), dtype=torch.int32, device="cuda")
    ranges = torch.zeros((nt, 2), dtype=torch.int64, device="cuda")
    rara.rara_frame_pairs(ctx, view, keys, vals, ranges)
    torch.cuda.synchronize()
    return keys[:p].cpu().numpy(), vals[:p].cpu().numpy(), ranges.cpu().numpy()


def _render_batch(r, sc_t, views, graph=False):
    vs = []
    for (si, cam, pl, bg) in views:
        img, T, nc = _outputs(cam)
        vs.append(rara.View(si, cam, pl, img, T, nc, bg))
    fn = rara.rara_render_batch_graph if graph else rara.rara_render_batch
    fn(r.ctx, sc_t, vs)
    rara.rara_ctx_sync(r.ctx)
    return [(v.image.cpu().numpy(), v.final_T.cpu().numpy(), v.n_contrib.cpu().numpy()) for v in vs]


def test_batch_views_equal_single_renders():
    sc, views = _batch_case(0)
    sc_t = [rara.GaussianTensors.from_scene(s) for s in sc]
    r = rara.Renderer()
    got = _render_batch(r, sc_t, views)
    for (si, cam, pl, bg), (img, T, nc) in zip(views, got):
        ref = parity.gpu_frame(sc[si], cam, pl, bg, export=False)
        assert np.array_equal(img, ref["image"].astype(np.float32))
        assert np.array_equal(T, ref["T"].astype(np.float32))
        assert np.array_equal(nc, ref["n_contrib"])
    r.close()


def test_batch_views_against_oracle():
    sc, views = _batch_case(1)
    sc_t = [rara.GaussianTensors.from_scene(s) for s in sc]
    r = rara.Renderer()
    got = _render_batch(r, sc_t, views)
    for k, ((si, cam, pl, bg), (img, T, nc)) in enumerate(zip(views, got)):
        report = {}
        fg = r.frame_gaussians(sc[si].n, view=k)
        keys, vals, ranges, info = r.frame_pairs(view=k)
        gpu = dict(image=img.astype(np.float64), T=T.astype(np.float64), n_contrib=nc,
                   g={kk: v.cpu().numpy() for kk, v in fg.items()}, keys=keys.cpu().numpy().view(np.uint64),
                   vals=vals.cpu().numpy().view(np.uint32), ranges=ranges.cpu().numpy())
        pre = oracle.preprocess(sc[si], cam, pl)
        kvr = oracle.build_keys(pre)
        parity.check_gaussians(pre, gpu["g"], report)
        parity.check_pairs(pre, kvr, gpu, report)
        ref = oracle.render(sc[si], pre, cam, pl, bg, kvr)
        parity.check_image(pre, ref, gpu, report, max_flag_frac=0.08)
        assert info["n_pairs"] == report["pairs_gpu"]
    r.close()


def test_graph_replay_with_new_cameras_matches_exact():
    sc, views = _batch_case(2)
    sc_t = [rara.GaussianTensors.from_scene(s) for s in sc]
    rg = rara.Renderer()
    _render_batch(rg, sc_t, views, graph=True)                # renders exactly, then captures
    _, views2 = _batch_case(3)                                 # same shape, new cameras and planes
    views2 = [(views[k][0],) + tuple(views2[k][1:]) for k in range(len(views))]
    l0 = rara.rara_ctx_launches(rg.ctx)
    got = _render_batch(rg, sc_t, views2, graph=True)         # replay
    assert rara.rara_ctx_launches(rg.ctx) - l0 >= 10           # the graph's kernels ran
    re = rara.Renderer()
    ref = _render_batch(re, sc_t, views2)
    for (a, b) in zip(got, ref):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    rg.close()
    re.close()


def test_graph_overflow_is_reported_and_recovers():
    """A replay whose pairs exceed the captured capacity writes none past it, is reported
    as RARA_ERR_OVERFLOW, and the next call recaptures with room for them. Same shape
    (same n and SH degree), but the second scene's Gaussians are about 7 times larger."""
    small = scenes.uniform_scene(20000, seed=5, sh_degree=0)
    big = scenes.uniform_scene(20000, seed=5, sh_degree=0)
    big.log_scales = np.ascontiguousarray(big.log_scales + np.float32(2.0))
    pl = scenes.Plane(np.float32([0, 0, 1]), 0.0, 3.0, scenes.MODE_RARA)
    view = [(0, scenes.look_at_camera((0, 0, -3.0), (0, 0, 0), 128, 128, 60.0), pl, (0, 0, 0))]
    r = rara.Renderer()
    _render_batch(r, [rara.GaussianTensors.from_scene(small)], view, graph=True)
    big_t = [rara.GaussianTensors.from_scene(big)]
    with pytest.raises(rara.RaraError) as e:
        _render_batch(r, big_t, view, graph=True)
    assert e.value.code == rara.RARA_ERR_OVERFLOW
    got = _render_batch(r, big_t, view, graph=True)            # recaptures with a larger capacity
    got2 = _render_batch(r, big_t, view, graph=True)           # and replays it
    ref = _render_batch(rara.Renderer(), big_t, view)
    for a in (got, got2):
        for x, y in zip(a[0], ref[0]):
            assert np.array_equal(x, y)
    r.close()


def test_plane_sweep_from_one_camera_equals_single_renders():
    """Views that share a camera reuse the preprocess's projection (a plane sweep from one
    viewpoint): every view must still equal the view rendered alone bit for bit, including a
    view with another camera in the middle of the run and views whose mode labels a Gaussian
    invisible for one plane and visible for the next."""
    sc = scenes.general_scene(20_000, seed=7, sh_degree=3)
    cam = scenes.look_at_camera((0.4, -0.6, -2.8), (0.0, 0.0, 0.0), 200, 136, 60.0)
    other = scenes.look_at_camera((-1.5, 0.3, -2.5), (0.0, 0.0, 0.0), 200, 136, 60.0)
    nrm = np.float32(scenes.random_unit_normal(5))
    offs = np.linspace(-0.8, 0.8, 9)
    modes = [scenes.MODE_RARA, scenes.MODE_HARD, scenes.MODE_RARA, scenes.MODE_NONE, scenes.MODE_RARA_ALL,
             scenes.MODE_RARA, scenes.MODE_RARA, scenes.MODE_HARD, scenes.MODE_RARA]
    views = [(0, other if k == 4 else cam, scenes.Plane(nrm, float(d), 3.0, m), (0.1, 0.0, 0.2))
             for k, (d, m) in enumerate(zip(offs, modes))]
    gs = [rara.GaussianTensors.from_scene(sc)]
    r = rara.Renderer()
    try:
        got = _render_batch(r, gs, views)
        for (si, c, pl, bg), (img, T, nc) in zip(views, got):
            i0, T0, n0 = _outputs(c)
            r.render(gs[0], c, pl, bg, out=(i0, T0, n0))
            torch.cuda.synchronize()
            assert np.array_equal(img, i0.cpu().numpy()) and np.array_equal(T, T0.cpu().numpy())
            assert np.array_equal(nc, n0.cpu().numpy())
    finally:
        r.close()


def test_one_camera_batch_sorts_once_and_equals_single_renders():
    """A batch of one scene whose views all share one camera sorts the Gaussians by depth once
    and lists and tile-sorts them once, every view's lists then being the union's without the
    Gaussians it does not render: every view equals its single render bit for bit (image, T,
    contributor counts and tile lists), exactly and through graph replays with new planes,
    and a replay whose cameras differ recaptures (the depth order then differs per view)."""
    sc = scenes.general_scene(20_000, seed=9, sh_degree=2)
    cam = scenes.look_at_camera((0.3, 0.5, -2.9), (0.0, 0.0, 0.0), 176, 120, 60.0)
    nrm = np.float32(scenes.random_unit_normal(11))
    modes = [scenes.MODE_RARA, scenes.MODE_HARD, scenes.MODE_RARA_ALL, scenes.MODE_RARA, scenes.MODE_NONE,
             scenes.MODE_RARA]
    gs = [rara.GaussianTensors.from_scene(sc)]

    def views_for(offsets, cams):
        return [(0, c, scenes.Plane(nrm, float(d), 3.0, m), (0.0, 0.1, 0.2)) for d, m, c in zip(offsets, modes, cams)]

    def check(r, views, graph):
        got = _render_batch(r, gs, views, graph=graph)
        single = rara.Renderer()
        try:
            for k, ((si, c, pl, bg), (img, T, nc)) in enumerate(zip(views, got)):
                i0, T0, n0 = _outputs(c)
                single.render(gs[0], c, pl, bg, out=(i0, T0, n0))
                torch.cuda.synchronize()
                assert np.array_equal(img, i0.cpu().numpy()) and np.array_equal(T, T0.cpu().numpy())
                assert np.array_equal(nc, n0.cpu().numpy())
                if not graph:   # the same tile lists and per-Gaussian exports as the single render's
                    for a, b in zip(_pairs(r.ctx, k), _pairs(single.ctx, 0)):
                        assert np.array_equal(a, b)
                    ga, gb = r.frame_gaussians(sc.n, k), single.frame_gaussians(sc.n, 0)
                    for key in ga:
                        assert torch.equal(ga[key], gb[key]), key
        finally:
            single.close()

    r = rara.Renderer()
    try:
        v1 = views_for(np.linspace(-0.7, 0.7, 6), [cam] * 6)
        check(r, v1, graph=False)
        info = [rara.rara_frame_info_get(r.ctx, k) for k in range(6)]
        assert info[0]["n_depth_keys"] < sum(i["n_rendered"] for i in info)   # sorted once, not per view
        assert info[0]["n_depth_keys"] >= max(i["n_rendered"] for i in info)
        check(r, v1, graph=True)                                   # capture
        check(r, views_for(np.linspace(-0.5, 0.9, 6), [cam] * 6), graph=True)   # replay, new planes
        other = scenes.look_at_camera((-1.2, 0.2, -2.6), (0.0, 0.0, 0.0), 176, 120, 60.0)
        check(r, views_for(np.linspace(-0.5, 0.9, 6), [cam, other] * 3), graph=True)   # recapture
    finally:
        r.close()


@pytest.mark.parametrize("tiling", [(16, 16, 256, 33, 33), (8, 8, 128, 9, 11), (32, 16, 32, 10, 12)])
def test_one_camera_shared_lists_with_tilings_and_splits(tiling):
    """The shared tile lists under other tile shapes, blend depths and split thresholds (tiles
    split into 2 or 4 lanes per pixel by the per-view list lengths): still every view equals
    its single render with the same setting, including views whose plane hides everything."""
    from paper_2506_20202_gb300 import autotune
    sc = scenes.general_scene(30_000, seed=4, sh_degree=3)
    cam = scenes.look_at_camera((1.9, 0.6, -2.2), (0.0, 0.0, 0.0), 224, 160, 60.0)
    nrm = np.float32(scenes.random_unit_normal(5))
    gs = [rara.GaussianTensors.from_scene(sc)]
    offsets = list(np.linspace(-0.8, 0.8, 7)) + [-50.0]      # the last view hides every Gaussian
    views = [(0, cam, scenes.Plane(nrm, float(d), 3.0, scenes.MODE_RARA), (0.2, 0.1, 0.0)) for d in offsets]
    r, single = rara.Renderer(), rara.Renderer()
    try:
        autotune.apply(r.ctx, tiling)
        autotune.apply(single.ctx, tiling)
        got = _render_batch(r, gs, views)
        for k, ((si, c, pl, bg), (img, T, nc)) in enumerate(zip(views, got)):
            i0, T0, n0 = _outputs(c)
            single.render(gs[0], c, pl, bg, out=(i0, T0, n0))
            torch.cuda.synchronize()
            assert np.array_equal(img, i0.cpu().numpy()) and np.array_equal(T, T0.cpu().numpy())
            assert np.array_equal(nc, n0.cpu().numpy())
            for a, b in zip(_pairs(r.ctx, k), _pairs(single.ctx, 0)):
                assert np.array_equal(a, b)
        assert rara.rara_frame_info_get(r.ctx, len(views) - 1)["n_pairs"] == 0
        assert np.all(got[-1][0] == np.float32([0.2, 0.1, 0.0])[:, None, None])
    finally:
        r.close()
        single.close()


def test_one_camera_batch_beyond_shared_list_views():
    """A one-camera batch of more views than the shared listing's 32 keeps the per-view
    listing over the expanded depth order; every view still equals its single render."""
    sc = scenes.general_scene(6000, seed=6, sh_degree=1)
    cam = scenes.look_at_camera((0.4, -0.3, -2.8), (0.0, 0.0, 0.0), 64, 48, 60.0)
    nrm = np.float32(scenes.random_unit_normal(8))
    gs = [rara.GaussianTensors.from_scene(sc)]
    views = [(0, cam, scenes.Plane(nrm, float(d), 3.0, scenes.MODE_RARA), (0.0, 0.0, 0.0))
             for d in np.linspace(-0.9, 0.9, 35)]
    r, single = rara.Renderer(), rara.Renderer()
    try:
        got = _render_batch(r, gs, views)
        for k, ((si, c, pl, bg), (img, T, nc)) in enumerate(zip(views, got)):
            i0, T0, n0 = _outputs(c)
            single.render(gs[0], c, pl, bg, out=(i0, T0, n0))
            torch.cuda.synchronize()
            assert np.array_equal(img, i0.cpu().numpy()) and np.array_equal(T, T0.cpu().numpy())
            if k % 7 == 0:
                for a, b in zip(_pairs(r.ctx, k), _pairs(single.ctx, 0)):
                    assert np.array_equal(a, b)
    finally:
        r.close()
        single.close()


def test_one_camera_batch_backward_equals_single_view_backwards():
    """The backward of a one-camera batch (shared lists and records) against the sum of the
    views' single-frame backwards: the parameter gradients agree up to the order of the
    floating-point atomics, and every view's plane gradient too."""
    sc = scenes.general_scene(12_000, seed=17, sh_degree=2)
    cam = scenes.look_at_camera((0.9, -0.4, -2.6), (0.0, 0.0, 0.0), 144, 112, 60.0)
    nrm = np.float32(scenes.random_unit_normal(19))
    planes = [scenes.Plane(nrm, float(d), 3.0, m) for d, m in
              zip(np.linspace(-0.5, 0.5, 5), [scenes.MODE_RARA, scenes.MODE_RARA_ALL, scenes.MODE_HARD,
                                               scenes.MODE_RARA, scenes.MODE_NONE])]
    gs = rara.GaussianTensors.from_scene(sc)
    rng = np.random.default_rng(5)
    dimgs = [torch.from_numpy(np.float32(rng.standard_normal((3, cam.height, cam.width)))).cuda() for _ in planes]

    def grads_of(views_planes, dims):
        ctx = rara.rara_ctx_create(0)
        try:
            vs = [rara.View(0, cam, p, torch.empty((3, cam.height, cam.width), device="cuda"),
                            torch.empty((cam.height, cam.width), device="cuda"),
                            torch.empty((cam.height, cam.width), dtype=torch.int32, device="cuda"))
                  for p in views_planes]
            rara.rara_render_batch(ctx, [gs], vs)
            g = gs.empty_like()
            pg = torch.empty((len(vs), 4), device="cuda")
            rara.rara_render_backward(ctx, dims, [g], pg)
            torch.cuda.synchronize()
            return [t.cpu().numpy().astype(np.float64) for t in
                    (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)], pg.cpu().numpy().astype(np.float64)
        finally:
            rara.rara_ctx_destroy(ctx)

    batch, batch_pg = grads_of(planes, dimgs)
    total = None
    for k, p in enumerate(planes):
        one, one_pg = grads_of([p], [dimgs[k]])
        total = one if total is None else [a + b for a, b in zip(total, one)]
        assert np.allclose(batch_pg[k], one_pg[0], rtol=1e-4, atol=1e-6)
    for a, b in zip(batch, total):
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-7
