"""Tile shapes and blend batch depths (the autotuner's knobs) against the FP64 oracle.

The oracle bins with the same tile shape; images must not depend on the tile (a tile lists
a Gaussian wherever one of its pixel centres can blend it) nor on the batch depth, and the
backward must give the same gradients whatever the tiling.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2506_20202_gb300 import autotune, rara, scenes
from tests import parity

pytestmark = pytest.mark.gpu

# (tile_w, tile_h, blend batch depth)
TILINGS = [(16, 16, 256), (32, 8, 256), (8, 32, 128), (8, 8, 512), (32, 16, 256), (16, 32, 512),
           (16, 16, 128), (16, 16, 512), (16, 16, 32), (16, 32, 32), (8, 8, 32)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()
    oracle.build()


def _workload():
    # 200 x 136: ragged in every tile shape (not a multiple of 32 or 16 in x, of 32 or 16 in y)
    return scenes.small_uniform_workload(n=8000, width=200, height=136, seed=23)


@pytest.mark.parametrize("tiling", TILINGS)
@pytest.mark.parametrize("tuning", [(33, 33), (0, 1)])
def test_tiling_against_the_oracle(tiling, tuning):
    scene, cam, pl = _workload()
    tw, th, _ = tiling
    report = {}
    gpu = parity.gpu_frame(scene, cam, pl, (0.05, 0.1, 0.2), tuning=tuning, tiling=tiling)
    pre = oracle.preprocess(scene, cam, pl, tile=(tw, th))
    kvr = oracle.build_keys(pre)
    parity.check_gaussians(pre, gpu["g"], report)
    parity.check_pairs(pre, kvr, gpu, report)
    ref = oracle.render(scene, pre, cam, pl, (0.05, 0.1, 0.2), kvr)
    parity.check_image(pre, ref, gpu, report)
    assert gpu["info"]["tiles_x"] == -(-cam.width // tw) and gpu["info"]["tiles_y"] == -(-cam.height // th)
    assert report["tiles_exact"] >= report["tiles"] - 5


def test_images_do_not_depend_on_the_tile_or_the_depth():
    scene, cam, pl = _workload()
    ref = parity.gpu_frame(scene, cam, pl, export=False, tuning=(33, 33), tiling=(16, 16, 256))
    for tiling in TILINGS[1:]:
        got = parity.gpu_frame(scene, cam, pl, export=False, tuning=(33, 33), tiling=tiling)
        if tiling[:2] == (8, 8):
            # 8x8 tiles always take 4 lanes per pixel: the same blends, summed in another order
            assert np.abs(got["image"] - ref["image"]).max() <= 1e-5
            assert np.abs(got["T"] - ref["T"]).max() <= 1e-5
        else:
            assert np.array_equal(got["image"], ref["image"]), tiling
            assert np.array_equal(got["T"], ref["T"]), tiling
        if tiling[:2] == (16, 16):
            assert np.array_equal(got["n_contrib"], ref["n_contrib"])   # the same lists


def test_backward_is_the_same_for_every_tiling():
    sc = scenes.gradient_scene(400, seed=4, sh_degree=2)
    cams = [scenes.look_at_camera((0.4, -0.3, -2.9), (0, 0, 0), 72, 56, 60.0),
            scenes.look_at_camera((-1.5, 0.5, -2.5), (0, 0, 0), 40, 64, 60.0)]
    pls = [scenes.Plane(np.float32(scenes.random_unit_normal(s)), 0.05, 3.0, scenes.MODE_RARA) for s in (3, 5)]
    gs = rara.GaussianTensors.from_scene(sc)
    rng = np.random.default_rng(1)
    dimgs = [torch.from_numpy(np.float32(rng.standard_normal((3, c.height, c.width)))).cuda() for c in cams]
    out = {}
    for tiling in ((16, 16, 256), (8, 8, 128), (32, 16, 512), (8, 32, 256), (16, 32, 32)):
        ctx = rara.rara_ctx_create(0)
        try:
            rara.rara_ctx_set_tiling(ctx, *tiling)
            views = [rara.View(0, c, p, torch.empty((3, c.height, c.width), device="cuda"),
                               torch.empty((c.height, c.width), device="cuda"),
                               torch.empty((c.height, c.width), dtype=torch.int32, device="cuda"))
                     for c, p in zip(cams, pls)]
            rara.rara_render_batch(ctx, [gs], views)
            g = gs.empty_like()
            pg = torch.empty((2, 4), device="cuda")
            rara.rara_render_backward(ctx, dimgs, [g], pg)
            torch.cuda.synchronize()
            out[tiling] = [t.cpu().numpy().astype(np.float64) for t in
                           (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, pg)]
        finally:
            rara.rara_ctx_destroy(ctx)
    ref = out[(16, 16, 256)]
    for tiling, got in out.items():
        for a, b in zip(got, ref):
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-7, tiling


def test_autotune_picks_a_supported_setting_that_matches_the_oracle():
    scene, cam, pl = scenes.small_uniform_workload(n=6000, width=160, height=120, seed=24)
    gs = rara.GaussianTensors.from_scene(scene)
    ctx = rara.rara_ctx_create(0)
    try:
        views = [rara.View(0, cam, pl, torch.empty((3, 120, 160), device="cuda"), torch.empty((120, 160), device="cuda"),
                         torch.empty((120, 160), dtype=torch.int32, device="cuda"))]
        best, ms = autotune.autotune(ctx, [gs], views, reps=2,
                                     candidates=[(33, 33), (11, 12), (0, 1)])
        assert best in ms and ms[best] == min(ms.values())
        assert best[:2] in autotune.TILES and best[2] in autotune.DEPTHS
        assert len({k[:2] for k in ms}) == len(autotune.TILES)       # every tile shape was timed
        rara.rara_render_batch(ctx, [gs], views)
        torch.cuda.synchronize()
        pre = oracle.preprocess(scene, cam, pl, tile=best[:2])
        ref = oracle.render(scene, pre, cam, pl, (0, 0, 0), oracle.build_keys(pre))
        parity.check_image(pre, ref, {"image": views[0].image.cpu().numpy().astype(np.float64),
                                      "T": views[0].final_T.cpu().numpy().astype(np.float64)}, {})
    finally:
        rara.rara_ctx_destroy(ctx)


def test_unsupported_tilings_are_refused():
    ctx = rara.rara_ctx_create(0)
    try:
        for bad in ((16, 8, 256), (64, 4, 256), (12, 12, 256), (16, 16, 64), (16, 16, 1024), (16, 16, 16)):
            with pytest.raises(rara.RaraError) as e:
                rara.rara_ctx_set_tiling(ctx, *bad)
            assert e.value.code == rara.RARA_ERR_INVALID_ARG
    finally:
        rara.rara_ctx_destroy(ctx)
    with pytest.raises(rara.RaraError):
        rara.rara_ctx_create(0, 16, 8)
