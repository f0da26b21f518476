"""Error paths of the C ABI: argument checks, errors the kernels detect on the device,
budget refusals and a bounded device-side wait that gives up. No test faults, traps or
hangs the GPU: the time-out is a look-back word that nothing writes, waited on with a
lowered poll limit, and the kernel returns with a status the host reads."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20202_gb300 import rara, scenes
from tests.parity import IMG_MAX_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()


def _frame(n=20_000, seed=0, sh_degree=1, size=(160, 120)):
    sc = scenes.uniform_scene(n, seed=seed, sh_degree=sh_degree)
    cam = scenes.look_at_camera((0.3, -0.4, -3.0), (0.0, 0.0, 0.0), size[0], size[1], 60.0)
    pl = scenes.Plane(np.float32(scenes.random_unit_normal(seed + 1)), 0.05, 3.0, scenes.MODE_RARA)
    return sc, cam, pl


def _out(cam):
    H, W = cam.height, cam.width
    return (torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
            torch.empty((H, W), dtype=torch.int32, device="cuda"))


def _call_frame(ctx, g, cam, pl, img):
    """rara_render_frame through the raw C ABI (structs built by hand); returns the status."""
    c, p = rara.camera_struct(cam), rara.plane_struct(pl)
    bg = (C.c_float * 3)(0.0, 0.0, 0.0)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return rara.load().rara_render_frame(ctx, C.byref(g), C.byref(c), C.byref(p), bg, C.c_void_p(img.data_ptr()),
                                         None, None, s)


def test_invalid_arguments_are_refused_before_any_work():
    sc, cam, pl = _frame(2000)
    gs = rara.GaussianTensors.from_scene(sc)
    img = _out(cam)[0]
    ctx = rara.rara_ctx_create(0)
    lib = rara.load()
    try:
        launches0 = rara.rara_ctx_launches(ctx)
        bad = []
        g = gs.c_struct(); g.n = -1; bad.append((g, cam, pl))
        g = gs.c_struct(); g.n = 1 << 31; bad.append((g, cam, pl))
        g = gs.c_struct(); g.sh_degree = 4; bad.append((g, cam, pl))
        g = gs.c_struct(); g.sh_degree = -1; bad.append((g, cam, pl))
        g = gs.c_struct(); g.means = None; bad.append((g, cam, pl))
        for w, h in ((0, 64), (64, 0), (-5, 64)):
            c2 = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64)
            c2.width, c2.height = w, h
            bad.append((gs.c_struct(), c2, pl))
        for field, val in (("d", float("nan")), ("d", float("inf")), ("k_sigma", 0.0), ("mode", 7)):
            p2 = scenes.Plane(pl.n, pl.d, pl.k_sigma, pl.mode)
            setattr(p2, field, val)
            bad.append((gs.c_struct(), cam, p2))
        p2 = scenes.Plane(np.float32([np.nan, 0, 1]), 0.0)
        bad.append((gs.c_struct(), cam, p2))
        c2 = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64)
        c2.fx = float("nan")
        bad.append((gs.c_struct(), c2, pl))
        for g, c2, p2 in bad:
            assert _call_frame(ctx, g, c2, p2, img) == rara.RARA_ERR_INVALID_ARG
            assert lib.rara_last_error(ctx)
        # calls out of order: render and bin before any preprocess
        assert lib.rara_bin(ctx, None) == rara.RARA_ERR_INVALID_ARG
        bg = (C.c_float * 3)(0, 0, 0)
        assert lib.rara_render(ctx, bg, C.c_void_p(img.data_ptr()), None, None, None) == rara.RARA_ERR_INVALID_ARG
        assert lib.rara_ctx_create(0, 16, 16, None) == rara.RARA_ERR_INVALID_ARG
        assert rara.rara_ctx_launches(ctx) == launches0          # nothing was queued
        # the context still renders
        rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), img)
        torch.cuda.synchronize()
    finally:
        rara.rara_ctx_destroy(ctx)


@pytest.mark.parametrize("what", ["nan_mean", "zero_scale", "zero_quat", "nan_logit", "inf_sh"])
def test_non_finite_gaussians_are_reported_and_the_context_recovers(what):
    sc, cam, pl = _frame(5000, seed=3)
    ref_img = _out(cam)[0]
    ctx = rara.rara_ctx_create(0)
    try:
        gs = rara.GaussianTensors.from_scene(sc)
        rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), ref_img)
        torch.cuda.synchronize()
        broken = rara.GaussianTensors.from_scene(sc)
        k = 1234
        if what == "nan_mean":
            broken.means[1, k] = float("nan")
        elif what == "zero_scale":
            broken.log_scales[0, k] = float("-inf")
        elif what == "zero_quat":
            broken.quats[:, k] = 0.0
        elif what == "nan_logit":
            broken.opacity_logits[k] = float("nan")
        else:
            broken.sh[0, :] = float("inf")
        img = _out(cam)[0]
        with pytest.raises(rara.RaraError) as e:
            rara.rara_render_frame(ctx, broken, cam, pl, (0, 0, 0), img)
        assert e.value.code == rara.RARA_ERR_INVALID_ARG
        assert "non-finite" in str(e.value)
        # the next frame on the same context is clean and equal to the first render
        img.fill_(-1)
        rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), img)
        torch.cuda.synchronize()
        assert torch.equal(img, ref_img)
    finally:
        rara.rara_ctx_destroy(ctx)


def test_budget_refusal_keeps_within_the_budget():
    sc, cam, pl = _frame(20_000)
    gs = rara.GaussianTensors.from_scene(sc)
    img = _out(cam)[0]
    budget = 1 << 20                      # 1 MiB: below one frame's per-Gaussian records
    ctx = rara.rara_ctx_create(budget)
    try:
        with pytest.raises(rara.RaraError) as e:
            rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), img)
        assert e.value.code == rara.RARA_ERR_BUDGET
        assert rara.rara_ctx_bytes(ctx) <= budget
        small, scam, spl = _frame(200, seed=5, size=(64, 48))   # a frame that fits still renders
        simg = _out(scam)[0]
        rara.rara_render_frame(ctx, rara.GaussianTensors.from_scene(small), scam, spl, (0, 0, 0), simg)
        torch.cuda.synchronize()
        assert rara.rara_ctx_bytes(ctx) <= budget
    finally:
        rara.rara_ctx_destroy(ctx)


def test_a_lookback_wait_that_nothing_ends_gives_up_and_reports():
    # Partition 0 of the compaction is left unprocessed, so its look-back word is never
    # written; the other partitions' waits give up after 2000 polls (a few milliseconds),
    # record the time-out and return.
    sc, cam, pl = _frame(20_000, seed=7)
    gs = rara.GaussianTensors.from_scene(sc)
    ref = _out(cam)
    ctx = rara.rara_ctx_create(0)
    try:
        rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), *ref)
        torch.cuda.synchronize()
        rara.rara_ctx_debug_waits(ctx, 2000, True)
        out = _out(cam)
        with pytest.raises(rara.RaraError) as e:
            rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), *out)
        assert e.value.code == rara.RARA_ERR_TIMEOUT
        # the hook applied to that frame only: the context renders the frame again, exactly
        rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), *out)
        torch.cuda.synchronize()
        assert torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[2])
        # the same wait, bounded but not orphaned, completes normally
        rara.rara_ctx_debug_waits(ctx, 1 << 20, False)
        rara.rara_render_frame(ctx, gs, cam, pl, (0, 0, 0), *out)
        rara.rara_ctx_sync(ctx)
        assert float((out[0] - ref[0]).abs().max()) <= IMG_MAX_ABS
    finally:
        rara.rara_ctx_destroy(ctx)
