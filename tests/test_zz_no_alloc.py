"""The allocation-free frame render against the regular one, through the C ABI.

Some callers cannot allocate device memory (a plug-in inside another engine's frame loop,
a host callback, a process whose device memory another allocator owns). For them
rara_render_frame_noalloc keeps all scratch in a static device array; it must produce the
same frame as rara_render_frame. This file is collected last so that a run stopping at the
first failure has run every other test; it also passes alone in a fresh process.
"""
import dataclasses
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20202_gb300 import rara, scenes
from tests.parity import IMG_MAX_ABS, IMG_MEAN_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()


def _outputs(cam):
    H, W = cam.height, cam.width
    return (torch.zeros((3, H, W), dtype=torch.float32, device="cuda"),
            torch.zeros((H, W), dtype=torch.float32, device="cuda"),
            torch.zeros((H, W), dtype=torch.int32, device="cuda"))


def test_noalloc_matches_regular_render_twice_in_a_row():
    cases = []
    for seed, plane_seed in ((0, 1), (5, 9)):   # two calls in a row, different frames
        scene = scenes.uniform_scene(20_000, seed=seed, sh_degree=2)
        cam = scenes.look_at_camera((0.3, -0.4, -3.0), (0.0, 0.0, 0.0), 320, 240, 60.0)
        pl = scenes.Plane(np.float32(scenes.random_unit_normal(plane_seed)), 0.05, 3.0, scenes.MODE_RARA)
        cases.append((rara.GaussianTensors.from_scene(scene), cam, pl))
    ref = []
    r = rara.Renderer()
    for gs, cam, pl in cases:
        out = _outputs(cam)
        r.render(gs, cam, pl, (0.1, 0.2, 0.3), out=out)
        torch.cuda.synchronize()
        ref.append([t.clone() for t in out])
    r.close()
    for (gs, cam, pl), (img0, T0, nc0) in zip(cases, ref):
        img, T, nc = _outputs(cam)
        img.fill_(-1.0)
        rara.rara_render_frame_noalloc(gs, cam, pl, (0.1, 0.2, 0.3), img, T, nc)
        torch.cuda.synchronize()
        d = (img - img0).abs()
        assert float(d.max()) <= IMG_MAX_ABS and float(d.mean()) <= IMG_MEAN_ABS
        assert float((T - T0).abs().max()) <= IMG_MAX_ABS
        assert torch.equal(nc, nc0)


def test_noalloc_rejects_sizes_beyond_its_limit():
    scene = scenes.uniform_scene(70_000, seed=1)      # above the 65536-Gaussian limit
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 64, 64, 60.0)
    pl = scenes.Plane(np.float32([0, 0, 1]), 0.0)
    img, T, nc = _outputs(cam)
    with pytest.raises(rara.RaraError) as e:
        rara.rara_render_frame_noalloc(rara.GaussianTensors.from_scene(scene), cam, pl, (0, 0, 0), img, T, nc)
    assert e.value.code == rara.RARA_ERR_BUDGET
    big = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 4096, 4096, 60.0)  # 65536 tiles
    small = scenes.uniform_scene(100, seed=2)
    img, T, nc = _outputs(big)
    with pytest.raises(rara.RaraError) as e:
        rara.rara_render_frame_noalloc(rara.GaussianTensors.from_scene(small), big, pl, (0, 0, 0), img, T, nc)
    assert e.value.code == rara.RARA_ERR_BUDGET


def _case(seed, plane_seed):
    scene = scenes.uniform_scene(20_000, seed=seed, sh_degree=2)
    cam = scenes.look_at_camera((0.3, -0.4, -3.0), (0.0, 0.0, 0.0), 320, 240, 60.0)
    pl = scenes.Plane(np.float32(scenes.random_unit_normal(plane_seed)), 0.05, 3.0, scenes.MODE_RARA)
    return rara.GaussianTensors.from_scene(scene), cam, pl


def test_noalloc_allocates_nothing_and_recovers_after_the_pair_limit():
    gs, cam, pl = _case(3, 4)
    ref = _outputs(cam)
    r = rara.Renderer()
    r.render(gs, cam, pl, (0.0, 0.0, 0.0), out=ref)
    r.close()
    out = _outputs(cam)
    # 3000 wide splats (sigma 0.1 at distance 3, about 500 rectangle tiles each) at 2048^2:
    # within the Gaussian and tile limits, but 1.5M pairs, above the 2^19 pair limit, which
    # is found only after the preprocess has run on the shared array
    wide = scenes.uniform_scene(3000, seed=6)
    wide = dataclasses.replace(wide, log_scales=np.full_like(wide.log_scales, np.log(0.1)))
    gw = rara.GaussianTensors.from_scene(wide)
    big = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 2048, 2048, 60.0)
    bimg, bT, bnc = _outputs(big)
    rara.rara_render_frame_noalloc(gs, cam, pl, (0, 0, 0), *out)   # set-up done before measuring
    first = [torch.empty_like(t) for t in out]
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    count0 = torch.cuda.memory_stats()["allocation.all.allocated"]   # allocations made through torch
    with pytest.raises(rara.RaraError) as e:
        rara.rara_render_frame_noalloc(gw, big, pl, (0, 0, 0), bimg, bT, bnc)
    assert e.value.code == rara.RARA_ERR_BUDGET
    # the next calls render normally, over what the refused one left (in-place copies only, so
    # nothing in this span allocates through torch either)
    for t in out:
        t.fill_(-1)
    rara.rara_render_frame_noalloc(gs, cam, pl, (0, 0, 0), *out)
    for a, b in zip(first, out):
        a.copy_(b)
    for t in out:
        t.fill_(-1)
    rara.rara_render_frame_noalloc(gs, cam, pl, (0, 0, 0), *out)
    torch.cuda.synchronize()
    # nothing was allocated on the device across the calls, by the library or through torch
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == count0
    for got in (first, out):
        assert torch.equal(got[2], ref[2])
        assert float((got[0] - ref[0]).abs().max()) <= IMG_MAX_ABS
        assert float((got[1] - ref[1]).abs().max()) <= IMG_MAX_ABS
