"""The allocation-free frame render against the regular one, through the C ABI.

Some callers cannot allocate device memory (a plug-in inside another engine's frame loop,
a host callback, a process whose device memory another allocator owns). For them
rara_render_frame_noalloc keeps all scratch in a static device array; it must produce the
same frame as rara_render_frame. This file is collected last so that a run stopping at the
first failure has run every other test; it also passes alone in a fresh process.
"""
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
