"""Baking a clip into the Gaussians on the GPU (an extension: the paper leaves re-fitting
after clipping to future work): the unclipped render of the baked scene must come closer to
the RaRa render of the original than the fit's starting point, than the cut Gaussians left
as they were, and than hard clipping, on the fitting cameras and on cameras it did not see."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20202_gb300 import bake, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()


def _orbit(k, count, W=160, H=120, elev=-0.4):
    a = 2.0 * np.pi * (k + 0.5) / count
    return scenes.look_at_camera((2.6 * np.sin(a), elev, -2.6 * np.cos(a)), (0.0, 0.0, 0.0), W, H, 60.0)


def test_bake_beats_the_unfitted_and_hard_clipped_scenes():
    sc = scenes.general_scene(30_000, seed=41, sh_degree=1)
    pl = scenes.Plane(np.float32(scenes.random_unit_normal(6)), 0.05, 3.0, scenes.MODE_RARA)
    cams = [_orbit(k, 8) for k in range(8)]
    held = [_orbit(k + 0.37, 3, elev=0.3) for k in range(3)]
    baked, rep = bake.bake_on_gpu(sc, pl, cams, steps=60, held_out=held)
    print({k: v for k, v in rep.items() if k != "losses"}, rep["losses"][::10])
    assert rep["free"] > 100 and rep["dropped"] > 100
    assert baked.n == rep["kept"]
    after, ho = rep["mse_after"], rep["held_out"]
    assert rep["losses"][-1] < 0.8 * rep["losses"][0]
    assert after["baked"] < after["start"] < after["kept_unclipped"]
    assert after["baked"] < after["hard_clip"]
    assert ho["baked"] < ho["kept_unclipped"] and ho["baked"] < ho["hard_clip"]
    for k in bake.PARAMS:
        assert np.all(np.isfinite(getattr(baked, k)))
