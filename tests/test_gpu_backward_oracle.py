"""The GPU backward against the oracle's analytic FP64 gradient on scenes of 10k+ Gaussians
(finite differences of the oracle, the other reference, cost one render per parameter and
stay on tiny scenes). Loss L = sum(weights * image) with seeded weights, zero on pixels whose
oracle sequence passes within tolerance of a discontinuity of the method, where a float32
renderer may decide differently; per parameter group relative L2 error <= 1e-3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import grad as ograd
from paper_2506_20202_gb300 import rara, scenes
from tests import fd, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()
    oracle.build()


def _mask(scene, cam, pl, bg):
    pre = oracle.preprocess(scene, cam, pl)
    out = oracle.render(scene, pre, cam, pl, bg, oracle.build_keys(pre))
    bad = out["events"] != 0
    near = np.nonzero(((pre["margin_class"] <= 1e-5) | (pre["margin_gauss"] <= 1e-5)) & (pre["culled"] == 0))[0]
    if near.size:
        bad |= oracle.support_mask(pre, near, cam.height, cam.width)
    return ~bad


def _compare(scene, views, tiling=(16, 16, 256)):
    rng = np.random.default_rng(17)
    weights = [rng.standard_normal((3, c.height, c.width)) * _mask(scene, c, p, bg) for c, p, bg in views]
    ref = {k: 0.0 for k in ograd.PARAMS}
    ref_planes = []
    for (cam, pl, bg), w in zip(views, weights):
        g = ograd.render_and_grad(scene, cam, pl, bg, w)
        for k in ograd.PARAMS:
            ref[k] = ref[k] + g[k]
        ref_planes.append(g["plane"])
    gs = rara.GaussianTensors.from_scene(scene)
    ctx = rara.rara_ctx_create(0)
    try:
        rara.rara_ctx_set_tiling(ctx, *tiling)
        vv = [rara.View(0, c, p, torch.empty((3, c.height, c.width), device="cuda"),
                        torch.empty((c.height, c.width), device="cuda"),
                        torch.empty((c.height, c.width), dtype=torch.int32, device="cuda"), bg)
              for c, p, bg in views]
        rara.rara_render_batch(ctx, [gs], vv)
        grads = gs.empty_like()
        pg = torch.empty((len(views), 4), device="cuda")
        rara.rara_render_backward(ctx, [torch.from_numpy(np.float32(w)).cuda() for w in weights], [grads], pg)
        torch.cuda.synchronize()
    finally:
        rara.rara_ctx_destroy(ctx)
    got = {k: getattr(grads, k).cpu().numpy().astype(np.float64) for k in ograd.PARAMS}
    errs = {k: fd.rel_l2(got[k], ref[k]) for k in ograd.PARAMS}
    errs["planes"] = fd.rel_l2(pg.cpu().numpy(), np.array(ref_planes))
    print(errs)
    for k, e in errs.items():
        assert e <= 1e-3, (k, e)
    return errs


def test_backward_against_the_oracle_gradient_12k_gaussians():
    scene = scenes.general_scene(12_000, seed=31, sh_degree=3)
    views = [(scenes.look_at_camera((0.3, -0.4, -2.4), (0.0, 0.0, 0.0), 128, 96, 60.0),
              scenes.Plane(np.float32(scenes.random_unit_normal(5)), 0.05, 3.0, scenes.MODE_RARA), (0.0, 0.0, 0.0)),
             (scenes.look_at_camera((-1.6, 0.6, -1.9), (0.0, 0.0, 0.0), 96, 112, 60.0),
              scenes.Plane(np.float32(scenes.random_unit_normal(8)), -0.1, 3.0, scenes.MODE_RARA), (0.1, 0.2, 0.3))]
    _compare(scene, views)


def test_backward_against_the_oracle_gradient_cutoff_heavy():
    # 10k wide Gaussians (a few pixels) around the plane: most rendered Gaussians are cutoff
    scene = scenes.gradient_scene(10_000, seed=32, sh_degree=1)
    pl = scenes.Plane(np.float32(scenes.random_unit_normal(12)), 0.0, 3.0, scenes.MODE_RARA)
    cam = scenes.look_at_camera((0.5, 0.3, -2.7), (0.0, 0.0, 0.0), 96, 80, 60.0)
    pre = oracle.preprocess(scene, cam, pl)
    rendered = pre["culled"] == 0
    assert (pre["label"][rendered] == oracle.CUTOFF).mean() > 0.3
    _compare(scene, [(cam, pl, (0.0, 0.0, 0.0))], tiling=(8, 8, 128))
