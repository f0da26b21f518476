"""Serving loop: continuous batching gives each request the same image as rendering it
alone, and that image matches the FP64 oracle; the slots' contexts stay within their
share of the budget and, once warmed, allocate nothing while serving."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2506_20202_gb300 import rara, scenes, serve
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20202_gb300 import build
    build.build()


def _scenes():
    return {"a": rara.GaussianTensors.from_scene(scenes.uniform_scene(5000, seed=1, sh_degree=1)),
            "b": rara.GaussianTensors.from_scene(scenes.general_scene(12000, seed=2, sh_degree=3))}


def test_each_result_equals_the_request_rendered_alone():
    sc = _scenes()
    reqs = serve.poisson_requests(["a", "b"], serve.orbit_camera, rate_hz=4000.0, duration_s=0.012, seed=3,
                                  resolutions=((128, 128), (200, 120), (96, 160)))
    assert len(reqs) >= 20
    srv = serve.Server(sc, budget_bytes=4 << 30, slots=2, max_batch=8)
    try:
        results = srv.run(reqs)
    finally:
        srv.close()
    assert len(results) == len(reqs) and srv.rejected == 0
    assert srv.batches < len(reqs)                       # requests were batched
    # a seeded sample of the served images against the FP64 oracle at the image bars
    host = {"a": scenes.uniform_scene(5000, seed=1, sh_degree=1), "b": scenes.general_scene(12000, seed=2, sh_degree=3)}
    rng = np.random.default_rng(5)
    for k in rng.choice(len(reqs), size=8, replace=False):
        req, res = reqs[int(k)], results[int(k)]
        pre, kvr, ref = oracle.render_frame(host[req.scene], req.camera, req.plane, req.bg)
        report = {}
        parity.check_image(pre, ref, {"image": res.image.numpy().astype(np.float64)}, report, max_flag_frac=0.08)
    ctx = rara.rara_ctx_create(0)
    try:
        for req, res in zip(reqs, results):
            H, W = req.camera.height, req.camera.width
            img = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
            rara.rara_render_frame(ctx, sc[req.scene], req.camera, req.plane, req.bg, img)
            torch.cuda.synchronize()
            assert torch.equal(img.cpu(), res.image), req.rid
            assert res.latency_ms > 0
    finally:
        rara.rara_ctx_destroy(ctx)


def test_admission_refuses_requests_beyond_the_budget():
    sc = _scenes()
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64)
    pl = scenes.Plane(np.float32([0, 0, 1]), 0.0)
    resident = sum(sum(t.numel() * 4 for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh))
                   for g in sc.values())
    need = serve.request_bytes(sc["b"].n, 64, 64)
    srv = serve.Server(sc, budget_bytes=resident + need, slots=2)   # each slot gets half of `need`
    try:
        res = srv.run([serve.Request(0, "b", cam, pl, (0, 0, 0), 0.0), serve.Request(1, "a", cam, pl, (0, 0, 0), 0.0)])
    finally:
        srv.close()
    assert srv.rejected == 1 and [r.rid for r in res] == [1]


def test_plain_baseline_serves_in_order():
    sc = _scenes()
    reqs = serve.poisson_requests(["a"], serve.orbit_camera, rate_hz=500.0, duration_s=0.02, seed=4,
                                  resolutions=((96, 96),))
    res = serve.serve_plain(sc, reqs)
    assert [r.rid for r in res] == [r.rid for r in reqs]
    s = serve.summarize(res)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_warmed_server_reserves_within_its_share_and_allocates_nothing_while_serving():
    sc = _scenes()
    res_list = ((128, 128), (200, 120))
    srv = serve.Server(sc, budget_bytes=2 << 30, slots=2, max_batch=8, resolutions=res_list, reserve_batch=4)
    try:
        srv.warm(serve.orbit_camera, seed=1, per_shape=1, pinned_per_res=4)
        held = [rara.rara_ctx_bytes(s.ctx) for s in srv.slots]
        assert all(0 < h <= srv.share for h in held)
        reqs = serve.poisson_requests(["a", "b"], serve.orbit_camera, rate_hz=3000.0, duration_s=0.02, seed=9,
                                      resolutions=res_list)
        results = srv.run(reqs)
        assert len(results) == len(reqs) and srv.rejected == 0
        assert [rara.rara_ctx_bytes(s.ctx) for s in srv.slots] == held
    finally:
        srv.close()
