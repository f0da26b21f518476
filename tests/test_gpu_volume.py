"""Convex clip volumes (several planes, visible region = the intersection of their visible
sides) on the CUDA path, through the C ABI, against the FP64 oracle: labels, tile lists and
images at the same bars as the single plane; batches that mix single planes and volumes;
graph replays; and the calls that accept single planes only."""
import math

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


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def _volume(name, mode=scenes.MODE_RARA, shift=0.0):
    """A plane plus further planes (nx, ny, nz, d) through the middle of the uniform scenes."""
    if name == "wedge":
        planes = [(_unit([0.3, 0.8, -0.5]), 0.05 + shift), (_unit([-0.7, 0.2, 0.4]), -0.1)]
    elif name == "slab":
        n = _unit([0.2, -0.4, 0.9])
        planes = [(n, 0.15 + shift), (-n, 0.15)]
    elif name == "corner4":
        planes = [(_unit([1, 0, 0]), 0.3 + shift), (_unit([0, -1, 0]), 0.4), (_unit([0, 0, 1]), 0.2),
                  (_unit([1, 1, 1]), 0.2)]
    else:
        raise KeyError(name)
    n0, d0 = planes[0]
    extra = tuple(tuple(float(x) for x in np.float32(n)) + (float(np.float32(d)),) for n, d in planes[1:])
    return scenes.Plane(np.float32(n0), float(np.float32(d0)), 3.0, mode, extra)


def _multi_split(scene, vol):
    """Gaussians whose traced 3-sigma ellipsoid two or more planes of the volume cut and none
    leaves wholly behind it (the ones the render clips against several planes)."""
    p4 = oracle.plane4(vol).reshape(-1, 4)
    mu = scene.means.astype(np.float64)
    sig = np.exp(scene.log_scales.astype(np.float64))
    q = scene.quats.astype(np.float64)
    q = q / np.linalg.norm(q, axis=0)
    w, x, y, z = q
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)])])
    split = np.zeros(scene.n, int)
    hidden = np.zeros(scene.n, bool)
    for nx, ny, nz, d in p4:
        dep = nx * mu[0] + ny * mu[1] + nz * mu[2] + d
        rn = np.einsum("abn,a->bn", R, np.array([nx, ny, nz]))  # R^T n per Gaussian
        supp = 3.0 * np.linalg.norm(sig * rn, axis=0)
        split += np.abs(dep) <= supp
        hidden |= dep < -supp
    return int(((split >= 2) & ~hidden).sum())


def full_check(scene, cam, pl, bg=(0.0, 0.0, 0.0), rows=None, tuning=None, max_flag_frac=0.05):
    report = {}
    gpu = parity.gpu_frame(scene, cam, pl, bg, tuning=tuning)
    pre = oracle.preprocess(scene, cam, pl)
    kvr = oracle.build_keys(pre)
    parity.check_gaussians(pre, gpu["g"], report)
    parity.check_pairs(pre, kvr, gpu, report)
    ref = oracle.render(scene, pre, cam, pl, bg, kvr, rows=rows)
    parity.check_image(pre, ref, gpu, report, rows=rows, max_flag_frac=max_flag_frac)
    print(report)
    return report, gpu, ref


def _case(seed=2):
    return scenes.small_uniform_workload(n=6000, width=160, height=128, seed=seed)


@pytest.mark.parametrize("mode", [scenes.MODE_RARA, scenes.MODE_RARA_ALL, scenes.MODE_HARD])
@pytest.mark.parametrize("name", ["wedge", "slab", "corner4"])
def test_volume_parity(name, mode):
    scene, cam, _ = _case()
    vol = _volume(name, mode)
    if mode == scenes.MODE_RARA:
        assert _multi_split(scene, vol) >= 20  # the case clips Gaussians against several planes
    rep, gpu, _ = full_check(scene, cam, vol, bg=(0.2, 0.1, 0.05))
    if mode != scenes.MODE_HARD:
        assert gpu["info"]["n_cutoff"] > 100


@pytest.mark.parametrize("tuning", [(0, 1), (1, 33), (5, 7)])
def test_volume_multi_lane_pixels(tuning):
    """The 2- and 4-lane pixel paths of the render evaluate the volume weight too."""
    scene, cam, _ = _case(seed=5)
    full_check(scene, cam, _volume("corner4"), tuning=tuning)


def test_far_planes_drop_out():
    """Further planes with every Gaussian far in front of them leave labels, lists and image
    as the single plane gives them."""
    scene, cam, pl = _case(seed=3)
    vol = scenes.Plane(pl.n, pl.d, pl.k_sigma, pl.mode, ((0.0, 1.0, 0.0, 1e6), (1.0, 0.0, 0.0, 1e6)))
    a = parity.gpu_frame(scene, cam, pl)
    b = parity.gpu_frame(scene, cam, vol)
    assert np.array_equal(a["g"]["labels"], b["g"]["labels"])
    assert np.array_equal(a["keys"], b["keys"]) and np.array_equal(a["vals"], b["vals"])
    assert np.abs(a["image"] - b["image"]).max() <= 1e-6
    assert np.array_equal(a["n_contrib"], b["n_contrib"])


def _outputs(cam):
    H, W = cam.height, cam.width
    return (torch.full((3, H, W), -1.0, dtype=torch.float32, device="cuda"),
            torch.full((H, W), -1.0, dtype=torch.float32, device="cuda"),
            torch.zeros((H, W), dtype=torch.int32, device="cuda"))


def _mixed_views(shift=0.0):
    sizes = [(160, 120), (96, 200), (128, 128), (33, 47), (200, 136)]
    rng = np.random.default_rng(17)
    out = []
    for k, (w, h) in enumerate(sizes):
        eye = rng.normal(0, 1, 3)
        cam = scenes.look_at_camera(3.0 * eye / np.linalg.norm(eye), (0.0, 0.0, 0.0), w, h, 60.0)
        if k == 0:
            pl = scenes.Plane(np.float32(scenes.random_unit_normal(40)), 0.05 + shift, 3.0, scenes.MODE_RARA)
        else:
            name, mode = [("wedge", scenes.MODE_RARA), ("corner4", scenes.MODE_RARA_ALL), ("slab", scenes.MODE_HARD),
                          ("corner4", scenes.MODE_RARA)][k - 1]
            pl = _volume(name, mode, shift)
        out.append((k % 2, cam, pl, tuple(rng.uniform(0, 0.3, 3))))
    return out


def _render_batch(r, sc_t, views, graph=False):
    vs = []
    for (si, cam, pl, bg) in views:
        img, T, nc = _outputs(cam)
        vs.append(rara.View(si, cam, pl, img, T, nc, bg))
    fn = rara.rara_render_batch_graph if graph else rara.rara_render_batch
    fn(r.ctx, sc_t, vs)
    rara.rara_ctx_sync(r.ctx)
    return [(v.image.cpu().numpy(), v.final_T.cpu().numpy(), v.n_contrib.cpu().numpy()) for v in vs]


def test_volume_batch_mixed_equals_alone_and_oracle():
    """A batch mixing a single plane with volumes of 2-4 planes in every mode: each view equals
    the view rendered alone (bit for bit for the volumes, which run the same kernel variant
    alone; within 1e-6 for the single plane, whose lone render runs the single-plane variant)
    and the oracle."""
    sc = [scenes.uniform_scene(6000, seed=1, sh_degree=1), scenes.general_scene(8000, seed=2, sh_degree=3)]
    views = _mixed_views()
    r = rara.Renderer()
    try:
        sc_t = [rara.GaussianTensors.from_scene(s) for s in sc]
        batch = _render_batch(r, sc_t, views)
        for k, (si, cam, pl, bg) in enumerate(views):
            alone = _render_batch(r, [sc_t[si]], [(0, cam, pl, bg)])[0]
            if k == 0:
                assert np.abs(batch[k][0] - alone[0]).max() <= 1e-6
            else:
                for a, b in zip(batch[k], alone):
                    assert np.array_equal(a, b), f"view {k}"
            pre = oracle.preprocess(sc[si], cam, pl)
            kvr = oracle.build_keys(pre)
            ref = oracle.render(sc[si], pre, cam, pl, bg, kvr)
            gpu = dict(image=batch[k][0].astype(np.float64), T=batch[k][1].astype(np.float64))
            parity.check_image(pre, ref, gpu, {})
    finally:
        r.close()


def test_volume_graph_replay_and_recapture():
    """Graph replays of a batch with volumes, with moved planes, equal the exact batch render;
    a batch of the same sizes with single planes only is recaptured and also equals its exact
    render."""
    sc = [scenes.uniform_scene(6000, seed=1, sh_degree=1), scenes.general_scene(8000, seed=2, sh_degree=3)]
    r = rara.Renderer()
    try:
        sc_t = [rara.GaussianTensors.from_scene(s) for s in sc]
        for shift in (0.0, 0.07, -0.05):
            views = _mixed_views(shift)
            g = _render_batch(r, sc_t, views, graph=True)
            e = _render_batch(r, sc_t, views, graph=False)
            for a, b in zip(g, e):
                for x, y in zip(a, b):
                    assert np.array_equal(x, y)
        single = [(si, cam, scenes.Plane(np.float32(scenes.random_unit_normal(50 + k)), 0.0, 3.0, scenes.MODE_RARA), bg)
                  for k, (si, cam, _, bg) in enumerate(_mixed_views())]
        g = _render_batch(r, sc_t, single, graph=True)
        e = _render_batch(r, sc_t, single, graph=False)
        for a, b in zip(g, e):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    finally:
        r.close()


def test_volume_full_size_sampled_rows():
    """The benchmark workload (1M Gaussians, SH 3, 1920x1080) clipped by a wedge of two planes
    through the scene: 32 full rows against the oracle."""
    scene, cam, planes = scenes.general_workload(1_000_000, 1920, 1080, seed=0, sweep=16)
    p0 = planes[8]
    m = np.cross(np.asarray(p0.n, np.float64), [0.0, 1.0, 0.0])
    m = m / np.linalg.norm(m)
    vol = scenes.Plane(p0.n, p0.d, 3.0, scenes.MODE_RARA,
                       (tuple(float(x) for x in np.float32(m)) + (0.05,),))
    assert _multi_split(scene, vol) >= 1000
    rep, _, _ = full_check(scene, cam, vol, rows=(520, 552))
    assert rep["pixels"] == 32 * 1920


def test_volume_argument_errors():
    scene, cam, pl = _case(seed=4)
    gs = rara.GaussianTensors.from_scene(scene)
    r = rara.Renderer()
    try:
        too_many = scenes.Plane(pl.n, pl.d, 3.0, pl.mode, ((1.0, 0, 0, 1),) * 4)
        with pytest.raises(rara.RaraError) as e:
            r.render(gs, cam, too_many)
        assert e.value.code == rara.RARA_ERR_INVALID_ARG
        nan = scenes.Plane(pl.n, pl.d, 3.0, pl.mode, ((1.0, 0, 0, math.nan),))
        with pytest.raises(rara.RaraError) as e:
            r.render(gs, cam, nan)
        assert e.value.code == rara.RARA_ERR_INVALID_ARG
        # the backward takes single planes only
        vol = _volume("wedge")
        img, T, nc = _outputs(cam)
        rara.rara_render_batch(r.ctx, [gs], [rara.View(0, cam, vol, img, T, nc)])
        with pytest.raises(rara.RaraError) as e:
            rara.rara_render_backward(r.ctx, [torch.ones_like(img)], [gs.empty_like()])
        assert e.value.code == rara.RARA_ERR_INVALID_ARG
    finally:
        r.close()
    img, T, nc = _outputs(cam)
    with pytest.raises(rara.RaraError) as e:
        rara.rara_render_frame_noalloc(gs, cam, _volume("wedge"), (0, 0, 0), img, T, nc)
    assert e.value.code == rara.RARA_ERR_INVALID_ARG
