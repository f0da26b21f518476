"""Pins of the oracle's convex clip volume (several planes; the visible region is the
intersection of their visible sides), the extension the paper's Discussion names for other
clipping primitives. Closed forms, brute force along the ray, reduction to the one-plane
weight of Eq. 11 (computed there by a different formulation: chord-end visibility and the
plane hit t_p), invariants, and the three-way classification against every plane."""
import math

import numpy as np
import pytest

from paper_2506_20202_gb300 import scenes
from scipy.spatial.transform import Rotation

from tests.helpers import axis_camera, make_scene, plane


def rot_from_wxyz(q):
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def _vol(n, d, mode=scenes.MODE_RARA, extra=(), k=3.0):
    p = plane(n, d, mode, k)
    p.extra = tuple(tuple(float(v) for v in e) for e in extra)
    return p


def test_volume_of_one_plane_is_eq11(orc):
    """K = 1: the interval form equals Eq. 11 as the single-plane routine computes it."""
    rng = np.random.default_rng(21)
    for _ in range(300):
        q = rng.standard_normal(4)
        sig = rng.uniform(0.02, 0.12, 3)
        mu = rng.uniform(-0.2, 0.2, 3)
        e = np.array([0.1, -0.2, -3.0])
        tgt = mu + rng.normal(0, 0.1, 3)
        d = (tgt - e) / np.linalg.norm(tgt - e)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        dpl = -(n @ (mu + rng.normal(0, 0.1, 3)))
        w1, _ = orc.rara_weight(e, d, mu, q, sig, 3.0, n, dpl)
        wv = orc.rara_weight_volume(e, d, mu, q, sig, 3.0, [list(n) + [dpl]])
        assert wv == pytest.approx(w1, abs=1e-12)


def test_volume_slab_closed_form(orc):
    """Sphere of radius R, ray along +z at lateral offset b: the chord is z in [-h, h],
    h = sqrt(R^2 - b^2). The slab a <= z <= c keeps (min(c, h) - max(a, -h)) / (2h) of it
    (0 when that is negative), whatever the order of the two planes."""
    R, D = 0.2, 3.0
    sig = [R / 3] * 3
    quat = [0.3, -0.4, 0.5, 0.7]
    for b in (0.0, 0.5 * R, 0.95 * R):
        h = math.sqrt(R * R - b * b)
        for a, c in [(-0.5 * h, 0.5 * h), (-2 * h, 0.3 * h), (0.2 * h, 3 * h), (-3 * h, 3 * h),
                     (0.4 * h, 0.1 * h), (1.5 * h, 2.0 * h), (-0.9 * h, -0.7 * h)]:
            lower = [0, 0, 1, -a]   # z >= a
            upper = [0, 0, -1, c]   # z <= c
            want = max(0.0, min(c, h) - max(a, -h)) / (2 * h)
            for planes in ([lower, upper], [upper, lower]):
                w = orc.rara_weight_volume([b, 0, -D], [0, 0, 1], [0, 0, 0], quat, sig, 3.0, planes)
                assert w == pytest.approx(want, abs=1e-12)


def test_volume_wedge_closed_form(orc):
    """Ray along +x through a sphere at (0, y0, z0): planes x >= a and y >= c (the second is
    parallel to the ray). The chord is x in [-h, h]; w = the part with x >= a if y0 >= c,
    else 0."""
    R, D = 0.3, 4.0
    sig = [R / 3] * 3
    for y0, z0 in [(0.0, 0.0), (0.1, -0.05)]:
        h = math.sqrt(R * R - y0 * y0 - z0 * z0)
        for a in (-0.5 * h, 0.2 * h):
            for c in (y0 - 0.01, y0 + 0.01):
                w = orc.rara_weight_volume([-D, y0, z0], [1, 0, 0], [0, 0, 0], [1, 0, 0, 0], sig, 3.0,
                                           [[1, 0, 0, -a], [0, 1, 0, -c]])
                want = (h - a) / (2 * h) if y0 >= c else 0.0
                assert w == pytest.approx(want, abs=1e-12)


def test_volume_brute_force_chord_sampling(orc):
    """Rotated anisotropic ellipsoids and 2-3 random planes: w equals the fraction of chord
    samples (ray marched, inside test (x-mu)^T V^-1 (x-mu) <= 9 with V from scipy) that are
    on the visible side of every plane."""
    rng = np.random.default_rng(23)
    checked = 0
    for it in range(40):
        q = rng.standard_normal(4)
        sig = rng.uniform(0.03, 0.12, 3)
        mu = rng.uniform(-0.2, 0.2, 3)
        e = np.array([0.1, -0.2, -3.0])
        tgt = mu + rng.normal(0, 0.08, 3)
        d = (tgt - e) / np.linalg.norm(tgt - e)
        planes = []
        for _ in range(2 + it % 2):
            n = rng.standard_normal(3)
            n /= np.linalg.norm(n)
            planes.append(list(n) + [-(n @ (mu + rng.normal(0, 0.1, 3)))])
        w = orc.rara_weight_volume(e, d, mu, q, sig, 3.0, planes)
        Rm = rot_from_wxyz(q)
        Vinv = Rm @ np.diag(1 / sig ** 2) @ Rm.T
        ts = np.linspace(0.0, 6.0, 400_001)
        x = e[None, :] + ts[:, None] * d[None, :]
        dx = x - mu
        inside = np.einsum("ij,jk,ik->i", dx, Vinv, dx) <= 9.0
        if inside.sum() < 2000:
            continue
        vis = np.ones_like(inside)
        for p in planes:
            vis &= x @ np.asarray(p[:3]) + p[3] >= 0
        assert w == pytest.approx((inside & vis).sum() / inside.sum(), abs=2e-3)
        checked += 1
    assert checked >= 15


def test_volume_invariants(orc):
    """Plane order does not matter; a repeated plane changes nothing; a plane with the whole
    ellipsoid on its visible side changes nothing; adding a plane never raises w; a plane
    with the whole chord behind it gives 0; the two sides of one plane leave only the
    measure-zero plane, w = 0."""
    rng = np.random.default_rng(29)
    for _ in range(200):
        q = rng.standard_normal(4)
        sig = rng.uniform(0.02, 0.1, 3)
        mu = rng.uniform(-0.2, 0.2, 3)
        e = np.array([0.0, 0.3, -3.0])
        tgt = mu + rng.normal(0, 0.05, 3)
        d = (tgt - e) / np.linalg.norm(tgt - e)
        ps = []
        for _ in range(3):
            n = rng.standard_normal(3)
            n /= np.linalg.norm(n)
            ps.append(list(n) + [-(n @ (mu + rng.normal(0, 0.1, 3)))])
        W = lambda planes: orc.rara_weight_volume(e, d, mu, q, sig, 3.0, planes)
        w3 = W(ps)
        assert W([ps[2], ps[0], ps[1]]) == pytest.approx(w3, abs=1e-12)
        assert W(ps + [ps[1]]) == pytest.approx(w3, abs=1e-12)
        n = np.asarray(ps[0][:3])
        assert W(ps + [list(n) + [-(n @ mu) + 10.0]]) == pytest.approx(w3, abs=1e-12)
        assert W(ps[:2]) >= w3 - 1e-12 and W(ps[:1]) >= W(ps[:2]) - 1e-12
        # Eq. 11 for a plane with the ellipsoid wholly behind it: 0 if the ray meets the
        # ellipsoid twice in front, else 1
        hit0 = orc.rara_weight(e, d, mu, q, sig, 3.0, n, -(n @ mu) - 10.0)[0]
        assert hit0 in (0.0, 1.0)
        assert W(ps + [list(n) + [-(n @ mu) - 10.0]]) == pytest.approx(hit0 * w3, abs=1e-12)
        assert W([ps[0], list(-n) + [-ps[0][3]]]) == hit0


def test_volume_classification_every_plane(orc):
    """Two planes z >= 0 and x >= 0: invisible if the radius-r sphere is wholly behind either
    (d_ep,k < -r for some k), visible if wholly in front of both, cutoff otherwise; hard
    clipping: invisible iff the centre is behind either; the weight-on-all mode labels
    every non-invisible Gaussian cutoff."""
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 64, 64)
    sig = [0.01, 0.02, 0.015]
    r = 3 * np.exp(np.log(np.array(sig)).astype(np.float32).astype(np.float64)).max()
    eps = 1e-4
    offs = [-r - eps, -r + eps, 0.5 * r, r + eps, 3 * r]
    pts = [(x, 0.05, z) for x in offs for z in offs]
    sc = make_scene(pts, [sig] * len(pts))

    def rule(dk, mode):
        if mode == scenes.MODE_HARD:
            return 0 if min(dk) < 0 else 1
        if min(dk) < -r:
            return 0
        if mode == scenes.MODE_RARA_ALL:
            return 2
        return 1 if min(dk) > r else 2

    for mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL, scenes.MODE_HARD):
        pre = orc.preprocess(sc, cam, _vol([0, 0, 1], 0.0, mode, extra=[(1, 0, 0, 0)]))
        want = [rule((np.float32(z), np.float32(x)), mode) for x, _, z in pts]
        assert list(pre["label"]) == want, mode
        assert {0, 1, 2} <= set(want) or mode != scenes.MODE_RARA


def _tiny_scene(seed, n=80):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.6, 0.6, (n, 3))
    means[:, 2] += 2.5
    sig = np.exp(rng.normal(-2.8, 0.4, (n, 3)))
    return make_scene(means, sig, quats=rng.standard_normal((n, 4)), opacity=rng.uniform(0.05, 0.95, n),
                      rgb=rng.uniform(0, 1, (n, 3)))


@pytest.mark.parametrize("seed", [0, 1])
def test_volume_render_reductions(orc, seed):
    """Whole frames: extra planes with every Gaussian far in front of them, or a repeat of the
    first plane, render the single-plane image (the one-plane weight routine there, the
    interval form here); an extra plane with everything behind it leaves the background;
    hard clipping by two planes renders exactly the unclipped image of the Gaussians whose
    centres are in front of both; brute force and the tile lists agree exactly."""
    sc = _tiny_scene(seed)
    cam = axis_camera(32, 32, 32.0)
    rng = np.random.default_rng(200 + seed)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    d = -float(n @ [0, 0, 2.5])
    bg = (0.1, 0.2, 0.3)
    for mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL):
        one = orc.render_frame(sc, cam, plane(n, d, mode), bg=bg)[2]
        far = orc.render_frame(sc, cam, _vol(n, d, mode, extra=[(0, 1, 0, 1e20), (1, 0, 0, 1e20)]), bg=bg)[2]
        rep = orc.render_frame(sc, cam, _vol(n, d, mode, extra=[tuple(n) + (d,)]), bg=bg)[2]
        for o in (far, rep):
            assert np.abs(o["image"] - one["image"]).max() <= 1e-12
            assert np.abs(o["T"] - one["T"]).max() <= 1e-12
        none = orc.render_frame(sc, cam, _vol(n, d, mode, extra=[(0, 1, 0, -1e20)]), bg=bg)[2]
        for c in range(3):
            assert np.all(none["image"][c] == bg[c])
    # a wedge: two planes through the scene, both cutting Gaussians
    m = np.cross(n, [0.0, 1.0, 0.0])
    m /= np.linalg.norm(m)
    vol = _vol(n, d, scenes.MODE_RARA, extra=[tuple(m) + (-float(m @ [0.1, 0, 2.5]),)])
    pre = orc.preprocess(sc, cam, vol)
    assert (pre["label"] == 2).sum() > 0 and (pre["label"] == 0).sum() > 0
    kvr = orc.build_keys(pre)
    a = orc.render(sc, pre, cam, vol, bg, kvr, threads=2)
    b = orc.render(sc, pre, cam, vol, bg, None, threads=2)
    assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["T"], b["T"])
    hard = _vol(n, d, scenes.MODE_HARD, extra=vol.extra)
    p4 = orc.plane4(hard).reshape(-1, 4)
    mus = sc.means.astype(np.float64)
    keep = np.all(p4[:, :3] @ mus + p4[:, 3:4] >= 0.0, axis=0)
    sub = sc.subset(np.nonzero(keep)[0])
    ref = orc.render_frame(sub, cam, plane(n, 1e20, scenes.MODE_NONE), bg=bg)[2]
    got = orc.render_frame(sc, cam, hard, bg=bg)[2]
    assert np.array_equal(ref["image"], got["image"])
