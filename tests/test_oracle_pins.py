"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, a special
case that reduces to a library routine (scipy), brute force on a tiny input, or an
invariant the paper states. None of these calls the CUDA library.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

from paper_2506_20202_gb300 import scenes
from tests.helpers import Y00, axis_camera, make_scene, plane

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def scipy_real_sh(l, m, d):
    d = np.asarray(d, np.float64) / np.linalg.norm(d)
    th, ph = math.acos(max(-1.0, min(1.0, d[2]))), math.atan2(d[1], d[0])
    y = sph_harm_y(l, abs(m), th, ph)
    if m == 0:
        return float(y.real)
    sgn = (-1.0) ** abs(m)
    return float(math.sqrt(2.0) * sgn * (y.real if m > 0 else y.imag))


def rot_from_wxyz(q):
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


# ------------------------------------------------------------------------------------
# Spherical harmonics colour (the Gaussians' colour attribute, Section 3.1)
# ------------------------------------------------------------------------------------

def test_real_sh_matches_scipy(orc):
    rng = np.random.default_rng(3)
    for _ in range(16):
        d = rng.standard_normal(3)
        for l in range(4):
            for m in range(-l, l + 1):
                assert orc.real_sh(l, m, d) == pytest.approx(scipy_real_sh(l, m, d), abs=1e-12)


def test_sh_degree0_returns_rgb(orc):
    rng = np.random.default_rng(4)
    for _ in range(8):
        rgb = rng.uniform(0, 1, 3)
        coeff = np.float32((rgb - 0.5) / Y00)
        out = orc.sh_colour(0, coeff, rng.standard_normal(3))
        assert np.allclose(out, coeff.astype(np.float64) * Y00 + 0.5, atol=1e-12)
        assert np.allclose(out, rgb, atol=1e-6)


def test_sh_single_basis_function_and_layout(orc):
    """Coefficient plane k*3+c holds basis k = l^2+l+m of channel c."""
    rng = np.random.default_rng(5)
    d = rng.standard_normal(3)
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            for c in range(3):
                coeffs = np.zeros((16, 3), np.float32)
                coeffs[k, c] = 0.25
                out = orc.sh_colour(3, coeffs.reshape(-1), d)
                exp = np.full(3, 0.5)
                exp[c] = max(0.0, 0.5 + 0.25 * scipy_real_sh(l, m, d))
                assert np.allclose(out, exp, atol=1e-12), (l, m, c)


def test_sh_clamps_negative_colour(orc):
    coeffs = np.array([-5.0, 0.0, 1.0], np.float32)
    out = orc.sh_colour(0, coeffs, [0, 0, 1])
    assert out[0] == 0.0 and out[1] == 0.5 and out[2] == pytest.approx(0.5 + Y00, abs=1e-7)


# ------------------------------------------------------------------------------------
# Projection (Section 3.4, Eq. 9-10; conventions of the 3DGS rasterizer)
# ------------------------------------------------------------------------------------

def test_projection_on_axis_rotated_anisotropic(orc):
    """On the optical axis J = diag(f/z) on x, y, so Sigma2 = (f/z)^2 V[:2,:2] + 0.3 I,
    with V = R S^2 R^T built from scipy's rotation of the same quaternion."""
    cam = axis_camera(64, 64, f=80.0)
    rng = np.random.default_rng(6)
    for _ in range(6):
        q = rng.standard_normal(4)
        sig = rng.uniform(0.01, 0.05, 3)
        z = 2.5
        sc = make_scene([[0, 0, z]], [sig], quats=[q])
        pre = orc.preprocess(sc, cam, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
        Rm = rot_from_wxyz(np.float32(q))
        s32 = np.exp(np.log(sig).astype(np.float32).astype(np.float64))
        V = Rm @ np.diag(s32 ** 2) @ Rm.T
        exp = (80.0 / z) ** 2 * V[:2, :2] + 0.3 * np.eye(2)
        a, b, c = pre["cov2d"][0]
        assert np.allclose([a, b, c], [exp[0, 0], exp[0, 1], exp[1, 1]], rtol=1e-9, atol=1e-12)
        inv = np.linalg.inv(exp)
        assert np.allclose(pre["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-9)
        assert np.allclose(pre["mean2d"][0], [32.0, 32.0])
        assert pre["depth"][0] == pytest.approx(z)


def test_projection_off_axis_and_jacobian_clamp(orc):
    """Isotropic Gaussian at (X, Y, Z): Sigma2 = s^2 (f/Z)^2 [[1+x^2, xy],[xy, 1+y^2]] + 0.3 I
    with x = X/Z, y = Y/Z clamped to 1.3 tan(half FOV) inside J only."""
    W, H, f = 64, 48, 40.0
    cam = axis_camera(W, H, f=f)
    limx, limy = 1.3 * (W / 2) / f, 1.3 * (H / 2) / f
    s = 0.02
    for X, Y, Z in [(0.3, -0.2, 2.0), (0.9, 0.1, 1.0), (-3.0, 0.5, 1.5), (0.1, 2.5, 1.0)]:
        sc = make_scene([[X, Y, Z]], [[s, s, s]])
        pre = orc.preprocess(sc, cam, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
        X32, Y32, Z32 = (float(np.float32(v)) for v in (X, Y, Z))
        s32 = float(np.exp(np.float64(np.float32(math.log(s)))))
        x = min(limx, max(-limx, X32 / Z32))
        y = min(limy, max(-limy, Y32 / Z32))
        k = s32 ** 2 * (f / Z32) ** 2
        exp = [k * (1 + x * x) + 0.3, k * x * y, k * (1 + y * y) + 0.3]
        assert np.allclose(pre["cov2d"][0], exp, rtol=1e-9)
        assert np.allclose(pre["mean2d"][0], [f * X32 / Z32 + W / 2, f * Y32 / Z32 + H / 2], rtol=1e-12)


def test_projection_look_at_camera_axes(orc):
    """Camera at (3,0,0) looking at the origin with world -y up: world +z maps to image
    right (x = fwd cross up), world +y to image down."""
    cam = scenes.look_at_camera((3.0, 0.0, 0.0), (0.0, 0.0, 0.0), 64, 64, 60.0)
    f = float(np.float32(cam.fx))
    sc = make_scene([[0, 0, 0], [0, 0.3, 0], [0, 0, 0.3]], [[0.01] * 3] * 3)
    pre = orc.preprocess(sc, cam, plane([1, 0, 0], 1e20, scenes.MODE_NONE))
    assert np.allclose(pre["depth"], 3.0, atol=1e-6)
    assert np.allclose(pre["mean2d"][0], [32, 32], atol=1e-6)
    assert np.allclose(pre["mean2d"][1], [32, 32 + f * np.float32(0.3) / 3.0], atol=1e-5)
    assert np.allclose(pre["mean2d"][2], [32 + f * np.float32(0.3) / 3.0, 32], atol=1e-5)


def test_near_cull_rect_tiles_opacity(orc):
    cam = axis_camera(64, 64, f=64.0)
    s = 0.02
    sc = make_scene([[0, 0, 0.19], [0, 0, 0.21], [0, 0, 2.0], [100.0, 0, 2.0]], [[s] * 3] * 4,
                    opacity=[0.3, 0.4, 0.7, 0.5])
    pre = orc.preprocess(sc, cam, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
    assert list(pre["culled"]) == [1, 0, 0, 1]
    s32 = float(np.exp(np.float64(np.float32(math.log(s)))))
    var = (64.0 * s32 / 2.0) ** 2 + 0.3
    h = 3.0 * math.sqrt(var)
    lo, hi = math.floor((32 - h) / 16), math.floor((32 + h) / 16)
    assert list(pre["rect"][2]) == [lo, lo, hi, hi]
    assert pre["tiles"][2] == (hi - lo + 1) ** 2
    assert pre["tiles"][3] == 0
    logit = float(np.float32(math.log(0.7 / 0.3)))
    assert pre["opacity"][2] == pytest.approx(1 / (1 + math.exp(-logit)), abs=1e-15)


def test_colour_direction_is_centre_minus_eye(orc):
    """SH is evaluated at normalize(mu - e): a Y_{1,1} (x) coefficient brightens a Gaussian
    to the right of an axis camera and darkens one to the left."""
    cam = axis_camera(64, 64, f=64.0)
    sh = np.zeros((12, 2))
    sh[3 * 3 + 0, :] = 0.5          # basis k = 3 (l=1, m=1), channel R
    sc = make_scene([[0.4, 0, 2.0], [-0.4, 0, 2.0]], [[0.01] * 3] * 2, sh=sh, sh_degree=1)
    pre = orc.preprocess(sc, cam, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
    x = np.float32(0.4) / math.hypot(np.float32(0.4), 2.0)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert pre["rgb"][0][0] == pytest.approx(0.5 + 0.5 * c1 * x, abs=1e-7)
    assert pre["rgb"][1][0] == pytest.approx(0.5 - 0.5 * c1 * x, abs=1e-7)


# ------------------------------------------------------------------------------------
# Classification (Section 3.2; Algorithm 1 step 1)
# ------------------------------------------------------------------------------------

def test_classification_thresholds_all_modes(orc):
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 64, 64)
    sig = [0.01, 0.02, 0.015]
    s32 = np.exp(np.log(np.array(sig)).astype(np.float32).astype(np.float64))
    r = 3 * s32.max()
    eps = 1e-4
    zs = [-r - eps, -r + eps, -0.5 * r, 0.0, 0.5 * r, r - eps, r + eps, 5 * r, -5 * r]
    rng = np.random.default_rng(8)
    sc = make_scene([[0.1, 0.1, z] for z in zs], [sig] * len(zs), quats=rng.standard_normal((len(zs), 4)))
    exp = {
        scenes.MODE_RARA: [0, 2, 2, 2, 2, 2, 1, 1, 0],
        scenes.MODE_RARA_ALL: [0, 2, 2, 2, 2, 2, 2, 2, 0],
        scenes.MODE_HARD: [0, 0, 0, 1, 1, 1, 1, 1, 0],
        scenes.MODE_NONE: [1] * 9,
    }
    for mode, lab in exp.items():
        pre = orc.preprocess(sc, cam, plane([0, 0, 1], 0.0, mode))
        assert list(pre["label"]) == lab, mode
        assert np.allclose(pre["radius"], r)
        assert np.allclose(pre["d_ep"], np.float32(zs), atol=1e-12)


# ------------------------------------------------------------------------------------
# Ray-ellipsoid chord and decay weight (Eq. 4-8, Eq. 11, Algorithm 1 step 2)
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("k", [3.0, 1.0])
def test_weight_sphere_closed_form(orc, k):
    """Sphere of radius R = k sigma, ray along +z at lateral offset b from (b, 0, -D):
    chord [D - h, D + h] with h = sqrt(R^2 - b^2); plane z = s (visible z >= s) keeps the
    fraction (h - s) / (2h) of it."""
    R, D = 0.2, 3.0
    sig = [R / k] * 3
    q = [0.3, -0.4, 0.5, 0.7]
    for b in [0.0, 0.3 * R, 0.9 * R]:
        h = math.sqrt(R * R - b * b)
        for s in [-1.2 * h, -0.5 * h, 0.0, 0.3 * h, 0.99 * h, 1.5 * h]:
            w, (t1, t2, tp) = orc.rara_weight([b, 0, -D], [0, 0, 1], [0, 0, 0], q, sig, k, [0, 0, 1], -s)
            assert w == pytest.approx(min(1.0, max(0.0, (h - s) / (2 * h))), abs=1e-12)
            assert t1 == pytest.approx(D - h, abs=1e-12) and t2 == pytest.approx(D + h, abs=1e-12)
            assert t2 - t1 == pytest.approx(2 * math.sqrt(R * R - b * b), abs=1e-12)
            assert tp == pytest.approx(D + s, abs=1e-12)
            # flipped normal: visible side is z <= s
            w2, _ = orc.rara_weight([b, 0, -D], [0, 0, 1], [0, 0, 0], q, sig, k, [0, 0, -1], s)
            assert w2 == pytest.approx(min(1.0, max(0.0, (h + s) / (2 * h))), abs=1e-12)


def test_weight_axis_aligned_ellipsoid(orc):
    ax, ay, az = 0.3, 0.15, 0.45   # semi-axes = 3 sigma
    for x0, y0 in [(0.0, 0.0), (0.1, 0.05), (-0.2, 0.1)]:
        h = az * math.sqrt(1 - (x0 / ax) ** 2 - (y0 / ay) ** 2)
        for s in [-0.3 * h, 0.2 * h, 0.8 * h]:
            w, (t1, t2, _) = orc.rara_weight([x0, y0, -4.0], [0, 0, 2.0], [0, 0, 0], [1, 0, 0, 0],
                                             [ax / 3, ay / 3, az / 3], 3.0, [0, 0, 1], -s)
            assert t2 - t1 == pytest.approx(2 * h, abs=1e-12)
            assert w == pytest.approx((h - s) / (2 * h), abs=1e-12)


def test_weight_brute_force_chord_sampling(orc):
    """Rotated anisotropic ellipsoids: w equals the visible fraction of chord samples found
    by marching the ray and testing (x-mu)^T V^-1 (x-mu) <= k^2 with V from scipy."""
    rng = np.random.default_rng(9)
    checked = 0
    for _ in range(40):
        q = rng.standard_normal(4)
        sig = rng.uniform(0.02, 0.12, 3)
        k = 3.0
        mu = rng.uniform(-0.2, 0.2, 3)
        e = np.array([0.1, -0.2, -3.0])
        target = mu + rng.normal(0, 0.08, 3)
        d = (target - e) / np.linalg.norm(target - e)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        dpl = -(n @ (mu + rng.normal(0, 0.1, 3)))
        w, (t1, t2, tp) = orc.rara_weight(e, d, mu, q, sig, k, n, dpl)
        Rm = rot_from_wxyz(q)
        Vinv = Rm @ np.diag(1 / sig ** 2) @ Rm.T
        ts = np.linspace(0.0, 6.0, 400_001)
        x = e[None, :] + ts[:, None] * d[None, :]
        dx = x - mu
        inside = np.einsum("ij,jk,ik->i", dx, Vinv, dx) <= k * k
        if inside.sum() < 2000:
            continue
        vis = x @ n + dpl >= 0
        wbf = (inside & vis).sum() / inside.sum()
        assert w == pytest.approx(wbf, abs=2e-3)
        assert (t2 - t1) == pytest.approx(inside.sum() * (ts[1] - ts[0]), rel=2e-3)
        checked += 1
    assert checked >= 15


def test_weight_degenerate_cases(orc):
    sig = [0.05, 0.05, 0.05]
    q = [1, 0, 0, 0]
    # miss: one intersection or none -> keep rasterization (w = 1)
    assert orc.rara_weight([0.5, 0, -3], [0, 0, 1], [0, 0, 0], q, sig, 3, [0, 0, 1], 0)[0] == 1.0
    # camera inside the ellipsoid -> w = 1 (t1 <= 0)
    assert orc.rara_weight([0, 0, 0.01], [0, 0, 1], [0, 0, 0], q, sig, 3, [0, 0, 1], 0)[0] == 1.0
    # ellipsoid behind the camera -> w = 1
    assert orc.rara_weight([0, 0, 3], [0, 0, 1], [0, 0, 0], q, sig, 3, [0, 0, 1], 0)[0] == 1.0
    # ray parallel to the plane, chord entirely visible / invisible
    assert orc.rara_weight([0, 0, -3], [0, 0, 1], [0, 0, 0], q, sig, 3, [1, 0, 0], 0.01)[0] == 1.0
    assert orc.rara_weight([0, 0, -3], [0, 0, 1], [0, 0, 0], q, sig, 3, [1, 0, 0], -0.01)[0] == 0.0
    # plane behind the camera, chord all on the invisible side: Eq. 11 gives w = 0
    assert orc.rara_weight([0, 0, -3], [0, 0, 1], [0, 0, 0], q, sig, 3, [0, 0, -1], -5.0)[0] == 0.0


def test_weight_monotone_in_plane_offset(orc):
    rng = np.random.default_rng(10)
    for _ in range(20):
        q = rng.standard_normal(4)
        sig = rng.uniform(0.02, 0.1, 3)
        mu = rng.uniform(-0.1, 0.1, 3)
        e = np.array([0.0, 0.0, -3.0])
        d = mu + rng.normal(0, 0.05, 3) - e
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        ws = [orc.rara_weight(e, d, mu, q, sig, 3.0, n, dd)[0] for dd in np.linspace(-1, 1, 81)]
        assert all(b >= a - 1e-12 for a, b in zip(ws, ws[1:]))
        assert ws[0] in (0.0, 1.0) and ws[-1] == 1.0


# ------------------------------------------------------------------------------------
# Compositing (Eq. 2, Eq. 10, Eq. 12, Algorithm 1 step 3)
# ------------------------------------------------------------------------------------

F = 64.0


def _at_pixel(px, py, z):
    """World point on the axis camera (f = 64, 64x64) that projects to pixel centre (px+.5, py+.5)."""
    return [(px + 0.5 - 32) * z / F, (py + 0.5 - 32) * z / F, z]


def _f32sig(p):
    return 1.0 / (1.0 + math.exp(-float(np.float32(math.log(p / (1 - p))))))


def _f32rgb(v):
    return float(np.float32((v - 0.5) / Y00)) * Y00 + 0.5


def _render(orc, sc, pl, bg=(0, 0, 0), cam=None, brute=False):
    cam = cam or axis_camera(64, 64, F)
    return orc.render_frame(sc, cam, pl, bg=bg, brute=brute, threads=2)


def test_single_gaussian_blend(orc):
    z = 2.0
    sc = make_scene([_at_pixel(40, 20, z)], [[0.01] * 3], opacity=[0.6], rgb=[[0.2, 0.7, 0.9]])
    bg = (0.1, 0.2, 0.3)
    pre, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE), bg)
    a = min(0.99, _f32sig(0.6))
    for c, v in enumerate([0.2, 0.7, 0.9]):
        assert out["image"][c, 20, 40] == pytest.approx(_f32rgb(v) * a + (1 - a) * bg[c], abs=1e-12)
    assert out["T"][20, 40] == pytest.approx(1 - a, abs=1e-12)
    assert out["n_contrib"][20, 40] == 1


def test_two_gaussians_front_to_back_by_depth(orc):
    # index 0 is behind index 1: order is by depth, not by index
    sc = make_scene([_at_pixel(10, 10, 3.0), _at_pixel(10, 10, 2.0)], [[0.01] * 3] * 2,
                    opacity=[0.5, 0.4], rgb=[[1, 0, 0], [0, 0, 1]])
    bg = (0.0, 1.0, 0.0)
    _, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE), bg)
    af, ab = _f32sig(0.4), _f32sig(0.5)
    cf = np.array([_f32rgb(0), _f32rgb(0), _f32rgb(1)])
    cb = np.array([_f32rgb(1), _f32rgb(0), _f32rgb(0)])
    exp = cf * af + cb * ab * (1 - af) + np.array(bg) * (1 - af) * (1 - ab)
    assert np.allclose(out["image"][:, 10, 10], exp, atol=1e-12)


def test_early_termination_and_clamp(orc):
    # three stacked Gaussians of alpha 0.96: T = 0.04, 1.6e-3, then 6.4e-5 < 1e-4 stops
    # before the third is blended (a 1e-5 stop would blend it)
    p = 0.96
    sc = make_scene([_at_pixel(5, 5, z) for z in (2.0, 2.5, 3.0)], [[0.01] * 3] * 3, opacity=[p] * 3,
                    rgb=[[1, 1, 1]] * 3)
    _, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
    a = _f32sig(p)
    assert out["n_contrib"][5, 5] == 2
    assert out["T"][5, 5] == pytest.approx((1 - a) ** 2, rel=1e-12)
    assert out["image"][0, 5, 5] == pytest.approx(_f32rgb(1) * (a + a * (1 - a)), abs=1e-12)
    # the 0.99 clamp of Algorithm 1 step 3
    sc = make_scene([_at_pixel(5, 5, 2.0)], [[0.01] * 3], opacity=[0.9999])
    _, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
    assert out["T"][5, 5] == pytest.approx(0.01, abs=1e-12)


def test_anisotropic_footprint_alpha(orc):
    """alpha at pixel offsets D from an on-axis rotated anisotropic splat equals
    delta exp(-D^T Sigma2^-1 D / 2), with Sigma2 = (f/z)^2 V[:2,:2] + 0.3 I from scipy's
    rotation and numpy's inverse."""
    rng = np.random.default_rng(13)
    z = 2.0
    for _ in range(3):
        q = rng.standard_normal(4)
        sig = np.array([0.08, 0.012, 0.03])
        sc = make_scene([[0.0, 0.0, z]], [sig], quats=[q], opacity=[0.7])
        _, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
        Rm = rot_from_wxyz(np.float32(q))
        s32 = np.exp(np.log(sig).astype(np.float32).astype(np.float64))
        V = Rm @ np.diag(s32 ** 2) @ Rm.T
        S2 = (F / z) ** 2 * V[:2, :2] + 0.3 * np.eye(2)
        Si = np.linalg.inv(S2)
        delta = _f32sig(0.7)
        seen = 0
        for py in range(20, 45):
            for px in range(20, 45):
                D = np.array([px + 0.5 - 32.0, py + 0.5 - 32.0])
                qv = D @ Si @ D
                a = delta * math.exp(-0.5 * qv)
                if qv > 8.9 or a < 1.2 / 255:
                    continue
                assert out["T"][py, px] == pytest.approx(1.0 - a, abs=1e-9)
                seen += 1
        assert seen > 30


def test_alpha_skip_threshold(orc):
    for p, hit in [(0.0035, False), (0.0045, True)]:
        sc = make_scene([_at_pixel(5, 5, 2.0)], [[0.01] * 3], opacity=[p])
        _, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
        assert (out["T"][5, 5] < 1.0) == hit


def test_support_bound_q9(orc):
    """A pixel 3 px right of the centre of an isotropic splat has q = 9 c / (a c - b^2) with
    the off-axis closed form of Sigma2 (see test_projection_off_axis_and_jacobian_clamp);
    sigma is solved so that q lands just outside / inside the 3-sigma support."""
    z = 2.0
    mu = _at_pixel(20, 20, z)
    x, y = mu[0] / z, mu[1] / z

    def q_of(kk):
        a, b, c = kk * (1 + x * x) + 0.3, kk * x * y, kk * (1 + y * y) + 0.3
        return 9.0 * c / (a * c - b * b)

    for qtarget, hit in [(9.02, False), (8.98, True)]:
        lo, hi = 1e-6, 100.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if q_of(mid) > qtarget else (lo, mid)
        sigma = math.sqrt(lo) * z / F
        sc = make_scene([mu], [[sigma] * 3], opacity=[0.99])
        pre, _, out = _render(orc, sc, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
        assert (out["T"][20, 23] < 1.0) == hit
        assert out["T"][20, 22] < 1.0


def _unproject(cam, px, py, depth):
    """World point at camera depth `depth` on the ray through pixel centre (px+.5, py+.5)."""
    Rw = cam.world_to_cam[:, :3].astype(np.float64)
    t = cam.world_to_cam[:, 3].astype(np.float64)
    xc = np.array([(px + 0.5 - cam.cx) / cam.fx * depth, (py + 0.5 - cam.cy) / cam.fy * depth, depth])
    return Rw.T @ (xc - t)


def test_ray_through_pixel_centre_hits_projected_centre(orc):
    """The pixel ray (Algorithm 1 ProjectRay / CameraOrigin) through the pixel where the centre
    projects passes through mu, so a tilted plane through mu halves the chord:
    alpha = delta / 2. A translated, rotated camera pins the camera origin e = -R^T t."""
    rng = np.random.default_rng(11)
    cams = [axis_camera(64, 64, F),
            scenes.look_at_camera((0.7, -0.4, -2.6), (0.1, 0.05, 0.2), 64, 64, 50.0)]
    for cam in cams:
        for _ in range(4):
            px, py = int(rng.integers(8, 56)), int(rng.integers(8, 56))
            mu = np.float32(_unproject(cam, px, py, 2.0)).astype(np.float64)
            n = rng.standard_normal(3)
            n /= np.linalg.norm(n)
            sc = make_scene([mu], [rng.uniform(0.02, 0.05, 3)], quats=[rng.standard_normal(4)], opacity=[0.5])
            n32 = np.float32(n).astype(np.float64)
            pl = plane(n, float(-(n32 @ mu)))
            pre, _, out = _render(orc, sc, pl, cam=cam)
            assert pre["label"][0] == 2
            a = _f32sig(0.5) * 0.5
            assert out["T"][py, px] == pytest.approx(1 - a, abs=2e-4)


def test_colour_direction_translated_camera(orc):
    """normalize(mu - e) with e = -R^T t for a translated camera: a Y_{1,0} (z) coefficient."""
    cam = scenes.look_at_camera((0.5, -0.3, -3.0), (0.0, 0.0, 0.0), 64, 64, 60.0)
    sh = np.zeros((12, 1))
    sh[2 * 3 + 1, 0] = 0.5          # basis k = 2 (l=1, m=0), channel G
    mu = np.array([0.1, 0.2, 0.3])
    sc = make_scene([mu], [[0.01] * 3], sh=sh, sh_degree=1)
    pre = orc.preprocess(sc, cam, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
    eye = np.array([0.5, -0.3, -3.0])
    d = np.float32(mu).astype(np.float64) - eye
    d /= np.linalg.norm(d)
    assert pre["rgb"][0][1] == pytest.approx(0.5 + 0.5 * math.sqrt(3 / (4 * math.pi)) * d[2], abs=1e-6)


def _tiny_random_scene(seed, n=64):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.6, 0.6, (n, 3))
    means[:, 2] += 2.5
    sig = np.exp(rng.normal(-2.8, 0.4, (n, 3)))
    return make_scene(means, sig, quats=rng.standard_normal((n, 4)), opacity=rng.uniform(0.05, 0.95, n),
                      rgb=rng.uniform(0, 1, (n, 3)))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_equals_binned(orc, seed):
    sc = _tiny_random_scene(seed)
    cam = axis_camera(32, 32, 32.0)
    rng = np.random.default_rng(100 + seed)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    for mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL, scenes.MODE_HARD, scenes.MODE_NONE):
        pl = plane(n, -float(n @ [0, 0, 2.5]), mode)
        pre = orc.preprocess(sc, cam, pl)
        if mode == scenes.MODE_RARA:
            assert (pre["label"] == 2).sum() > 0
        kvr = orc.build_keys(pre)
        a = orc.render(sc, pre, cam, pl, (0.1, 0.2, 0.3), kvr, threads=2)
        b = orc.render(sc, pre, cam, pl, (0.1, 0.2, 0.3), None, threads=2)
        assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["T"], b["T"])


def test_plane_at_infinity_is_unclipped(orc):
    """Section 4.3 / Table 2: with the plane at infinity RaRa reproduces the unclipped render
    exactly (L1 = 0, SSIM = 1); so does applying the weight to every Gaussian."""
    with open(os.path.join(GOLDEN, "table2_plane_at_infinity.json")) as fh:
        gold = json.load(fh)
    sc, cam, _ = scenes.small_uniform_workload(n=2000, width=64, height=64, seed=3)
    nrm = scenes.random_unit_normal(5)
    ref = orc.render_frame(sc, cam, plane(nrm, 1e20, scenes.MODE_NONE), bg=(0.1, 0.1, 0.1))[2]["image"]
    for mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL):
        img = orc.render_frame(sc, cam, plane(nrm, 1e20, mode), bg=(0.1, 0.1, 0.1))[2]["image"]
        l1 = float(np.abs(img - ref).mean())
        assert l1 == gold["w_rara"]["L1"]
        assert _ssim(img, ref) == gold["w_rara"]["SSIM"]


def _ssim(a, b, c1=0.01 ** 2, c2=0.03 ** 2):
    from scipy.ndimage import uniform_filter
    vals = []
    for ch in range(a.shape[0]):
        x, y = a[ch], b[ch]
        mx, my = uniform_filter(x, 7), uniform_filter(y, 7)
        sxx = uniform_filter(x * x, 7) - mx * mx
        syy = uniform_filter(y * y, 7) - my * my
        sxy = uniform_filter(x * y, 7) - mx * my
        s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        vals.append(s.mean())
    return float(np.mean(vals))


def test_fully_invisible_scene_is_background(orc):
    sc, cam, _ = scenes.small_uniform_workload(n=2000, width=64, height=64, seed=4)
    bg = (0.2, 0.4, 0.6)
    for mode in (scenes.MODE_RARA, scenes.MODE_RARA_ALL, scenes.MODE_HARD):
        out = orc.render_frame(sc, cam, plane([0.3, 0.5, 0.8], -1e20, mode), bg=bg)[2]
        for c in range(3):
            assert np.all(out["image"][c] == bg[c])
        assert np.all(out["T"] == 1.0)


def test_hard_and_far_planes_equal_unclipped_subset(orc):
    """Hard clipping renders exactly the unclipped image of the Gaussians whose centres are on
    the visible side; RaRa with no cutoff Gaussian does the same."""
    sc, cam, _ = scenes.small_uniform_workload(n=3000, width=64, height=64, seed=5)
    n = np.float32([0.0, 0.6, 0.8]).astype(np.float64)
    keep = (n @ sc.means.astype(np.float64)) >= 0.0
    sub = sc.subset(np.nonzero(keep)[0])
    ref = orc.render_frame(sub, cam, plane(n, 1e20, scenes.MODE_NONE))[2]
    hard = orc.render_frame(sc, cam, plane(n, 0.0, scenes.MODE_HARD))[2]
    assert np.array_equal(ref["image"], hard["image"])


def test_single_gaussian_coverage_monotone_in_offset(orc):
    rng = np.random.default_rng(12)
    cam = axis_camera(32, 32, 32.0)
    for _ in range(3):
        sc = make_scene([[0.0, 0.0, 2.0]], [rng.uniform(0.05, 0.12, 3)], quats=[rng.standard_normal(4)],
                        opacity=[0.9])
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        prev = None
        for dd in np.linspace(-1.0, 1.0, 41):
            cov = 1 - orc.render_frame(sc, cam, plane(n, -(n @ [0, 0, 2.0]) + dd), threads=2)[2]["T"]
            if prev is not None:
                assert np.all(cov >= prev - 1e-12)
            prev = cov


# ------------------------------------------------------------------------------------
# Binning keys (Section 3.1 depth order; tile binning)
# ------------------------------------------------------------------------------------

def test_keys_single_gaussian_by_hand(orc):
    """One isotropic Gaussian: q = |d|^2 / var, so a tile lists it iff the squared distance
    from the centre to the tile's rectangle of pixel centres is at most var q_cut, with
    q_cut = min(9, 2 ln(255 opacity)); the candidates are the tiles of the 3-sigma box."""
    cam = axis_camera(64, 64, 64.0)
    z = 2.0
    for op in (0.5, 0.02):
        sc = make_scene([[0.1, -0.2, z]], [[0.03] * 3], opacity=[op])
        pre = orc.preprocess(sc, cam, plane([0, 0, 1], 1e20, scenes.MODE_NONE))
        keys, vals, ranges = orc.build_keys(pre)
        s32 = float(np.exp(np.float64(np.float32(math.log(0.03)))))
        var = (64 * s32 / z) ** 2 + 0.3
        h = 3 * math.sqrt(var)
        mx = 64 * float(np.float32(0.1)) / z + 32
        my = 64 * float(np.float32(-0.2)) / z + 32
        lg = float(np.float32(math.log(op / (1 - op))))
        qc = min(9.0, 2 * math.log(255 / (1 + math.exp(-lg))))
        tx = range(max(0, math.floor((mx - h) / 16)), min(3, math.floor((mx + h) / 16)) + 1)
        ty = range(max(0, math.floor((my - h) / 16)), min(3, math.floor((my + h) / 16)) + 1)

        def dist2(x, y):
            ddx = max(x * 16 + 0.5 - mx, 0.0, mx - (x * 16 + 15.5))
            ddy = max(y * 16 + 0.5 - my, 0.0, my - (y * 16 + 15.5))
            return ddx * ddx + ddy * ddy

        dbits = int(np.float32(z).view(np.uint32))
        exp = sorted(((y * 4 + x) << 32) | dbits for y in ty for x in tx if dist2(x, y) <= var * qc)
        assert exp
        assert list(keys) == exp and list(vals) == [0] * len(exp)
        for k, key in enumerate(exp):
            t = key >> 32
            assert tuple(ranges[t]) == (k, k + 1)


def _box_min_q_lsq(conic, x0, x1, y0, y1):
    """Smallest q over a box by bounded least squares (scipy): q = |L^T d|^2, conic = L L^T."""
    from scipy.optimize import lsq_linear
    a, b, c = conic
    L = np.linalg.cholesky(np.array([[a, b], [b, c]]))
    r = lsq_linear(L.T, np.zeros(2), bounds=([x0, y0], [x1, y1]), tol=1e-14, method="bvls")
    return float(r.cost * 2.0)


def test_box_min_q_against_bounded_least_squares(orc):
    rng = np.random.default_rng(31)
    for _ in range(300):
        A = rng.standard_normal((2, 2)) * rng.uniform(0.05, 2.0)
        C = A @ A.T + 0.05 * np.eye(2)
        conic = (C[0, 0], C[0, 1], C[1, 1])
        x0, y0 = rng.uniform(-12, 8, 2)
        x1, y1 = x0 + rng.uniform(0, 15), y0 + rng.uniform(0, 15)
        got = orc.box_min_q(conic, x0, x1, y0, y1)
        ref = _box_min_q_lsq(conic, x0, x1, y0, y1)
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-12)
    assert orc.box_min_q((1.0, 0.2, 2.0), -1.0, 3.0, -2.0, 0.5) == 0.0   # centre inside


def _numpy_tile_lists(pre, i, x, y):
    """Tile-listing rule restated in numpy: the minimum of the convex q over the tile's
    pixel-centre rectangle, 0 if it holds the centre, else the smallest edge minimum."""
    a, b, c = pre["conic"][i]
    mx, my = pre["mean2d"][i]
    x0, x1 = x * 16 + 0.5 - mx, min(x * 16 + 16, pre["W"]) - 0.5 - mx
    y0, y1 = y * 16 + 0.5 - my, min(y * 16 + 16, pre["H"]) - 0.5 - my
    if x0 <= 0 <= x1 and y0 <= 0 <= y1:
        m = 0.0
    else:
        cand = []
        for dy in (y0, y1):
            dx = np.clip(-b * dy / a, x0, x1)
            cand.append(a * dx * dx + 2 * b * dx * dy + c * dy * dy)
        for dx in (x0, x1):
            dy = np.clip(-b * dx / c, y0, y1)
            cand.append(a * dx * dx + 2 * b * dx * dy + c * dy * dy)
        m = min(cand)
    return m <= min(9.0, 2 * np.log(255 * pre["opacity"][i]))


def test_keys_match_numpy_stable_sort(orc):
    sc, cam, pl = scenes.small_uniform_workload(n=3000, width=96, height=80, seed=6)
    pre = orc.preprocess(sc, cam, pl)
    keys, vals, ranges = orc.build_keys(pre)
    ek, ev = [], []
    tx = pre["tiles_x"]
    dropped = 0
    for i in range(sc.n):
        if pre["culled"][i]:
            continue
        x0, y0, x1, y1 = pre["rect"][i]
        db = int(np.float32(pre["depth"][i]).view(np.uint32))
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                if not _numpy_tile_lists(pre, i, x, y):
                    dropped += 1
                    continue
                ek.append(((y * tx + x) << 32) | db)
                ev.append(i)
    assert dropped > 0
    ek, ev = np.array(ek, np.uint64), np.array(ev, np.uint32)
    order = np.argsort(ek, kind="stable")
    assert np.array_equal(keys, ek[order]) and np.array_equal(vals, ev[order])
    # ranges partition the list by tile
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t)
    assert (ranges[:, 1] - ranges[:, 0]).sum() == len(keys)


def test_every_blending_pixel_is_in_a_listing_tile(orc):
    """Brute force over pixels: wherever alpha0 = opacity exp(-q/2) >= 1/255 with q <= 9,
    the pixel's tile lists the Gaussian (so the tiles left out cannot change a pixel)."""
    sc, cam, pl = scenes.small_uniform_workload(n=1500, width=80, height=64, seed=8)
    pre = orc.preprocess(sc, cam, pl)
    keys, vals, ranges = orc.build_keys(pre)
    listed = set(zip((keys >> np.uint64(32)).astype(np.int64).tolist(), vals.tolist()))
    ys, xs = np.mgrid[0:64, 0:80]
    checked = 0
    for i in np.nonzero(pre["culled"] == 0)[0]:
        a, b, c = pre["conic"][i]
        dx, dy = xs + 0.5 - pre["mean2d"][i][0], ys + 0.5 - pre["mean2d"][i][1]
        q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        hit = (q <= 9.0) & (pre["opacity"][i] * np.exp(-0.5 * q) >= 1.0 / 255.0)
        for y, x in zip(*np.nonzero(hit)):
            assert ((y // 16) * pre["tiles_x"] + x // 16, int(i)) in listed
            checked += 1
    assert checked > 1000


# ------------------------------------------------------------------------------------
# The class thresholds where the image jumps (Section 3.2, Algorithm 1 step 1, Eq. 11)
# ------------------------------------------------------------------------------------

def _threshold_frames(orc, side, eps, mode=scenes.MODE_RARA):
    """One isotropic Gaussian (sigma 0.01 at depth 2 on the axis camera: 0.32 px, so its
    dilated q <= 9 footprint reaches 1.9 px while the 3-sigma ellipsoid's silhouette is
    0.96 px) and the plane x = -d whose offset puts the centre at d_ep = side * r + eps."""
    mu = _at_pixel(32, 32, 2.0)
    sc = make_scene([mu], [[0.01] * 3], opacity=[0.9], rgb=[[1.0, 1.0, 1.0]])
    r = 3.0 * math.exp(float(np.float32(math.log(0.01))))
    d = float(np.float32(side * r + eps - np.float32(mu[0])))
    pre, _, out = _render(orc, sc, plane([1, 0, 0], d, mode))
    return pre, out, float(np.float32(mu[0])) + d - side * r


@pytest.mark.parametrize("mode", [scenes.MODE_RARA, scenes.MODE_RARA_ALL])
def test_invisible_threshold_is_an_image_jump_and_flagged(orc, mode):
    # Pixel (33, 32) is 1 px from the projected centre: inside the footprint (q = 2.5,
    # alpha0 = 0.26) but its ray misses the ellipsoid, so w = 1 while the Gaussian is
    # cutoff and 0 once it turns invisible at d_ep = -r.
    pre_c, out_c, off_c = _threshold_frames(orc, -1.0, +1e-7, mode)
    pre_i, out_i, off_i = _threshold_frames(orc, -1.0, -1e-7, mode)
    assert 0 < off_c < 1e-6 and -1e-6 < off_i < 0
    assert pre_c["label"][0] == orc.CUTOFF and pre_i["label"][0] == orc.INVISIBLE
    assert out_c["image"][0, 32, 33] > 0.2          # blended with w = 1 just inside
    assert out_i["image"][0, 32, 33] == 0.0         # background just outside
    assert out_c["image"][0, 32, 32] < 1e-3         # the central ray hits: w ~ 0 already
    # the oracle marks the jump: the Gaussian's margin and the footprint's pixels, on both
    # sides (as a candidate when cutoff, as a hazard when invisible)
    for pre, out in ((pre_c, out_c), (pre_i, out_i)):
        assert pre["margin_gauss"][0] <= 1e-6
        assert out["events"][32, 33] & orc.EV_GAUSS
        assert out["events"][32, 31] & orc.EV_GAUSS
        assert out["events"][10, 10] == 0           # far outside the footprint
    # away from the threshold nothing is flagged
    pre_f, out_f, _ = _threshold_frames(orc, -1.0, -1e-3, mode)
    assert pre_f["margin_gauss"][0] > 1e-4 and not (out_f["events"][32, 33] & orc.EV_GAUSS)


def test_visible_threshold_is_continuous(orc):
    # At d_ep = +r (k_sigma = 3) the traced ellipsoid lies inside the radius-r sphere: every
    # chord is visible on both sides of the threshold, so the image does not jump there and
    # the oracle does not flag it.
    pre_c, out_c, _ = _threshold_frames(orc, +1.0, -1e-7)
    pre_v, out_v, _ = _threshold_frames(orc, +1.0, +1e-7)
    assert pre_c["label"][0] == orc.CUTOFF and pre_v["label"][0] == orc.VISIBLE
    assert np.abs(out_c["image"] - out_v["image"]).max() < 1e-5
    assert out_v["image"][0, 32, 32] > 0.5
    assert pre_c["margin_gauss"][0] > 1e-4 and pre_v["margin_gauss"][0] > 1e-4
    assert not (out_c["events"] & orc.EV_GAUSS).any()
