"""FP64 CPU oracle of the RaRa clipped Gaussian-splat render (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the entry-point smoke check and by
the benchmark's CPU-baseline / reference leg. The product path never imports it.
The arithmetic lives in rara_oracle.c (plain C, double precision, no code shared with
the CUDA library); this module only compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rara_oracle.c")
_LIB = os.path.join(_HERE, "liborc_rara.so")
_lib = None

INVISIBLE, VISIBLE, CUTOFF = 0, 1, 2
EV_Q, EV_ALPHA, EV_T, EV_GAUSS, EV_DISC, EV_DEPTH, EV_T1 = 1, 2, 4, 8, 16, 32, 64

# Event tolerances: q relative to 9, alpha relative to 1/255, T relative to 1e-4,
# 1 - b^2 absolute, threshold distance (world units), projected-position error (pixels),
# depth ulps for near-tie flags (0: only identical float32 depths, ordered by index on
# both sides, so never a hazard). They bound the float32 error of the CUDA path.
DEFAULT_TOL = (2e-5, 2e-4, 2e-3, 2e-4, 1e-6, 3e-4, 0)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over pixel rows) into oracle/liborc_rara.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        lib.orc_preprocess.restype = C.c_int
        lib.orc_preprocess.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, C.c_int, C.c_int, P,
                                       C.c_int, C.c_double, C.c_int, C.c_int, C.c_int] + [P] * 15
        lib.orc_count_pairs.restype = C.c_int64
        lib.orc_count_pairs.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_build_keys.restype = C.c_int
        lib.orc_build_keys.argtypes = [C.c_int64, P, P, P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_int,
                                       P, P, P]
        lib.orc_box_min_q.restype = C.c_double
        lib.orc_box_min_q.argtypes = [C.c_double] * 7
        lib.orc_render.restype = C.c_int
        lib.orc_render.argtypes = ([C.c_int64, P, P, P, P, P, P, P, P, P, P, P, P, C.c_int, C.c_int,
                                    P, C.c_int, C.c_double, C.c_int, C.c_int, P, P, P, P, P, C.c_int,
                                    C.c_int, C.c_int, P, P, P, P])
        lib.orc_rara_weight.restype = C.c_double
        lib.orc_rara_weight.argtypes = [P, P, P, P, P, C.c_double, P, P]
        lib.orc_rara_weight_vol.restype = C.c_double
        lib.orc_rara_weight_vol.argtypes = [P, P, P, P, P, C.c_double, P, C.c_int]
        lib.orc_sh_colour.restype = None
        lib.orc_sh_colour.argtypes = [C.c_int, P, P, P]
        lib.orc_real_sh.restype = C.c_double
        lib.orc_real_sh.argtypes = [C.c_int, C.c_int, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    """Gaussian parameters as double: float32 arrays widen exactly, float64 arrays (finite-
    difference perturbations) are passed through unrounded."""
    a = np.asarray(a)
    if a.dtype != np.float64:
        a = np.asarray(a, np.float32).astype(np.float64)
    return np.ascontiguousarray(a)


def cam16(cam) -> np.ndarray:
    w2c = np.asarray(cam.world_to_cam, np.float32).astype(np.float64)
    return np.ascontiguousarray(np.concatenate([w2c[:, :3].reshape(-1), w2c[:, 3],
                                                [np.float32(cam.fx), np.float32(cam.fy),
                                                 np.float32(cam.cx), np.float32(cam.cy)]]).astype(np.float64))


def plane4(plane) -> np.ndarray:
    """The clip planes (n, d), four doubles each: the plane's own, then its extra planes
    (plane.extra, rows (nx, ny, nz, d)) of a convex clip volume. As the GPU receives them
    (float32), or unrounded when the plane carries an attribute exact=True (finite-difference
    perturbations of the plane)."""
    rows = [list(np.asarray(plane.n).reshape(3)) + [plane.d]]
    rows += [list(np.asarray(e).reshape(4)) for e in getattr(plane, "extra", ())]
    a = np.asarray(rows, np.float64)
    if not getattr(plane, "exact", False):
        a = np.asarray(rows, np.float32).astype(np.float64)
    return np.ascontiguousarray(a.reshape(-1))


def preprocess(scene, cam, plane, tile=(16, 16)) -> dict:
    lib = _load()
    n = scene.n
    out = dict(
        label=np.zeros(n, np.uint8), culled=np.zeros(n, np.uint8), depth=np.zeros(n),
        mean2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)),
        rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32), rgb=np.zeros((n, 3)),
        opacity=np.zeros(n), d_ep=np.zeros(n), radius=np.zeros(n), margin_class=np.zeros(n),
        margin_gauss=np.zeros(n), margin_rect=np.zeros(n))
    sc = [_f64(scene.means), _f64(scene.log_scales), _f64(scene.quats),
          _f64(scene.opacity_logits), _f64(scene.sh)]
    c16, p4 = cam16(cam), plane4(plane)
    rc = lib.orc_preprocess(n, *[_p(a) for a in sc], int(scene.sh_degree), _p(c16),
                            int(cam.width), int(cam.height), _p(p4), p4.size // 4,
                            float(np.float32(plane.k_sigma)),
                            int(plane.mode), int(tile[0]), int(tile[1]),
                            *[_p(out[k]) for k in ("label", "culled", "depth", "mean2d", "cov2d",
                                                   "conic", "rect", "tiles", "rgb", "opacity",
                                                   "d_ep", "radius", "margin_class", "margin_gauss",
                                                   "margin_rect")])
    assert rc == 0
    out["W"], out["H"] = int(cam.width), int(cam.height)
    out["tiles_x"] = (cam.width + tile[0] - 1) // tile[0]
    out["tiles_y"] = (cam.height + tile[1] - 1) // tile[1]
    out["tile"] = tuple(tile)
    return out


def build_keys(pre: dict):
    """Sorted (key, value) pairs and per-tile [start, end) ranges (see orc_build_keys)."""
    lib = _load()
    n = pre["label"].shape[0]
    geo = (_p(pre["rect"]), _p(pre["mean2d"]), _p(pre["conic"]), _p(pre["opacity"]),
           pre["W"], pre["H"], pre["tile"][0], pre["tile"][1])
    p = int(lib.orc_count_pairs(n, _p(pre["culled"]), *geo))
    keys = np.zeros(max(p, 1), np.uint64)
    vals = np.zeros(max(p, 1), np.uint32)
    nt = pre["tiles_x"] * pre["tiles_y"]
    ranges = np.zeros((nt, 2), np.int64)
    rc = lib.orc_build_keys(n, _p(pre["culled"]), _p(pre["rect"]), _p(pre["depth"]), *geo[1:],
                            _p(keys), _p(vals), _p(ranges))
    assert rc == 0
    return keys[:p], vals[:p], ranges


def box_min_q(conic, x0, x1, y0, y1) -> float:
    """Smallest q over the box [x0, x1] x [y0, y1] of offsets (see orc_box_min_q)."""
    a, b, c = (float(v) for v in conic)
    return float(_load().orc_box_min_q(a, b, c, float(x0), float(x1), float(y0), float(y1)))


def tile_margin(pre: dict, i: int, t: int) -> float:
    """|smallest q over tile t's pixel-centre rectangle - q_cut| for Gaussian i: how close the
    tile-listing decision of orc_build_keys is to its threshold."""
    tw, th = pre["tile"]
    tx, ty = t % pre["tiles_x"], t // pre["tiles_x"]
    mx, my = pre["mean2d"][i]
    x0, x1 = tx * tw + 0.5 - mx, min((tx + 1) * tw, pre["W"]) - 0.5 - mx
    y0, y1 = ty * th + 0.5 - my, min((ty + 1) * th, pre["H"]) - 0.5 - my
    qc = min(9.0, 2.0 * np.log(255.0 * pre["opacity"][i]))
    return abs(box_min_q(pre["conic"][i], x0, x1, y0, y1) - qc)


def render(scene, pre: dict, cam, plane, bg=(0.0, 0.0, 0.0), binned=None, tol=DEFAULT_TOL,
           threads: int | None = None, rows=None):
    """Render with the oracle. binned=(keys, vals, ranges) walks tile lists; None = brute force.
    rows=(begin, end) renders only that band of rows (the rest of the outputs stay zero).

    Returns dict(image [3,H,W], T [H,W], n_contrib [H,W] int32, events [H,W] uint8).
    """
    lib = _load()
    n = scene.n
    H, W = int(cam.height), int(cam.width)
    image = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    ev = np.zeros((H, W), np.uint8)
    sc = [_f64(scene.means), _f64(scene.log_scales), _f64(scene.quats)]
    c16, p4 = cam16(cam), plane4(plane)
    bgv = np.asarray(bg, np.float64).copy()
    tolv = np.asarray(tol, np.float64).copy()
    if binned is not None:
        keys, vals, ranges = (np.ascontiguousarray(x) for x in binned)
        kp, vp, rp = _p(keys if keys.size else np.zeros(1, np.uint64)), \
            _p(vals if vals.size else np.zeros(1, np.uint32)), _p(ranges)
    else:
        kp = vp = rp = None
    threads = threads or (os.cpu_count() or 1)
    rc = lib.orc_render(n, *[_p(a) for a in sc], _p(pre["label"]), _p(pre["culled"]),
                        _p(pre["depth"]), _p(pre["mean2d"]), _p(pre["conic"]), _p(pre["rgb"]),
                        _p(pre["opacity"]), _p(pre["margin_gauss"]), _p(c16), W, H, _p(p4), p4.size // 4,
                        float(np.float32(plane.k_sigma)), pre["tile"][0], pre["tile"][1], _p(bgv),
                        kp, vp, rp, _p(tolv), int(threads), int(rows[0] if rows else 0),
                        int(rows[1] if rows else H), _p(image), _p(T), _p(nc), _p(ev))
    assert rc == 0
    return dict(image=image, T=T, n_contrib=nc, events=ev)


def render_frame(scene, cam, plane, bg=(0.0, 0.0, 0.0), tile=(16, 16), brute=False, threads=None):
    """Preprocess + keys + render in one call; returns (pre, (keys, vals, ranges), out)."""
    pre = preprocess(scene, cam, plane, tile)
    kvr = build_keys(pre)
    out = render(scene, pre, cam, plane, bg, None if brute else kvr, threads=threads)
    return pre, kvr, out


def rara_weight(e, d, mu, quat, sigma, k_sigma, plane_n, plane_d):
    """Decay weight w (Eq. 11) for the ray e + t d against the ellipsoid k R S.

    Returns (w, (t1, t2, tp)); the t's are NaN unless two intersections lie in front."""
    lib = _load()
    arrs = [np.ascontiguousarray(np.asarray(x, np.float64)) for x in (e, d, mu, quat, sigma)]
    p4 = np.array(list(np.asarray(plane_n, np.float64)) + [float(plane_d)], np.float64)
    tout = np.zeros(3)
    w = lib.orc_rara_weight(*[_p(a) for a in arrs], float(k_sigma), _p(p4), _p(tout))
    return float(w), tuple(float(x) for x in tout)


def rara_weight_volume(e, d, mu, quat, sigma, k_sigma, planes):
    """Decay weight against the convex clip volume of `planes` (rows (nx, ny, nz, d)): the
    share of the chord of the ray e + t d through the ellipsoid k R S that lies on the
    visible side of every plane (1 when the ray meets the ellipsoid fewer than twice in
    front)."""
    lib = _load()
    arrs = [np.ascontiguousarray(np.asarray(x, np.float64)) for x in (e, d, mu, quat, sigma)]
    pl = np.ascontiguousarray(np.asarray(planes, np.float64).reshape(-1))
    return float(lib.orc_rara_weight_vol(*[_p(a) for a in arrs], float(k_sigma), _p(pl), pl.size // 4))


def sh_colour(degree: int, coeffs, direction):
    lib = _load()
    cf = _f64(coeffs).reshape(-1)
    assert cf.size == 3 * (degree + 1) ** 2
    d = np.ascontiguousarray(np.asarray(direction, np.float64))
    rgb = np.zeros(3)
    lib.orc_sh_colour(int(degree), _p(cf), _p(d), _p(rgb))
    return rgb


def real_sh(l: int, m: int, direction) -> float:
    lib = _load()
    d = np.ascontiguousarray(np.asarray(direction, np.float64))
    d = d / np.linalg.norm(d)
    return float(lib.orc_real_sh(int(l), int(m), _p(d)))


def support_mask(pre: dict, gauss_idx, H: int, W: int, q_max: float = 9.5) -> np.ndarray:
    """Pixels inside the q <= q_max footprint of the given Gaussians (projection fields of
    the oracle preprocess); used to exclude pixels touched by threshold-straddling Gaussians."""
    mask = np.zeros((H, W), bool)
    for i in np.asarray(gauss_idx).reshape(-1):
        ca, cb, cc = pre["cov2d"][i]
        if ca <= 0 or cc <= 0:
            continue
        mx, my = pre["mean2d"][i]
        hx, hy = 3.2 * np.sqrt(ca), 3.2 * np.sqrt(cc)
        x0, x1 = max(0, int(np.floor(mx - hx))), min(W - 1, int(np.ceil(mx + hx)))
        y0, y1 = max(0, int(np.floor(my - hy))), min(H - 1, int(np.ceil(my + hy)))
        if x0 > x1 or y0 > y1:
            continue
        ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        dx, dy = xs + 0.5 - mx, ys + 0.5 - my
        a, b, c = pre["conic"][i]
        q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        mask[y0:y1 + 1, x0:x1 + 1] |= q <= q_max
    return mask
