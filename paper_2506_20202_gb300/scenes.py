"""Seeded synthetic inputs for the clipped Gaussian-splat render.

This module builds inputs only: Gaussian clouds (structure-of-arrays float32),
pinhole cameras and clip planes. It holds none of the render's arithmetic
(no projection, no classification, no compositing), so both the CUDA path and
the FP64 oracle can consume the same arrays without sharing any method code.

Layouts (all float32, C-contiguous, planar so a warp reads one plane coalesced):
    means          [3, n]            x, y, z planes
    log_scales     [3, n]            log sigma per local axis
    quats          [4, n]            w, x, y, z planes (need not be unit length)
    opacity_logits [n]               delta = sigmoid(logit)
    sh             [(L+1)^2 * 3, n]  plane (k*3 + c) is SH coefficient k of channel c,
                                     k = l*l + l + m in the real SH basis
Camera: world_to_cam [3, 4] row-major [R | t] with OpenCV axes (x right, y down,
z forward), square pixels, principal point at the image centre.
Plane: n . x + d = 0 with the visible side where n points (Section 3.2, Eq. 3).

The scene shapes stand in for the paper's datasets (Section 4.1), which are not
available here: a general surface scene (Mip-NeRF360-like), a hair-strand scene
and a multi-layer shell scene.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Real SH band-0 basis value 1 / (2 sqrt(pi)). Only used to turn a target RGB into
# a degree-0 coefficient so that the evaluated colour equals that RGB.
_Y00 = 0.5 / math.sqrt(math.pi)

MODE_NONE = 0      # no clipping: every Gaussian is visible
MODE_HARD = 1      # centre-based hard clipping (Section 1, "Hard Clipping")
MODE_RARA = 2      # three-way classification + ray-traced weight for cutoff (Algorithm 1)
MODE_RARA_ALL = 3  # ablation "wo RaRa": ray-traced weight for every non-invisible Gaussian (Section 4.3)


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def nbytes(self) -> int:
        return sum(int(a.nbytes) for a in (self.means, self.log_scales, self.quats,
                                           self.opacity_logits, self.sh))

    def subset(self, idx: np.ndarray) -> "Scene":
        return Scene(np.ascontiguousarray(self.means[:, idx]),
                     np.ascontiguousarray(self.log_scales[:, idx]),
                     np.ascontiguousarray(self.quats[:, idx]),
                     np.ascontiguousarray(self.opacity_logits[idx]),
                     np.ascontiguousarray(self.sh[:, idx]), self.sh_degree)


@dataclasses.dataclass
class Camera:
    world_to_cam: np.ndarray  # [3, 4] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def eye(self) -> np.ndarray:
        r = self.world_to_cam[:, :3].astype(np.float64)
        t = self.world_to_cam[:, 3].astype(np.float64)
        return -r.T @ t


@dataclasses.dataclass
class Plane:
    n: np.ndarray          # [3] float32
    d: float
    k_sigma: float = 3.0
    mode: int = MODE_RARA
    # further planes (nx, ny, nz, d) of a convex clip volume, at most 3: the visible region
    # is the intersection of the visible sides of this plane and these
    extra: tuple = ()


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q


def look_at_camera(eye, target, width: int, height: int, fov_y_deg: float = 60.0,
                   up=(0.0, -1.0, 0.0)) -> Camera:
    """Pinhole camera at `eye` looking at `target`; fov is the vertical field of view.

    fx = fy = (H/2) / tan(fov_y/2); principal point (W/2, H/2).
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    right = np.cross(fwd, up)                    # x = y cross z with y = -up, z = fwd
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])           # rows: camera axes in world coords
    t = -rot @ eye
    w2c = np.concatenate([rot, t[:, None]], axis=1)
    f = 0.5 * height / math.tan(math.radians(fov_y_deg) * 0.5)
    return Camera(_f32(w2c), float(f), float(f), 0.5 * width, 0.5 * height, int(width), int(height))


def random_unit_normal(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def sweep_offsets(scene: Scene, normal, count: int = 16) -> np.ndarray:
    """Plane offsets d_i so that n.x + d_i = 0 passes through the (i+0.5)/count quantile
    point of the range [min n.mu, max n.mu] (the plane swept across the scene, Section 4.2)."""
    nrm = np.asarray(normal, np.float64)
    s = nrm @ scene.means.astype(np.float64)
    lo, hi = float(s.min()), float(s.max())
    return np.array([-(lo + (i + 0.5) / count * (hi - lo)) for i in range(count)])


def _random_sh(rng, n, degree, std):
    k = (degree + 1) ** 2
    return rng.normal(0.0, std, size=(k * 3, n))


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------

def uniform_scene(n: int = 10_000, seed: int = 0, sh_degree: int = 0) -> Scene:
    """Small plain scene: centres uniform in [-1,1]^3, log-scales N(-3.5, 0.5),
    uniform unit quaternions, opacity sigmoid(N(0,1)), RGB uniform [0,1] at degree 0
    (higher bands N(0, 0.3) when sh_degree > 0)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(3, n))
    log_scales = rng.normal(-3.5, 0.5, size=(3, n))
    quats = random_unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, size=n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((k * 3, n))
    rgb = rng.uniform(0.0, 1.0, size=(3, n))
    sh[0:3] = (rgb - 0.5) / _Y00
    if sh_degree > 0:
        sh[3:] = rng.normal(0.0, 0.3, size=((k - 1) * 3, n))
    return Scene(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), sh_degree)


def gradient_scene(n: int = 24, seed: int = 0, sh_degree: int = 1) -> Scene:
    """Tiny scene for finite-difference gradient checks: centres uniform in [-0.6, 0.6]^3,
    log-scales N(-1.9, 0.25) (splats of a few pixels at 64 px and distance 3, overlapping
    about twice), uniform unit quaternions, opacity sigmoid(N(0, 1)), RGB uniform [0, 1]
    at degree 0 and higher bands N(0, 0.3)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.6, 0.6, size=(3, n))
    log_scales = rng.normal(-1.9, 0.25, size=(3, n))
    quats = random_unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, size=n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((k * 3, n))
    sh[0:3] = (rng.uniform(0.0, 1.0, size=(3, n)) - 0.5) / _Y00
    if sh_degree > 0:
        sh[3:] = rng.normal(0.0, 0.3, size=((k - 1) * 3, n))
    return Scene(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), sh_degree)


def _noisy_surface_points(rng, n, radius=0.8):
    """Points on a seeded radially perturbed sphere r(theta, phi) with N(0, 0.01) jitter."""
    v = rng.standard_normal((3, n))
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    theta = np.arccos(np.clip(v[2], -1, 1))
    phi = np.arctan2(v[1], v[0])
    pert = np.zeros(n)
    for l in range(1, 6):
        for m in range(0, l + 1):
            a = rng.normal(0.0, 0.08 / l)
            ph = rng.uniform(0, 2 * np.pi)
            pert += a * np.sin(theta) ** m * np.cos(l * theta) * np.cos(m * phi + ph)
    r = radius * (1.0 + pert) + rng.normal(0.0, 0.01, size=n)
    return v * r


def general_scene(n: int = 1_000_000, seed: int = 0, sh_degree: int = 3) -> Scene:
    """General surface scene (stand-in for a Mip-NeRF360 capture): 80% of centres on a
    noisy implicit surface, 20% uniform volume fill in [-1,1]^3, log-scales N(-4.5, 0.7),
    SH coefficients N(0, 0.3), opacity sigmoid(N(0.5, 1.5))."""
    rng = np.random.default_rng(seed)
    n_surf = int(round(0.8 * n))
    means = np.empty((3, n))
    means[:, :n_surf] = _noisy_surface_points(rng, n_surf)
    means[:, n_surf:] = rng.uniform(-1.0, 1.0, size=(3, n - n_surf))
    perm = rng.permutation(n)
    means = means[:, perm]
    log_scales = rng.normal(-4.5, 0.7, size=(3, n))
    quats = random_unit_quats(rng, n)
    logits = rng.normal(0.5, 1.5, size=n)
    sh = _random_sh(rng, n, sh_degree, 0.3)
    return Scene(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), sh_degree)


def _quat_from_x_axis(t):
    """Unit quaternions (w,x,y,z) of the shortest rotation taking e_x to unit vectors t [3, n]."""
    w = 1.0 + t[0]
    x = np.zeros_like(w)
    y = -t[2]
    z = t[1]
    q = np.stack([w, x, y, z])
    bad = w < 1e-6   # t = -e_x: rotate 180 degrees about z
    q[:, bad] = np.array([0.0, 0.0, 0.0, 1.0])[:, None]
    return q / np.linalg.norm(q, axis=0, keepdims=True)


def hair_scene(curves: int = 10_000, segments: int = 50, seed: int = 0,
               plane_normal=None, target_straddle: float = 0.40):
    """Hair-strand scene: one anisotropic Gaussian per segment of seeded cubic Bezier curves
    rooted on the upper half of a unit-sphere scalp. Axis scales 1:1:40 with the long axis
    tangent to the curve, SH degree 1, opacity uniform [0.3, 0.9].

    Returns (scene, plane_normal, plane_d). The plane is oblique to the mean strand
    direction; its offset goes through the median of n.mu and the common scale factor of
    the strand Gaussians is chosen so that `target_straddle` of the Gaussians have their
    3-sigma bounding sphere crossing the plane (the 30-50% band the workload asks for).
    """
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, curves))
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    v[1] = -np.abs(v[1])                     # roots on the upper half (y down is "up" negated)
    root = v.copy()
    length = rng.uniform(0.8, 1.4, size=curves)
    gravity = np.array([0.0, 1.0, 0.0])[:, None]
    p0 = root
    p1 = root + root * (length / 3.0)
    p2 = p1 + gravity * (length / 3.0) + rng.normal(0, 0.08, size=(3, curves))
    p3 = p2 + gravity * (length / 3.0) + root * 0.15 + rng.normal(0, 0.12, size=(3, curves))
    s = (np.arange(segments + 1) / segments)[None, :, None]          # [1, S+1, 1]

    def bez(u):
        a, b, c, d = (p[:, None, :] for p in (p0, p1, p2, p3))      # [3, 1, C]
        return ((1 - u) ** 3) * a + 3 * ((1 - u) ** 2) * u * b + 3 * (1 - u) * u * u * c + u ** 3 * d

    pts = bez(s)                                                      # [3, S+1, C]
    seg = pts[:, 1:, :] - pts[:, :-1, :]
    seglen = np.linalg.norm(seg, axis=0)                               # [S, C]
    tangent = seg / np.maximum(seglen, 1e-12)
    centre = 0.5 * (pts[:, 1:, :] + pts[:, :-1, :])
    n = curves * segments
    means = centre.reshape(3, n)
    tangent = tangent.reshape(3, n)
    seglen = seglen.reshape(n)
    quats = _quat_from_x_axis(tangent)

    if plane_normal is None:
        plane_normal = np.array([0.25, 0.9, 0.35])
    nrm = np.asarray(plane_normal, np.float64)
    nrm = nrm / np.linalg.norm(nrm)
    dist = nrm @ means
    d = -float(np.median(dist))
    sigma_long_unit = 0.5 * seglen
    # Common factor so that target_straddle of the 3-sigma bounding spheres cross the plane.
    ratio = np.abs(dist + d) / (3.0 * sigma_long_unit)
    factor = float(np.quantile(ratio, target_straddle))
    sigma_long = sigma_long_unit * max(factor, 1.0)
    log_scales = np.stack([np.log(sigma_long), np.log(sigma_long / 40.0), np.log(sigma_long / 40.0)])
    logits_p = rng.uniform(0.3, 0.9, size=n)
    logits = np.log(logits_p / (1 - logits_p))
    sh = _random_sh(rng, n, 1, 0.3)
    base = np.array([0.35, 0.22, 0.12])[:, None]
    sh[0:3] = (base + rng.normal(0, 0.05, size=(3, n)) - 0.5) / _Y00
    scene = Scene(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), 1)
    return scene, nrm.astype(np.float32), d


def shells_scene(per_shell: int = 700_000, seed: int = 0, shells: int = 3) -> Scene:
    """Multi-layer scene: nested ellipsoidal shells, per-shell SH degree-2 palettes plus noise."""
    rng = np.random.default_rng(seed)
    parts = []
    radii = [(0.95, 0.8, 0.7), (0.7, 0.6, 0.5), (0.45, 0.38, 0.3)][:shells]
    k = 9
    for si, (ax, ay, az) in enumerate(radii):
        v = rng.standard_normal((3, per_shell))
        v /= np.linalg.norm(v, axis=0, keepdims=True)
        pos = v * np.array([ax, ay, az])[:, None] * (1.0 + rng.normal(0, 0.01, size=per_shell))
        palette = rng.normal(0.0, 0.3, size=(k * 3, 1))
        sh = palette + rng.normal(0.0, 0.05, size=(k * 3, per_shell))
        parts.append((pos, sh))
    n = per_shell * len(radii)
    means = np.concatenate([p for p, _ in parts], axis=1)
    sh = np.concatenate([s for _, s in parts], axis=1)
    log_scales = rng.normal(-4.6, 0.5, size=(3, n))
    quats = random_unit_quats(rng, n)
    logits = rng.normal(0.5, 1.0, size=n)
    return Scene(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), 2)


# --------------------------------------------------------------------------------------
# Named workloads (scene, camera, plane set)
# --------------------------------------------------------------------------------------

def small_uniform_workload(n: int = 10_000, width: int = 256, height: int = 256, seed: int = 0):
    """10k Gaussians, SH degree 0, 256x256, camera at distance 3 looking at the origin,
    FOV 60 degrees, black background, one plane through the origin with a seeded normal."""
    scene = uniform_scene(n, seed=seed, sh_degree=0)
    cam = look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), width, height, 60.0)
    nrm = random_unit_normal(seed + 1)
    plane = Plane(_f32(nrm), 0.0, 3.0, MODE_RARA)
    return scene, cam, plane


def general_workload(n: int = 1_000_000, width: int = 1920, height: int = 1080, seed: int = 0,
                     sweep: int = 16):
    """1M-Gaussian general scene at 1920x1080 with a sweep of `sweep` parallel plane offsets."""
    scene = general_scene(n, seed=seed, sh_degree=3)
    eye = 3.0 * np.array([0.3, -0.35, -1.0]) / np.linalg.norm([0.3, -0.35, -1.0])
    cam = look_at_camera(eye, (0.0, 0.0, 0.0), width, height, 60.0)
    nrm = random_unit_normal(seed + 1)
    planes = [Plane(_f32(nrm), float(d), 3.0, MODE_RARA) for d in sweep_offsets(scene, nrm, sweep)]
    return scene, cam, planes


def shells_training_workload(per_shell: int = 700_000, views: int = 64, seed: int = 0,
                             resolutions=((512, 512), (1024, 1024), (1920, 1080))):
    """Multi-layer differentiation workload: the 3-shell scene (3 x per_shell Gaussians, SH
    degree 2), a perturbed copy of it whose renders are the L2 targets (colours N(0, 0.1)
    and opacity logits N(0, 0.3) added), and `views` seeded views at the resolutions in turn,
    each a camera on a sphere of radius 3 looking at the centre and a plane with a random
    unit normal and an offset uniform in [-0.5, 0.5] (cutting through the shells).
    Returns (scene, target_scene, [(camera, plane)])."""
    scene = shells_scene(per_shell, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    target = Scene(scene.means, scene.log_scales, scene.quats,
                   _f32(scene.opacity_logits + rng.normal(0.0, 0.3, size=scene.n)),
                   _f32(scene.sh + rng.normal(0.0, 0.1, size=scene.sh.shape)), scene.sh_degree)
    out = []
    for v in range(views):
        w, h = resolutions[v % len(resolutions)]
        e = rng.standard_normal(3)
        e = 3.0 * e / np.linalg.norm(e)
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        out.append((look_at_camera(e, (0.0, 0.0, 0.0), w, h, 60.0),
                    Plane(_f32(nrm), float(rng.uniform(-0.5, 0.5)), 3.0, MODE_RARA)))
    return scene, target, out
