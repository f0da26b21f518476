"""Analytic FP64 gradient of the clipped render (oracle; TEST INFRASTRUCTURE ONLY).

The paper renders only; the gradient of its forward is what the backward extension of the
CUDA library computes, so the oracle states that forward once more in plain PyTorch CPU
float64 operations, in the paper's order, and lets reverse-mode automatic differentiation
(a library primitive) take the derivative:

  per Gaussian  sigma = exp(log-scale), R from the normalised quaternion, V = R S^2 R^T
                (Section 3.1); camera-space centre, the Jacobian J of the projection at
                the centre with x/z, y/z clamped to 1.3 tan(half FOV), Sigma2 = (J W V W^T
                J^T)_2x2 + 0.3 I, conic = Sigma2^-1, projected centre (Eq. 9-10); opacity
                sigmoid(logit); colour from real spherical harmonics at normalize(mu - e),
                + 0.5, clamped at 0
  per pixel     q = d^T conic d, alpha0 = opacity exp(-q/2) (Eq. 10); for a cutoff Gaussian
                the pixel ray's chord [t1, t2] through the ellipsoid k R S (Eq. 4-7), the
                plane hit t_p (Eq. 8) and the visible share w of the chord (Eq. 11);
                alpha = min(0.99, alpha0 w) (Eq. 12, Algorithm 1 step 3); skip alpha < 1/255
                or q > 9; front-to-back compositing C = sum c alpha T, stopping before the
                Gaussian that takes T below 1e-4, plus T bg (Eq. 2).

The discrete decisions (labels, culling, each tile's depth-ordered list) are the C oracle's
(oracle/rara_oracle.c); every continuous quantity is recomputed here. The readings of the
gradient where the forward is piecewise constant or clamped are the ones the library
states: w passes gradient only where the plane splits the chord, a clamped alpha (0.99) or
colour (0) passes none through the clamp, and the thresholds are discontinuities. Work goes
tile by tile: the loss of a tile's pixels is built from the parameters and its gradient is
accumulated before the next tile, so memory stays bounded.

Only tests/ import this module; it shares nothing with the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

from . import preprocess as _preprocess, build_keys as _build_keys, CUTOFF

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _legendre_derivative_coeffs(l: int, m: int) -> np.ndarray:
    """Power-series coefficients (ascending) of d^m P_l(z) / dz^m (numpy's Legendre basis)."""
    from numpy.polynomial import Legendre, Polynomial
    return Legendre.basis(l).deriv(m).convert(kind=Polynomial).coef if m <= l else np.zeros(1)


def sh_basis(dirs, degree: int):
    """Real orthonormal spherical harmonics without the Condon-Shortley phase (Y_1,-1 ~ y,
    Y_1,0 ~ z, Y_1,1 ~ x), index l*l + l + m, at unit directions dirs [N, 3]: for m > 0
    sqrt(2) K_l^m Re((x + i y)^m) P_l^(m)(z), for m < 0 the same with Im and |m|, for m = 0
    K_l^0 P_l(z), K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^(m) the m-th derivative of
    the Legendre polynomial."""
    import torch
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            c = _legendre_derivative_coeffs(l, am)
            poly = torch.zeros_like(z)
            for k in range(len(c) - 1, -1, -1):          # Horner in z
                poly = poly * z + float(c[k])
            re, im = torch.ones_like(x), torch.zeros_like(x)
            for _ in range(am):                          # (x + i y)^|m|
                re, im = re * x - im * y, re * y + im * x
            if m == 0:
                out.append(K * poly)
            elif m > 0:
                out.append(math.sqrt(2.0) * K * re * poly)
            else:
                out.append(math.sqrt(2.0) * K * im * poly)
    return torch.stack(out, dim=1)


def _rotation(q):
    """Rotation matrices [N, 3, 3] of quaternions q [N, 4] = (w, x, y, z), normalised."""
    import torch
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)], 1)


def _safe(cond, value, fill):
    """value where cond, fill elsewhere, with no gradient leaking from the unused branch."""
    import torch
    return torch.where(cond, value, torch.as_tensor(fill, dtype=value.dtype))


def _tile_image(leaf, idx, cut, cam, Rc, tc, eye, pl_n, pl_d, k_sigma, degree, px, py, bg):
    """Image [3, P] and final transmittance [P] of the pixels (px, py) over the depth-ordered
    Gaussians idx of their tile, as differentiable functions of the leaves."""
    import torch
    f64 = torch.float64
    mu = leaf["means"][:, idx].T                        # [L, 3]
    sig = torch.exp(leaf["log_scales"][:, idx].T)       # [L, 3]
    Rg = _rotation(leaf["quats"][:, idx].T)             # [L, 3, 3]
    opac = torch.sigmoid(leaf["opacity_logits"][idx])   # [L]
    K = (degree + 1) ** 2
    sh = leaf["sh"][:, idx].T.reshape(-1, K, 3)         # [L, K, 3]: plane k*3 + c

    # Section 3.1 / Eq. 9-10
    V = Rg @ torch.diag_embed(sig * sig) @ Rg.transpose(1, 2)
    t = mu @ Rc.T + tc
    tz = t[:, 2]
    limx = 1.3 * (0.5 * cam.width / cam.fx)
    limy = 1.3 * (0.5 * cam.height / cam.fy)
    txz = torch.clamp(t[:, 0] / tz, -limx, limx)
    tyz = torch.clamp(t[:, 1] / tz, -limy, limy)
    zeros = torch.zeros_like(tz)
    J = torch.stack([torch.stack([cam.fx / tz, zeros, -cam.fx * txz / tz], 1),
                     torch.stack([zeros, cam.fy / tz, -cam.fy * tyz / tz], 1)], 1)   # [L, 2, 3]
    Tm = J @ Rc
    S2 = Tm @ V @ Tm.transpose(1, 2)
    ca, cb, cc = S2[:, 0, 0] + 0.3, S2[:, 0, 1], S2[:, 1, 1] + 0.3
    det = ca * cc - cb * cb
    con_a, con_b, con_c = cc / det, -cb / det, ca / det
    mx = cam.fx * t[:, 0] / tz + cam.cx
    my = cam.fy * t[:, 1] / tz + cam.cy

    # colour at normalize(mu - e)
    dirv = mu - eye
    dirv = dirv / torch.linalg.norm(dirv, dim=1, keepdim=True)
    basis = sh_basis(dirv, degree)                      # [L, K]
    rgb = torch.clamp_min(torch.einsum("lk,lkc->lc", basis, sh) + 0.5, 0.0)

    # per pixel (Eq. 10)
    dx = px[:, None] - mx[None, :]
    dy = py[:, None] - my[None, :]
    q = con_a * dx * dx + 2.0 * con_b * dx * dy + con_c * dy * dy      # [P, L]
    a0 = opac * torch.exp(-0.5 * q)

    # decay weight of the cutoff Gaussians (Eq. 4-8, Eq. 11)
    w = torch.ones_like(a0)
    if bool(cut.any()):
        dcam = torch.stack([(px - cam.cx) / cam.fx, (py - cam.cy) / cam.fy, torch.ones_like(px)], 1)
        dw = dcam @ Rc                                   # rows: R^T dcam
        dw = dw / torch.linalg.norm(dw, dim=1, keepdim=True)                # [P, 3]
        ks = k_sigma * sig                                                   # [L, 3]
        o = torch.einsum("lb,lba->la", eye - mu, Rg) / ks                    # M^-1 (e - mu)
        v = torch.einsum("pb,lba->pla", dw, Rg) / ks[None]                   # M^-1 d
        A = (v * v).sum(-1)
        B = 2.0 * (o[None] * v).sum(-1)
        C = (o * o).sum(-1) - 1.0
        disc = B * B - 4.0 * A * C
        two = disc > 0.0
        sq = torch.sqrt(_safe(two, disc, 1.0))
        t1 = (-B - sq) / (2.0 * A)
        t2 = (-B + sq) / (2.0 * A)
        front = two & (t1 > 0.0) & (t2 > 0.0)
        ne = (pl_n * eye).sum() + pl_d
        nd = (dw @ pl_n)[:, None]                                          # [P, 1]
        s1 = ne + t1 * nd
        s2 = ne + t2 * nd
        v1, v2 = s1 >= 0.0, s2 >= 0.0
        split = front & (v1 != v2)
        tp = -ne / _safe(nd != 0.0, nd, 1.0)
        lvis = torch.where(v1, tp - t1, t2 - tp)
        share = torch.clamp(_safe(split, lvis / (t2 - t1), 0.5), 0.0, 1.0)
        wc = torch.where(split, share, torch.where(front & ~v1 & ~v2, torch.zeros_like(share),
                                                   torch.ones_like(share)))
        w = torch.where(cut[None, :], wc, w)

    # Eq. 12, Algorithm 1 step 3, Eq. 2
    alpha = torch.clamp(a0 * w, max=0.99)
    valid = (q <= 9.0) & (alpha >= 1.0 / 255.0)
    one_m = torch.where(valid, 1.0 - alpha, torch.ones_like(alpha))
    with torch.no_grad():       # the stop is a discontinuity: decided on the values
        T_after = torch.cumprod(one_m, dim=1)
        stop = valid & (T_after < 1e-4)
        first = torch.where(stop.any(1), stop.to(torch.int64).argmax(1),
                            torch.full((stop.shape[0],), stop.shape[1], dtype=torch.int64))
        keep = torch.arange(stop.shape[1])[None, :] < first[:, None]
    blend = valid & keep
    one_b = torch.where(blend, 1.0 - alpha, torch.ones_like(alpha))
    T_excl = torch.cumprod(torch.cat([torch.ones_like(one_b[:, :1]), one_b[:, :-1]], 1), dim=1)
    wgt = torch.where(blend, alpha * T_excl, torch.zeros_like(alpha))
    T_fin = torch.prod(one_b, dim=1)
    img = wgt @ rgb + T_fin[:, None] * torch.as_tensor(bg, dtype=f64)[None, :]   # [P, 3]
    return img.T, T_fin


def render_and_grad(scene, cam, plane, bg=(0.0, 0.0, 0.0), weights=None, tile=(16, 16), grad=True):
    """Render one view and, with grad, the gradient of L = sum(weights * image).

    scene: Gaussian arrays (float32 values are widened exactly; float64 taken as given);
    plane: single clip plane (n, d used as float32 unless plane.exact). Returns dict with
    image [3, H, W], T [H, W] (float64 numpy), and with grad the gradients of L with respect
    to means, log_scales, quats, opacity_logits, sh (the scene's layouts) and plane [4]
    (dL/d(n.x, n.y, n.z, d))."""
    import torch
    from . import _f64, cam16, plane4
    f64 = torch.float64
    if getattr(plane, "extra", ()):
        raise ValueError("the oracle gradient takes single clip planes")
    pre = _preprocess(scene, cam, plane, tile)
    keys, vals, ranges = _build_keys(pre)
    c16 = cam16(cam)
    Rc = torch.tensor(c16[:9].reshape(3, 3), dtype=f64)
    tc = torch.tensor(c16[9:12], dtype=f64)
    fx, fy, cx, cy = (float(v) for v in c16[12:16])

    class _Cam:  # the camera as the oracle reads it (float32 values widened)
        pass

    cm = _Cam()
    cm.fx, cm.fy, cm.cx, cm.cy, cm.width, cm.height = fx, fy, cx, cy, int(cam.width), int(cam.height)
    eye = -(Rc.T @ tc)
    p4 = plane4(plane)
    pl_n = torch.tensor(p4[:3], dtype=f64, requires_grad=grad)
    pl_d = torch.tensor(p4[3], dtype=f64, requires_grad=grad)
    leaf = {k: torch.tensor(_f64(getattr(scene, k)), dtype=f64, requires_grad=grad) for k in PARAMS}
    k_sigma = float(np.float32(plane.k_sigma))
    H, W = int(cam.height), int(cam.width)
    tw, th = tile
    tiles_x = (W + tw - 1) // tw
    image = np.zeros((3, H, W))
    T = np.zeros((H, W))
    wts = None if weights is None else torch.as_tensor(np.asarray(weights, np.float64))
    bgv = [float(b) for b in bg]
    for t in range(ranges.shape[0]):
        ty, tx = divmod(t, tiles_x)
        x0, y0 = tx * tw, ty * th
        x1, y1 = min(W, x0 + tw), min(H, y0 + th)
        ys, xs = np.mgrid[y0:y1, x0:x1]
        pys, pxs = ys.reshape(-1), xs.reshape(-1)
        s, e = int(ranges[t, 0]), int(ranges[t, 1])
        if e <= s:
            for c in range(3):
                image[c, pys, pxs] = bgv[c]
            T[pys, pxs] = 1.0
            continue
        idx_np = vals[s:e].astype(np.int64)
        idx = torch.as_tensor(idx_np)
        cut = torch.as_tensor(pre["label"][idx_np] == CUTOFF)
        px = torch.as_tensor(pxs + 0.5, dtype=f64)
        py = torch.as_tensor(pys + 0.5, dtype=f64)
        img, Tf = _tile_image(leaf, idx, cut, cm, Rc, tc, eye, pl_n, pl_d, k_sigma, int(scene.sh_degree),
                              px, py, bgv)
        image[:, pys, pxs] = img.detach().numpy()
        T[pys, pxs] = Tf.detach().numpy()
        if grad and wts is not None:
            tile_loss = (wts[:, torch.as_tensor(pys), torch.as_tensor(pxs)] * img).sum()
            if tile_loss.requires_grad:
                tile_loss.backward()
    out = {"image": image, "T": T}
    if grad:
        z = lambda p: np.zeros(p.shape) if p.grad is None else p.grad.numpy().copy()
        for k in PARAMS:
            out[k] = z(leaf[k])
        out["plane"] = np.concatenate([z(pl_n), [0.0 if pl_d.grad is None else float(pl_d.grad)]])
    return out
