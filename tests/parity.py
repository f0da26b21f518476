"""Comparison helpers: CUDA path (through the C ABI) vs the FP64 oracle.

Tolerances (image max-abs 2e-3 and mean-abs 1e-4 per channel, values in [0,1] scale;
bit-exact labels, tiles and key order except near thresholds) are the ones the render
is specified to, and every exemption is counted and bounded by the caller.
"""
import numpy as np
import torch

import oracle
from paper_2506_20202_gb300 import rara

IMG_MAX_ABS = 2e-3
IMG_MEAN_ABS = 1e-4
CLASS_EXEMPT = 1e-6   # world units from a class threshold
RECT_EXEMPT = 2e-3    # pixels from a tile edge (float32 position + footprint error)
TILE_EXEMPT = 0.03    # |smallest q over a tile - q_cut| under which float32 may list differently


def gpu_frame(scene, cam, plane, bg=(0.0, 0.0, 0.0), renderer=None, export=True, tuning=None, tiling=None):
    r = renderer or rara.Renderer(tuning=tuning, tiling=tiling)
    gs = rara.GaussianTensors.from_scene(scene)
    img, T, nc = r.render(gs, cam, plane, bg)
    torch.cuda.synchronize()
    out = dict(image=img.cpu().numpy().astype(np.float64), T=T.cpu().numpy().astype(np.float64),
               n_contrib=nc.cpu().numpy())
    if export:
        fg = r.frame_gaussians(scene.n)
        out["g"] = {k: v.cpu().numpy() for k, v in fg.items()}
        keys, vals, ranges, info = r.frame_pairs()
        out["keys"] = keys.cpu().numpy().view(np.uint64)
        out["vals"] = vals.cpu().numpy().view(np.uint32)
        out["ranges"] = ranges.cpu().numpy()
        out["info"] = info
    if renderer is None:
        r.close()
    return out


def exempt_gaussians(pre):
    """Gaussians whose label, culling or tile rectangle may legitimately differ in float32."""
    return ((pre["margin_class"] <= CLASS_EXEMPT) | (pre["margin_gauss"] <= CLASS_EXEMPT)
            | (pre["margin_rect"] <= RECT_EXEMPT))


def check_gaussians(pre, g, report):
    n = pre["label"].shape[0]
    ex_class = (pre["margin_class"] <= CLASS_EXEMPT) | (pre["margin_gauss"] <= CLASS_EXEMPT)
    lab_bad = (g["labels"] != pre["label"]) & ~ex_class
    assert lab_bad.sum() == 0, f"{lab_bad.sum()} labels differ (first {np.nonzero(lab_bad)[0][:5]})"
    report["label_exempt"] = int(ex_class.sum())
    ex = exempt_gaussians(pre)
    orc_tiles = np.where(pre["culled"] == 1, 0, pre["tiles"])
    t_bad = (g["tiles"].astype(np.int64) != orc_tiles) & ~ex
    assert t_bad.sum() == 0, f"{t_bad.sum()} tile counts differ (first {np.nonzero(t_bad)[0][:5]})"
    both = (orc_tiles > 0) & (g["tiles"] > 0)
    rect_bad = np.any(g["rect"].T != pre["rect"], axis=1) & both & ~ex
    assert rect_bad.sum() == 0, f"{rect_bad.sum()} rects differ"
    report["rect_exempt"] = int((ex & ~ex_class).sum())
    idx = np.nonzero(both)[0]
    if idx.size == 0:
        return
    # depth key: the correctly rounded float32 of the depth (2 ulp allowed, 0 expected)
    od = pre["depth"][idx].astype(np.float32).view(np.int32).astype(np.int64)
    gd = g["depth"][idx].view(np.int32).astype(np.int64)
    report["depth_ulp_max"] = int(np.abs(od - gd).max())
    assert report["depth_ulp_max"] <= 2, "depth bits differ by more than 2 ulp"
    assert np.allclose(g["mean2d"].T[idx], pre["mean2d"][idx], rtol=0, atol=1e-3 + 2e-6 * np.abs(pre["mean2d"][idx]))
    con_o = pre["conic"][idx]
    con_g = g["conic"].T[idx]
    scale = np.abs(con_o).max(axis=1, keepdims=True)
    assert np.all(np.abs(con_g - con_o) <= 2e-4 * scale + 1e-9), \
        f"conic rel err {np.max(np.abs(con_g - con_o) / scale):.2e}"
    assert np.abs(g["rgb"].T[idx] - pre["rgb"][idx]).max() <= 2e-5
    assert np.abs(g["opacity"][idx] - pre["opacity"][idx]).max() <= 2e-6


def check_pairs(pre, kvr, gpu, report):
    okeys, ovals, oranges = kvr
    gkeys, gvals, granges = gpu["keys"], gpu["vals"], gpu["ranges"]
    ex = exempt_gaussians(pre)
    report["pairs_oracle"] = int(okeys.size)
    report["pairs_gpu"] = int(gkeys.size)
    nt = oranges.shape[0]
    # the GPU's own ranges partition its list by tile
    gt = (gkeys >> np.uint64(32)).astype(np.int64)
    assert np.all(np.diff(gt) >= 0), "GPU keys are not sorted by tile"
    for t in np.unique(gt):
        s, e = granges[t]
        assert e > s and np.all(gt[s:e] == t)
    assert (granges[:, 1] - granges[:, 0]).sum() == gkeys.size
    # depth bits of every pair within 2 ulp of the oracle's
    od = pre["depth"].astype(np.float32).view(np.int32).astype(np.int64)
    gd = (gkeys & np.uint64(0xffffffff)).astype(np.int64)
    assert np.abs(gd - od[gvals]).max(initial=0) <= 2
    # per tile: same non-exempt members in the same order, except near depth ties
    exact_tiles = 0
    tie_swaps = 0
    odepth32 = pre["depth"].astype(np.float32).view(np.int32).astype(np.int64)
    listing_exempt = 0
    for t in range(nt):
        o = ovals[oranges[t, 0]:oranges[t, 1]]
        g = gvals[granges[t, 0]:granges[t, 1]]
        o = o[~ex[o]]
        g = g[~ex[g]]
        if np.array_equal(o, g):
            exact_tiles += 1
            continue
        # a Gaussian listed on one side only must be at the listing threshold of that tile
        only = np.setxor1d(o, g)
        for i in only:
            m = oracle.tile_margin(pre, int(i), t)
            assert m <= TILE_EXEMPT, f"tile {t}: Gaussian {i} listed on one side only (margin {m:.3g})"
        listing_exempt += only.size
        o = o[~np.isin(o, only)]
        g = g[~np.isin(g, only)]
        if np.array_equal(o, g):
            continue
        assert np.array_equal(np.sort(o), np.sort(g)), f"tile {t}: member sets differ"
        # order may differ only among Gaussians whose float32 depths are within 2 ulp
        pos = {int(v): k for k, v in enumerate(o)}
        for a, b in zip(g[:-1], g[1:]):
            if pos[int(a)] > pos[int(b)]:
                assert abs(odepth32[a] - odepth32[b]) <= 2, f"tile {t}: order differs"
                tie_swaps += 1
    report["tiles_exact"] = exact_tiles
    report["tiles"] = nt
    report["tie_swaps"] = tie_swaps
    report["listing_exempt"] = listing_exempt
    assert listing_exempt <= 1e-3 * max(1, okeys.size) + 5, "too many pairs at the listing threshold"


def check_image(pre, ref, gpu, report, rows=None, max_flag_frac=0.05, extra_mask=None):
    H, W = ref["T"].shape
    sel = np.ones((H, W), bool)
    if rows is not None:
        sel[:] = False
        sel[rows[0]:rows[1]] = True
    ex_g = np.nonzero(pre["margin_gauss"] <= CLASS_EXEMPT)[0]
    flagged = (ref["events"] != 0)
    if ex_g.size:
        flagged |= oracle.support_mask(pre, ex_g, H, W)
    if extra_mask is not None:
        flagged |= extra_mask
    ok = sel & ~flagged
    report["pixels"] = int(sel.sum())
    report["flagged"] = int((sel & flagged).sum())
    assert report["flagged"] <= max_flag_frac * max(1, report["pixels"]), \
        f"{report['flagged']} of {report['pixels']} pixels flagged"
    d = np.abs(gpu["image"] - ref["image"])
    for c in range(3):
        dc = d[c][ok]
        if dc.size:
            report[f"max_abs_c{c}"] = float(dc.max())
            report[f"mean_abs_c{c}"] = float(dc.mean())
            assert dc.max() <= IMG_MAX_ABS, f"channel {c}: max abs {dc.max():.3e}"
            assert dc.mean() <= IMG_MEAN_ABS, f"channel {c}: mean abs {dc.mean():.3e}"
    dT = np.abs(gpu["T"] - ref["T"])[ok] if "T" in gpu else np.zeros(0)
    if dT.size:
        report["T_max_abs"] = float(dT.max())
        assert dT.max() <= IMG_MAX_ABS
    return ok
