"""Thin Python binding of librara.so (the C ABI in include/rara.h).

Argument marshalling only: every step of the render runs in the CUDA library. The
functions keep the C names; they take torch CUDA tensors (passed by data pointer) and a
CUDA stream (default: torch's current stream) and raise RaraError on a non-zero status.
There is no CPU fallback: if librara.so is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librara.so")

RARA_OK, RARA_ERR_INVALID_ARG, RARA_ERR_BUDGET, RARA_ERR_CUDA, RARA_ERR_TIMEOUT, RARA_ERR_OVERFLOW = 0, 1, 2, 3, 4, 5
MODE_NONE, MODE_HARD, MODE_RARA, MODE_RARA_ALL = 0, 1, 2, 3
INVISIBLE, VISIBLE, CUTOFF = 0, 1, 2


class RaraError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rara status {code}: {msg}")
        self.code = code


class rara_gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32)]


class rara_camera(C.Structure):
    _fields_ = [("world_to_cam", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class rara_plane(C.Structure):
    _fields_ = [("n", C.c_float * 3), ("d", C.c_float), ("k_sigma", C.c_float), ("mode", C.c_int32),
                ("n_extra", C.c_int32), ("extra", (C.c_float * 4) * 3)]


class rara_view(C.Structure):
    _fields_ = [("scene", C.c_int32), ("camera", rara_camera), ("plane", rara_plane), ("bg", C.c_float * 3),
                ("image", C.c_void_p), ("final_T", C.c_void_p), ("n_contrib", C.c_void_p)]


class rara_gaussian_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class rara_frame_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_rendered", C.c_int64), ("n_cutoff", C.c_int64),
                ("n_pairs", C.c_int64), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32),
                ("n_evaluated", C.c_int64), ("n_walked", C.c_int64), ("n_cut_evaluated", C.c_int64),
                ("n_tested", C.c_int64), ("n_pair_candidates", C.c_int64), ("n_depth_keys", C.c_int64),
                ("n_shared_pairs", C.c_int64)]


# name -> (restype, argtypes); every symbol declared in include/rara.h
_P = C.c_void_p
SIGNATURES = {
    "rara_ctx_create": (C.c_int, [C.c_size_t, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "rara_ctx_destroy": (C.c_int, [_P]),
    "rara_last_error": (C.c_char_p, [_P]),
    "rara_ctx_bytes": (C.c_size_t, [_P]),
    "rara_ctx_reserve": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int32, C.c_int32]),
    "rara_ctx_sync": (C.c_int, [_P, _P]),
    "rara_ctx_launches": (C.c_int64, [_P]),
    "rara_ctx_set_tuning": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "rara_ctx_set_tiling": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32]),
    "rara_ctx_count_work": (C.c_int, [_P, C.c_int32]),
    "rara_ctx_debug_waits": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "rara_ctx_stage_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "rara_ctx_kernel_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "rara_preprocess": (C.c_int, [_P, C.POINTER(rara_gaussians), C.POINTER(rara_camera),
                                  C.POINTER(rara_plane), _P]),
    "rara_bin": (C.c_int, [_P, _P]),
    "rara_render": (C.c_int, [_P, C.POINTER(C.c_float), _P, _P, _P, _P]),
    "rara_render_frame": (C.c_int, [_P, C.POINTER(rara_gaussians), C.POINTER(rara_camera),
                                    C.POINTER(rara_plane), C.POINTER(C.c_float), _P, _P, _P, _P]),
    "rara_render_batch": (C.c_int, [_P, C.POINTER(rara_gaussians), C.c_int32, C.POINTER(rara_view), C.c_int32, _P]),
    "rara_render_batch_graph": (C.c_int, [_P, C.POINTER(rara_gaussians), C.c_int32, C.POINTER(rara_view), C.c_int32,
                                          _P]),
    "rara_render_backward": (C.c_int, [_P, C.POINTER(C.c_void_p), C.POINTER(rara_gaussian_grads), _P, _P]),
    "rara_loss_l2": (C.c_int, [_P, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_float), _P, _P]),
    "rara_ctx_backward_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "rara_frame_info_get": (C.c_int, [_P, C.c_int32, C.POINTER(rara_frame_info)]),
    "rara_frame_gaussians": (C.c_int, [_P, C.c_int32] + [_P] * 9),
    "rara_frame_pairs": (C.c_int, [_P, C.c_int32] + [_P] * 4),
    "rara_render_frame_noalloc": (C.c_int, [C.POINTER(rara_gaussians), C.POINTER(rara_camera),
                                            C.POINTER(rara_plane), C.POINTER(C.c_float), _P, _P, _P, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load librara.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2506_20202_gb300.build.build() "
                               "(the renderer has no CPU fallback)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(ctx, rc: int):
    if rc != RARA_OK:
        msg = load().rara_last_error(ctx)
        raise RaraError(rc, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# --------------------------------------------------------------------------------------
# Marshalling helpers
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class GaussianTensors:
    """Device-resident Gaussians (planar float32 CUDA tensors, see include/rara.h)."""
    means: "torch.Tensor"
    log_scales: "torch.Tensor"
    quats: "torch.Tensor"
    opacity_logits: "torch.Tensor"
    sh: "torch.Tensor"
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    @staticmethod
    def from_scene(scene, device="cuda") -> "GaussianTensors":
        import torch
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return GaussianTensors(f(scene.means), f(scene.log_scales), f(scene.quats),
                               f(scene.opacity_logits), f(scene.sh), int(scene.sh_degree))

    def _check(self):
        for t in (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh):
            assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"

    def c_struct(self) -> rara_gaussians:
        self._check()
        return rara_gaussians(self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr(),
                              self.opacity_logits.data_ptr(), self.sh.data_ptr(), self.n, self.sh_degree)

    def grads_struct(self) -> rara_gaussian_grads:
        """These tensors as the gradient arrays of rara_render_backward."""
        self._check()
        return rara_gaussian_grads(self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr(),
                                   self.opacity_logits.data_ptr(), self.sh.data_ptr())

    def empty_like(self) -> "GaussianTensors":
        import torch
        return GaussianTensors(*(torch.empty_like(t) for t in (self.means, self.log_scales, self.quats,
                                                                 self.opacity_logits, self.sh)), self.sh_degree)


def camera_struct(cam) -> rara_camera:
    c = rara_camera()
    w2c = np.asarray(cam.world_to_cam, np.float32).reshape(-1)
    for k in range(12):
        c.world_to_cam[k] = float(w2c[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def plane_struct(plane) -> rara_plane:
    p = rara_plane()
    for k in range(3):
        p.n[k] = float(plane.n[k])
    p.d = float(plane.d)
    p.k_sigma = float(plane.k_sigma)
    p.mode = int(plane.mode)
    extra = getattr(plane, "extra", ())
    p.n_extra = len(extra)
    for e, row in enumerate(extra[:3]):
        for k in range(4):
            p.extra[e][k] = float(row[k])
    return p


# --------------------------------------------------------------------------------------
# C entry points (same names)
# --------------------------------------------------------------------------------------

def rara_ctx_create(budget_bytes: int = 0, tile_w: int = 16, tile_h: int = 16):
    lib = load()
    h = C.c_void_p()
    rc = lib.rara_ctx_create(int(budget_bytes), int(tile_w), int(tile_h), C.byref(h))
    if rc != RARA_OK:
        raise RaraError(rc, "rara_ctx_create failed")
    return h


def rara_ctx_destroy(ctx):
    load().rara_ctx_destroy(ctx)


def rara_ctx_bytes(ctx) -> int:
    return int(load().rara_ctx_bytes(ctx))


def rara_ctx_reserve(ctx, slots: int, pairs: int, views: int, max_view_tiles: int):
    """Allocate scratch up front for batches up to these sizes (see include/rara.h)."""
    _check(ctx, load().rara_ctx_reserve(ctx, int(slots), int(pairs), int(views), int(max_view_tiles)))


def rara_ctx_launches(ctx) -> int:
    return int(load().rara_ctx_launches(ctx))


def rara_ctx_set_tuning(ctx, split2_bits: int, split4_bits: int):
    _check(ctx, load().rara_ctx_set_tuning(ctx, int(split2_bits), int(split4_bits)))


def rara_ctx_set_tiling(ctx, tile_w: int, tile_h: int, blend_depth: int = 256):
    _check(ctx, load().rara_ctx_set_tiling(ctx, int(tile_w), int(tile_h), int(blend_depth)))


def rara_ctx_count_work(ctx, on: bool = True):
    _check(ctx, load().rara_ctx_count_work(ctx, int(bool(on))))


def rara_ctx_debug_waits(ctx, spin_limit: int, orphan_first_partition: bool):
    """Test hook: lower the next compaction's look-back poll limit and optionally leave its
    first partition unprocessed (see include/rara.h)."""
    _check(ctx, load().rara_ctx_debug_waits(ctx, int(spin_limit), int(bool(orphan_first_partition))))


def rara_ctx_stage_ms(ctx):
    """(preprocess, bin, render) GPU milliseconds of the last frame or batch rendered without a graph."""
    out = (C.c_float * 3)()
    _check(ctx, load().rara_ctx_stage_ms(ctx, out))
    return tuple(float(x) for x in out)


def rara_ctx_kernel_ms(ctx):
    """[preprocess, compaction, depth sort, emission, tile sort, ranges + order] GPU ms of the
    last render launched outside a graph."""
    out = (C.c_float * 6)()
    _check(ctx, load().rara_ctx_kernel_ms(ctx, out))
    return [float(v) for v in out]


def rara_ctx_sync(ctx, stream=None):
    _check(ctx, load().rara_ctx_sync(ctx, _stream(stream)))


def rara_preprocess(ctx, gaussians: GaussianTensors, cam, plane, stream=None):
    g, c, p = gaussians.c_struct(), camera_struct(cam), plane_struct(plane)
    _check(ctx, load().rara_preprocess(ctx, C.byref(g), C.byref(c), C.byref(p), _stream(stream)))


def rara_bin(ctx, stream=None):
    _check(ctx, load().rara_bin(ctx, _stream(stream)))


def rara_render(ctx, bg, image, final_T=None, n_contrib=None, stream=None):
    bgv = (C.c_float * 3)(*[float(x) for x in bg])
    _check(ctx, load().rara_render(ctx, bgv, _ptr(image), _ptr(final_T), _ptr(n_contrib), _stream(stream)))


def rara_render_frame(ctx, gaussians: GaussianTensors, cam, plane, bg, image, final_T=None, n_contrib=None,
                      stream=None):
    g, c, p = gaussians.c_struct(), camera_struct(cam), plane_struct(plane)
    bgv = (C.c_float * 3)(*[float(x) for x in bg])
    _check(ctx, load().rara_render_frame(ctx, C.byref(g), C.byref(c), C.byref(p), bgv, _ptr(image),
                                         _ptr(final_T), _ptr(n_contrib), _stream(stream)))


def rara_render_frame_noalloc(gaussians: GaussianTensors, cam, plane, bg, image, final_T=None, n_contrib=None,
                              stream=None):
    """Allocation-free frame render (static scratch, see include/rara.h); raises RaraError."""
    g, c, p = gaussians.c_struct(), camera_struct(cam), plane_struct(plane)
    bgv = (C.c_float * 3)(*[float(x) for x in bg])
    rc = load().rara_render_frame_noalloc(C.byref(g), C.byref(c), C.byref(p), bgv, _ptr(image), _ptr(final_T),
                                          _ptr(n_contrib), _stream(stream))
    if rc != RARA_OK:
        raise RaraError(rc, "rara_render_frame_noalloc failed (RARA_ERR_BUDGET: input beyond the static limits)")


@dataclasses.dataclass
class View:
    """One view of a batch: scene index, camera, plane, background and device outputs."""
    scene: int
    camera: object
    plane: object
    image: "torch.Tensor"
    final_T: "torch.Tensor" = None
    n_contrib: "torch.Tensor" = None
    bg: tuple = (0.0, 0.0, 0.0)

    def c_struct(self) -> rara_view:
        v = rara_view()
        v.scene = int(self.scene)
        v.camera = camera_struct(self.camera)
        v.plane = plane_struct(self.plane)
        for k in range(3):
            v.bg[k] = float(self.bg[k])
        v.image = self.image.data_ptr()
        v.final_T = None if self.final_T is None else self.final_T.data_ptr()
        v.n_contrib = None if self.n_contrib is None else self.n_contrib.data_ptr()
        return v


def _batch_structs(scenes, views):
    sc = (rara_gaussians * len(scenes))(*[g.c_struct() for g in scenes])
    vw = (rara_view * len(views))(*[v.c_struct() for v in views])
    return sc, vw


def rara_render_batch(ctx, scenes, views, stream=None):
    """Render every View of `views` (list) over the GaussianTensors of `scenes` (list)."""
    sc, vw = _batch_structs(scenes, views)
    _check(ctx, load().rara_render_batch(ctx, sc, len(scenes), vw, len(views), _stream(stream)))


def rara_render_batch_graph(ctx, scenes, views, stream=None):
    """As rara_render_batch, replaying a CUDA graph of the batch's stages once captured."""
    sc, vw = _batch_structs(scenes, views)
    _check(ctx, load().rara_render_batch_graph(ctx, sc, len(scenes), vw, len(views), _stream(stream)))


def rara_render_backward(ctx, dL_dimages, grads, plane_grads=None, stream=None):
    """Backward of the last render on ctx. dL_dimages: one [3, H, W] CUDA tensor per view
    (the forward's view order); grads: one GaussianTensors of gradient buffers per scene
    (written); plane_grads: [num_views, 4] CUDA tensor (written) or None."""
    for t in dL_dimages:
        assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"
    ptrs = (C.c_void_p * len(dL_dimages))(*[t.data_ptr() for t in dL_dimages])
    gs = (rara_gaussian_grads * len(grads))(*[g.grads_struct() for g in grads])
    if plane_grads is not None:
        assert plane_grads.is_cuda and plane_grads.is_contiguous() and plane_grads.shape[-1] == 4
    _check(ctx, load().rara_render_backward(ctx, ptrs, gs, _ptr(plane_grads), _stream(stream)))


def rara_loss_l2(ctx, targets, dL_dimages, scale, loss, stream=None):
    """L2 objective of the last render on ctx: per view v, loss[v] = scale[v] * sum((image -
    target)^2) and dL_dimages[v] = 2 scale[v] (image - target). targets, dL_dimages: one
    [3, H, W] float32 CUDA tensor per view (the forward's view order; an output may be its
    target); scale: floats; loss: [num_views] float64 CUDA tensor (written)."""
    for t in list(targets) + list(dL_dimages):
        assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"
    assert len(targets) == len(dL_dimages) == len(scale)
    assert loss.is_cuda and loss.is_contiguous() and str(loss.dtype) == "torch.float64" and loss.numel() >= len(scale)
    tp = (C.c_void_p * len(targets))(*[t.data_ptr() for t in targets])
    dp_ = (C.c_void_p * len(dL_dimages))(*[t.data_ptr() for t in dL_dimages])
    sc = (C.c_float * len(scale))(*[float(x) for x in scale])
    _check(ctx, load().rara_loss_l2(ctx, tp, dp_, sc, _ptr(loss), _stream(stream)))


def rara_ctx_backward_ms(ctx):
    """(render backward, preprocess backward) GPU milliseconds of the last backward."""
    out = (C.c_float * 2)()
    _check(ctx, load().rara_ctx_backward_ms(ctx, out))
    return tuple(float(x) for x in out)


def rara_frame_info_get(ctx, view: int = 0) -> dict:
    info = rara_frame_info()
    _check(ctx, load().rara_frame_info_get(ctx, int(view), C.byref(info)))
    return {k: getattr(info, k) for k, _ in rara_frame_info._fields_}


def rara_frame_gaussians(ctx, view: int = 0, labels=None, depth=None, mean2d=None, conic=None, rgb=None,
                         opacity=None, rect=None, tiles=None, stream=None):
    _check(ctx, load().rara_frame_gaussians(ctx, int(view), _ptr(labels), _ptr(depth), _ptr(mean2d), _ptr(conic),
                                            _ptr(rgb), _ptr(opacity), _ptr(rect), _ptr(tiles), _stream(stream)))


def rara_frame_pairs(ctx, view: int = 0, keys=None, values=None, ranges=None, stream=None):
    _check(ctx, load().rara_frame_pairs(ctx, int(view), _ptr(keys), _ptr(values), _ptr(ranges), _stream(stream)))


# --------------------------------------------------------------------------------------
# Convenience
# --------------------------------------------------------------------------------------

class Renderer:
    """Owns a context and output buffers; render() runs the three stages on a stream."""

    def __init__(self, budget_bytes: int = 0, tuning=None, tiling=None):
        self.ctx = rara_ctx_create(budget_bytes)
        self.generation = 0      # forwards run through this renderer (see autograd.py)
        if tuning is not None:
            rara_ctx_set_tuning(self.ctx, *tuning)
        if tiling is not None:   # (tile_w, tile_h[, blend_depth])
            rara_ctx_set_tiling(self.ctx, *tiling)

    def close(self):
        if self.ctx is not None:
            rara_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, gaussians: GaussianTensors, cam, plane, bg=(0.0, 0.0, 0.0), out=None, stream=None):
        import torch
        H, W = int(cam.height), int(cam.width)
        if out is None:
            out = (torch.empty((3, H, W), dtype=torch.float32, device="cuda"),
                   torch.empty((H, W), dtype=torch.float32, device="cuda"),
                   torch.empty((H, W), dtype=torch.int32, device="cuda"))
        image, T, nc = out
        self.generation += 1
        rara_render_frame(self.ctx, gaussians, cam, plane, bg, image, T, nc, stream)
        return image, T, nc

    def frame_gaussians(self, n: int, view: int = 0):
        import torch
        dev = "cuda"
        out = dict(labels=torch.zeros(n, dtype=torch.uint8, device=dev),
                   depth=torch.zeros(n, dtype=torch.float32, device=dev),
                   mean2d=torch.zeros((2, n), dtype=torch.float32, device=dev),
                   conic=torch.zeros((3, n), dtype=torch.float32, device=dev),
                   rgb=torch.zeros((3, n), dtype=torch.float32, device=dev),
                   opacity=torch.zeros(n, dtype=torch.float32, device=dev),
                   rect=torch.zeros((4, n), dtype=torch.int32, device=dev),
                   tiles=torch.zeros(n, dtype=torch.int32, device=dev))
        rara_frame_gaussians(self.ctx, view, **out)
        return out

    def frame_pairs(self, view: int = 0):
        import torch
        info = rara_frame_info_get(self.ctx, view)
        p = int(info["n_pairs"])
        nt = info["tiles_x"] * info["tiles_y"]
        keys = torch.zeros(max(p, 1), dtype=torch.int64, device="cuda")
        vals = torch.zeros(max(p, 1), dtype=torch.int32, device="cuda")
        ranges = torch.zeros((nt, 2), dtype=torch.int64, device="cuda")
        rara_frame_pairs(self.ctx, view, keys, vals, ranges)
        return keys[:p], vals[:p], ranges, info
