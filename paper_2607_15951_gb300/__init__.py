"""GB300 rasterizer for standard 3D Gaussian Splatting (forward pass).

Python binding of the C ABI in include/gs.h. Functions carry the C names
(``gs_render``, ``gs_project``, ``gs_bin``, ...) and only marshal arguments:
torch tensors become device pointers, the current torch CUDA stream becomes
the ``cudaStream_t``, and non-zero statuses become ``GSError``. Every step of
the pipeline runs in the CUDA kernels of libgs.so; if the library is not
built, importing the binding's entry points raises.

Torch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes

from . import _native as N

__all__ = ["GSError", "Context", "camera_struct", "options_struct", "gaussians_struct",
           "gs_create", "gs_destroy", "gs_project", "gs_bin", "gs_sort_pairs", "gs_tile_ranges",
           "gs_blend", "gs_render", "gs_sync_status", "gs_last_render_stats",
           "gs_set_stage_timing", "gs_last_stage_times", "gs_sort_pairs_noalloc", "gs_reserve_keys",
           "gs_render_backward", "gs_last_frame_id", "RasterizeGaussians",
           "RECORD_FLOATS"]

RECORD_FLOATS = 12  # gs_record is 48 bytes = 12 x 4-byte words


class GSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{N.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _lib():
    return N.load()


def _ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


_RAW_STREAM = None


def _stream(stream) -> int | None:
    """The cudaStream_t of a torch stream, or of the current one (read
    through torch's raw-stream query where it exists: a stream object costs
    several microseconds per call)."""
    global _RAW_STREAM
    if stream is not None:
        return int(stream.cuda_stream)
    import torch
    if _RAW_STREAM is None:
        c = torch._C
        _RAW_STREAM = ((lambda: c._cuda_getCurrentRawStream(c._cuda_getDevice()))
                       if hasattr(c, "_cuda_getCurrentRawStream") and hasattr(c, "_cuda_getDevice")
                       else (lambda: torch.cuda.current_stream().cuda_stream))
    return int(_RAW_STREAM())


def camera_struct(cam) -> N.gs_camera:
    """gs_camera from any object with world_to_cam (3x4), fx, fy, cx, cy,
    width, height, near_z (e.g. ``scenes.Camera``)."""
    import numpy as np
    c = N.gs_camera()
    c.world_to_cam[:] = np.asarray(cam.world_to_cam, dtype=np.float32).reshape(12).tolist()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near_z", 0.2))
    return c


def options_struct(tile=(16, 16), bg=(0.0, 0.0, 0.0), record_dtype: int = 0,
                   blend_variant: int = 0, deferred: bool = False, temporal: int = 0,
                   cluster: int = 0, list_tiles: int = 0, tile_order: int = 0) -> N.gs_options:
    o = N.gs_options()  # zero-filled, as gs_default_options starts; every field it sets is set below
    o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
    for i in range(3):
        o.bg[i] = float(bg[i])
    o.record_dtype = int(record_dtype)
    o.blend_variant = int(blend_variant)
    o.sync_mode = N.GS_SYNC_DEFERRED if deferred else N.GS_SYNC_FRAME
    o.temporal = int(temporal)  # False/0 off, True/1 adaptive, 2 re-bin whenever possible
    o.cluster = int(cluster)
    o.list_tiles = int(list_tiles)
    o.tile_order = int(tile_order)
    return o


def gaussians_struct(g: dict, sh_degree: int) -> N.gs_gaussians:
    """gs_gaussians from a dict of contiguous float32 CUDA tensors with keys
    means, log_scales, quats, opacity_logits, sh."""
    import torch
    s = N.gs_gaussians()
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        t = g[k]
        assert t.is_cuda and t.dtype is torch.float32 and t.is_contiguous(), k
        setattr(s, k, t.data_ptr())
    s.n = int(g["means"].shape[0])
    s.sh_degree = int(sh_degree)
    return s


class Context:
    """Owns one gs_context (workspace + device error word)."""

    def __init__(self, device: int | None = None):
        import torch
        dev = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        st = _lib().gs_create(ctypes.byref(h), dev)
        if st != N.GS_OK:
            raise GSError(st, "gs_create failed")
        self.handle = h
        self.device = dev

    def close(self):
        if getattr(self, "handle", None):
            _lib().gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status: int):
        if status != N.GS_OK:
            msg = _lib().gs_last_error(self.handle)
            raise GSError(status, msg.decode() if msg else "")

    def workspace_bytes(self) -> int:
        return int(_lib().gs_workspace_bytes(self.handle))


# ---------------------------------------------------------------------------
# Entry points (C names)
# ---------------------------------------------------------------------------

def gs_create(device: int | None = None) -> Context:
    return Context(device)


def gs_destroy(ctx: Context) -> None:
    ctx.close()


def gs_sync_status(ctx: Context, stream=None) -> None:
    ctx.check(_lib().gs_sync_status(ctx.handle, _stream(stream)))


def gs_project(ctx: Context, g: dict, sh_degree: int, cam, records, tiles, *, tile=(16, 16),
               stream=None) -> None:
    """records: (n, 12) float32 CUDA tensor (gs_record words); tiles: (n,) int32."""
    gs = gaussians_struct(g, sh_degree)
    c, o = camera_struct(cam), options_struct(tile)
    ctx.check(_lib().gs_project(ctx.handle, ctypes.byref(gs), ctypes.byref(c), ctypes.byref(o),
                                _ptr(records), _ptr(tiles), _stream(stream)))


def gs_bin(ctx: Context, records, tiles, n: int, cam, keys, values, ranges, *, tile=(16, 16),
           stream=None) -> int:
    """Returns K; raises GSError(GS_ERR_CAPACITY) with K in ``.n_keys`` if the
    key/value tensors are too small."""
    c, o = camera_struct(cam), options_struct(tile)
    nk = ctypes.c_int64(0)
    cap = 0 if keys is None else int(keys.numel())
    st = _lib().gs_bin(ctx.handle, _ptr(records), _ptr(tiles), int(n), ctypes.byref(c),
                       ctypes.byref(o), _ptr(keys), _ptr(values), cap, _ptr(ranges),
                       ctypes.byref(nk), _stream(stream))
    if st != N.GS_OK:
        msg = _lib().gs_last_error(ctx.handle)
        err = GSError(st, msg.decode() if msg else "")
        err.n_keys = int(nk.value)
        raise err
    return int(nk.value)


def gs_sort_pairs(ctx: Context, keys, values, n: int, key_bits: int, stream=None) -> None:
    ctx.check(_lib().gs_sort_pairs(ctx.handle, _ptr(keys), _ptr(values), int(n), int(key_bits),
                                   _stream(stream)))


def gs_sort_pairs_noalloc(keys, values, n: int, key_bits: int, stream=None) -> None:
    """The sort of gs_sort_pairs without a context and without any device
    allocation (scratch lives in an array inside libgs.so); for callers that
    may not allocate. n <= NOALLOC_SORT_MAX_PAIRS; calls must not overlap."""
    st = _lib().gs_sort_pairs_noalloc(_ptr(keys), _ptr(values), int(n), int(key_bits),
                                      _stream(stream))
    if st != N.GS_OK:
        raise GSError(st, "gs_sort_pairs_noalloc failed")


def gs_tile_ranges(ctx: Context, keys, n: int, n_tiles: int, ranges, stream=None) -> None:
    ctx.check(_lib().gs_tile_ranges(ctx.handle, _ptr(keys), int(n), int(n_tiles), _ptr(ranges),
                                    _stream(stream)))


def _fb(rgb, final_T=None, n_contrib=None, n_eval=None) -> N.gs_framebuffer:
    fb = N.gs_framebuffer()
    fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval = (_ptr(rgb), _ptr(final_T), _ptr(n_contrib),
                                                   _ptr(n_eval))
    return fb


def gs_blend(ctx: Context, records, values, ranges, cam, rgb, final_T=None, n_contrib=None,
             n_eval=None, *, tile=(16, 16), bg=(0.0, 0.0, 0.0), variant: int = 0,
             stream=None) -> None:
    c, o = camera_struct(cam), options_struct(tile, bg, blend_variant=variant)
    fb = _fb(rgb, final_T, n_contrib, n_eval)
    ctx.check(_lib().gs_blend(ctx.handle, _ptr(records), _ptr(values), _ptr(ranges),
                              ctypes.byref(c), ctypes.byref(o), ctypes.byref(fb), _stream(stream)))


def gs_render(ctx: Context, g: dict, sh_degree: int, cam, rgb, final_T=None, n_contrib=None,
              n_eval=None, *, tile=(16, 16), bg=(0.0, 0.0, 0.0), variant: int = 0,
              record_dtype: int = 0, deferred: bool = False, temporal: bool = False, cluster: int = 0,
              list_tiles: int = 0, tile_order: int = 0, direct: bool = False, stream=None) -> None:
    """deferred=True: GS_SYNC_DEFERRED (no host synchronisation; an overflow
    or device error is raised by a later call on the context).
    temporal=True (or 1): re-bin from the previous frame's lists when that
    measured faster (same results); 2: re-bin whenever possible.
    cluster: GS_CLUSTER_2X1 / _2X2 blend in thread-block clusters;
    list_tiles: GS_LISTS_2X1 / _2X2 / _4X4 / _8X8 lists of list tiles, read
    by every screen tile's block (no cluster);
    tile_order: GS_ORDER_LONGEST_FIRST (0) or GS_ORDER_GRID (1) blend blocks;
    direct=True: launch the kernels directly instead of replaying the
    context's CUDA graph of the frame."""
    gs = gaussians_struct(g, sh_degree)
    c, o = camera_struct(cam), options_struct(tile, bg, record_dtype, variant, deferred, temporal, cluster,
                                              list_tiles, tile_order)
    o.direct_launch = 1 if direct else 0
    fb = _fb(rgb, final_T, n_contrib, n_eval)
    ctx.check(_lib().gs_render(ctx.handle, ctypes.byref(gs), ctypes.byref(c), ctypes.byref(o),
                               ctypes.byref(fb), _stream(stream)))


def gs_render_backward(ctx: Context, g: dict, sh_degree: int, cam, final_T, n_contrib, d_rgb,
                       grads: dict, *, tile=(16, 16), bg=(0.0, 0.0, 0.0), record_dtype: int = 0,
                       cluster: int = 0, list_tiles: int = 0, stream=None) -> None:
    """grads: dict of CUDA tensors shaped like g (keys means, log_scales, quats,
    opacity_logits, sh) and optionally 'records' (n, 9)."""
    gs = gaussians_struct(g, sh_degree)
    c, o = camera_struct(cam), options_struct(tile, bg, record_dtype, cluster=cluster, list_tiles=list_tiles)
    fb = _fb(None, final_T, n_contrib, None)
    out = N.gs_grads()
    out.d_means, out.d_log_scales, out.d_quats = (_ptr(grads["means"]), _ptr(grads["log_scales"]),
                                                  _ptr(grads["quats"]))
    out.d_opacity_logits, out.d_sh = _ptr(grads["opacity_logits"]), _ptr(grads["sh"])
    out.d_records = _ptr(grads.get("records"))
    ctx.check(_lib().gs_render_backward(ctx.handle, ctypes.byref(gs), ctypes.byref(c), ctypes.byref(o),
                                        ctypes.byref(fb), _ptr(d_rgb), ctypes.byref(out),
                                        _stream(stream)))


def gs_last_render_stats(ctx: Context) -> dict:
    s = N.gs_render_stats()
    ctx.check(_lib().gs_last_render_stats(ctx.handle, ctypes.byref(s)))
    return {"n_visible": s.n_visible, "n_keys": s.n_keys, "key_bits": s.key_bits,
            "n_tiles": s.n_tiles, "n_moved": s.n_moved, "rebinned": bool(s.rebinned)}


def gs_last_frame_id(ctx: Context) -> int:
    """Number of the context's last frame a backward can differentiate (0: none)."""
    v = ctypes.c_uint64(0)
    ctx.check(_lib().gs_last_frame_id(ctx.handle, ctypes.byref(v)))
    return int(v.value)


def gs_reserve_keys(ctx: Context, key_capacity: int) -> None:
    ctx.check(_lib().gs_reserve_keys(ctx.handle, int(key_capacity)))


def gs_selftest_bounded_wait(ctx: Context, kind: int, timeout_ns: int, stream=None) -> int:
    """Runs the bounded-wait self-test and returns its raw status (expected:
    GS_ERR_TIMEOUT). Does not raise on that status."""
    return int(_lib().gs_selftest_bounded_wait(ctx.handle, int(kind), int(timeout_ns),
                                               _stream(stream)))


def gs_set_stage_timing(ctx: Context, enable: bool) -> None:
    ctx.check(_lib().gs_set_stage_timing(ctx.handle, 1 if enable else 0))


def gs_last_stage_times(ctx: Context) -> dict:
    t = N.gs_stage_times()
    ctx.check(_lib().gs_last_stage_times(ctx.handle, ctypes.byref(t)))
    return {name: float(getattr(t, name)) for name, _ in N.gs_stage_times._fields_}


# ---------------------------------------------------------------------------
# Convenience (still marshalling only)
# ---------------------------------------------------------------------------

def scene_to_device(scene, device="cuda") -> dict:
    """Copy a ``scenes.Scene`` to contiguous float32 CUDA tensors."""
    import torch
    return {k: torch.from_numpy(v).to(device=device, dtype=torch.float32).contiguous()
            for k, v in scene.arrays().items()}


def render(ctx: Context, g: dict, sh_degree: int, cam, *, tile=(16, 16), bg=(0.0, 0.0, 0.0),
           aux: bool = True, variant: int = 0, record_dtype: int = 0, deferred: bool = False,
           temporal: bool = False, cluster: int = 0, list_tiles: int = 0, tile_order: int = 0,
           direct: bool = False, stream=None) -> dict:
    """Allocate outputs with torch and call gs_render."""
    import torch
    H, W = int(cam.height), int(cam.width)
    dev = g["means"].device
    out = {"rgb": torch.empty((H, W, 3), dtype=torch.float32, device=dev)}
    if aux:
        out["final_T"] = torch.empty((H, W), dtype=torch.float32, device=dev)
        out["n_contrib"] = torch.empty((H, W), dtype=torch.int32, device=dev)
        out["n_eval"] = torch.empty((H, W), dtype=torch.int32, device=dev)
    gs_render(ctx, g, sh_degree, cam, out["rgb"], out.get("final_T"), out.get("n_contrib"),
              out.get("n_eval"), tile=tile, bg=bg, variant=variant, record_dtype=record_dtype,
              deferred=deferred, temporal=temporal, cluster=cluster, list_tiles=list_tiles,
              tile_order=tile_order, direct=direct, stream=stream)
    return out


# ---------------------------------------------------------------------------
# Autograd (marshalling only: forward -> gs_render, backward -> gs_render_backward)
# ---------------------------------------------------------------------------

def _autograd_function():
    import torch

    class _Rasterize(torch.autograd.Function):
        @staticmethod
        def forward(fctx, means, log_scales, quats, opacity_logits, sh, ctx, cam, sh_degree, tile, bg,
                    deferred, record_dtype, cluster, list_tiles):
            g = {"means": means.contiguous(), "log_scales": log_scales.contiguous(),
                 "quats": quats.contiguous(), "opacity_logits": opacity_logits.contiguous(),
                 "sh": sh.contiguous()}
            H, W = int(cam.height), int(cam.width)
            out = {"rgb": torch.empty((H, W, 3), dtype=torch.float32, device=means.device),
                   "final_T": torch.empty((H, W), dtype=torch.float32, device=means.device),
                   "n_contrib": torch.empty((H, W), dtype=torch.int32, device=means.device)}
            # The C structs are built once and kept for the backward.
            gs_s, c = gaussians_struct(g, sh_degree), camera_struct(cam)
            o = options_struct(tile, bg, record_dtype, 0, deferred, 0, cluster, list_tiles)
            fb = _fb(out["rgb"], out["final_T"], out["n_contrib"], None)
            ctx.check(_lib().gs_render(ctx.handle, ctypes.byref(gs_s), ctypes.byref(c), ctypes.byref(o),
                                       ctypes.byref(fb), _stream(None)))
            fctx.gs = (ctx, cam, sh_degree, tile, bg, g, record_dtype, deferred, cluster, list_tiles, gs_s, c, o)
            fctx.save_for_backward(out["final_T"], out["n_contrib"])
            fctx.mark_non_differentiable(out["final_T"])
            fctx.set_materialize_grads(False)  # no zero tensor for the non-differentiable final_T
            return out["rgb"], out["final_T"]

        @staticmethod
        def backward(fctx, d_rgb, d_T):
            if d_rgb is None:
                return (None,) * 14
            ctx, cam, sh_degree, tile, bg, g, record_dtype, deferred, cluster, list_tiles, gs_s, c, o = fctx.gs
            final_T, n_contrib = fctx.saved_tensors
            grads = {k: torch.empty_like(v) for k, v in g.items()}
            gr = N.gs_grads()
            gr.d_means, gr.d_log_scales, gr.d_quats = (grads["means"].data_ptr(), grads["log_scales"].data_ptr(),
                                                       grads["quats"].data_ptr())
            gr.d_opacity_logits, gr.d_sh = grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr()
            d = d_rgb.contiguous()

            def differentiate(T, nc):
                fb = _fb(None, T, nc, None)
                return _lib().gs_render_backward(ctx.handle, ctypes.byref(gs_s), ctypes.byref(c), ctypes.byref(o),
                                                 ctypes.byref(fb), d.data_ptr(), ctypes.byref(gr), _stream(None))

            st = differentiate(final_T, n_contrib)
            if st == N.GS_ERR_INVALID_ARG:
                # Another frame was rendered on the context since this one
                # (e.g. several views before one backward), which the call
                # refuses: render this frame again (the same lists, final_T
                # and n_contrib) and differentiate that.
                redo = render(ctx, g, sh_degree, cam, tile=tile, bg=bg, aux=True, record_dtype=record_dtype,
                              deferred=deferred, cluster=cluster, list_tiles=list_tiles)
                st = differentiate(redo["final_T"], redo["n_contrib"])
            ctx.check(st)
            return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"],
                    grads["sh"], None, None, None, None, None, None, None, None, None)

    return _Rasterize


_RASTERIZE = None


def RasterizeGaussians(means, log_scales, quats, opacity_logits, sh, ctx: Context, cam, sh_degree: int,
                       tile=(16, 16), bg=(0.0, 0.0, 0.0), deferred: bool = True, record_dtype: int = 0,
                       cluster: int = 0, list_tiles: int = 0):
    """Differentiable render: returns (rgb (H,W,3), final_T (H,W)); gradients
    flow to the five parameter tensors. Several renders may precede their
    backwards on one context: a backward whose frame is no longer the
    context's last renders it again first (same lists, same gradients).

    deferred=True (default) renders with GS_SYNC_DEFERRED: the forward does
    not wait for the GPU; the backward checks the forward's key count and
    raises GSError (GS_ERR_CAPACITY) if that frame overflowed its buffers,
    which have then grown, so the iteration can simply be repeated.
    record_dtype: precision of the blend records (GS_RECORD_F32 / F16 / BF16),
    used by the forward and the backward blend alike. cluster: thread-block
    clusters of the forward blend (GS_CLUSTER_*); list_tiles: lists of list
    tiles without clusters (GS_LISTS_*)."""
    global _RASTERIZE
    if _RASTERIZE is None:
        _RASTERIZE = _autograd_function()
    return _RASTERIZE.apply(means, log_scales, quats, opacity_logits, sh, ctx, cam, sh_degree,
                            tuple(tile), tuple(bg), bool(deferred), int(record_dtype), int(cluster),
                            int(list_tiles))


# ---------------------------------------------------------------------------
# Batched views (marshalling only)
# ---------------------------------------------------------------------------

def _cams_fbs(cams, outs):
    n = len(cams)
    carr = (N.gs_camera * n)(*[camera_struct(c) for c in cams])
    farr = (N.gs_framebuffer * n)(*[_fb(o["rgb"], o.get("final_T"), o.get("n_contrib"), o.get("n_eval"))
                                     for o in outs])
    return carr, farr


def alloc_outputs(cams, aux: bool = False, device="cuda") -> list:
    import torch
    outs = []
    for c in cams:
        H, W = int(c.height), int(c.width)
        o = {"rgb": torch.empty((H, W, 3), dtype=torch.float32, device=device)}
        if aux:
            o["final_T"] = torch.empty((H, W), dtype=torch.float32, device=device)
            o["n_contrib"] = torch.empty((H, W), dtype=torch.int32, device=device)
            o["n_eval"] = torch.empty((H, W), dtype=torch.int32, device=device)
        outs.append(o)
    return outs


def gs_render_batch(ctx: Context, g: dict, sh_degree: int, cams, outs, *, tile=(16, 16),
                    bg=(0.0, 0.0, 0.0), record_dtype: int = 0, direct: bool = False,
                    batch_mode: int = 0, batch_depth: int = 0, cluster: int = 0, list_tiles: int = 0,
                    stream=None):
    """batch_mode: N.GS_BATCH_AUTO (0), GS_BATCH_JOINT (1) or GS_BATCH_PER_VIEW (2);
    batch_depth: blend staging depth of the joint schedule (0 = 256);
    cluster / list_tiles: thread-block clusters of the blend, or lists of
    list tiles without clusters (the batch then renders view by view)."""
    gs = gaussians_struct(g, sh_degree)
    o = options_struct(tile, bg, record_dtype, cluster=cluster, list_tiles=list_tiles)
    o.direct_launch = 1 if direct else 0
    o.batch_mode = int(batch_mode)
    o.batch_depth = int(batch_depth)
    carr, farr = _cams_fbs(cams, outs)
    ctx.check(_lib().gs_render_batch(ctx.handle, ctypes.byref(gs), carr, len(cams), ctypes.byref(o), farr,
                                     _stream(stream)))


def gs_render_batch_backward(ctx: Context, g: dict, sh_degree: int, cams, outs, d_rgbs, grads: dict, *,
                             tile=(16, 16), bg=(0.0, 0.0, 0.0), record_dtype: int = 0, list_tiles: int = 0,
                             stream=None) -> None:
    """outs: the per-view dicts the joint gs_render_batch wrote (with final_T
    and n_contrib); d_rgbs: per-view CUDA tensors (H, W, 3); grads: dict of
    CUDA tensors shaped like g (and optionally 'records')."""
    gs = gaussians_struct(g, sh_degree)
    o = options_struct(tile, bg, record_dtype, list_tiles=list_tiles)
    carr, farr = _cams_fbs(cams, outs)
    ptrs = (ctypes.c_void_p * len(cams))(*[_ptr(d) for d in d_rgbs])
    out = N.gs_grads()
    out.d_means, out.d_log_scales, out.d_quats = (_ptr(grads["means"]), _ptr(grads["log_scales"]),
                                                  _ptr(grads["quats"]))
    out.d_opacity_logits, out.d_sh = _ptr(grads["opacity_logits"]), _ptr(grads["sh"])
    out.d_records = _ptr(grads.get("records"))
    ctx.check(_lib().gs_render_batch_backward(ctx.handle, ctypes.byref(gs), carr, len(cams), ctypes.byref(o), farr,
                                              ptrs, ctypes.byref(out), _stream(stream)))


def _batch_autograd_function():
    import torch

    class _RasterizeBatch(torch.autograd.Function):
        @staticmethod
        def forward(fctx, means, log_scales, quats, opacity_logits, sh, ctx, cams, sh_degree, tile, bg,
                    record_dtype):
            g = {"means": means.contiguous(), "log_scales": log_scales.contiguous(),
                 "quats": quats.contiguous(), "opacity_logits": opacity_logits.contiguous(),
                 "sh": sh.contiguous()}
            outs = alloc_outputs(cams, aux=True, device=means.device)
            gs_render_batch(ctx, g, sh_degree, cams, outs, tile=tile, bg=bg, record_dtype=record_dtype,
                            batch_mode=N.GS_BATCH_JOINT)
            fctx.gs = (ctx, cams, sh_degree, tile, bg, g, record_dtype, outs)
            for o in outs:
                fctx.mark_non_differentiable(o["final_T"])
            return tuple(o["rgb"] for o in outs)

        @staticmethod
        def backward(fctx, *d_rgbs):
            ctx, cams, sh_degree, tile, bg, g, record_dtype, outs = fctx.gs
            d = [x.contiguous() if x is not None else torch.zeros_like(o["rgb"]) for x, o in zip(d_rgbs, outs)]
            grads = {k: torch.empty_like(v) for k, v in g.items()}
            gs_render_batch_backward(ctx, g, sh_degree, cams, outs, d, grads, tile=tile, bg=bg,
                                     record_dtype=record_dtype)
            return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"],
                    grads["sh"], None, None, None, None, None, None)

    return _RasterizeBatch


_RASTERIZE_BATCH = None


def RasterizeGaussiansBatch(means, log_scales, quats, opacity_logits, sh, ctx: Context, cams, sh_degree: int,
                            tile=(16, 16), bg=(0.0, 0.0, 0.0), record_dtype: int = 0):
    """Differentiable joint render of several views: returns one rgb tensor
    (H, W, 3) per camera; the backward runs gs_render_batch_backward once for
    all views. The backward of a batch must run before the next batch on the
    same context."""
    global _RASTERIZE_BATCH
    if _RASTERIZE_BATCH is None:
        _RASTERIZE_BATCH = _batch_autograd_function()
    return _RASTERIZE_BATCH.apply(means, log_scales, quats, opacity_logits, sh, ctx, list(cams), sh_degree,
                                  tuple(tile), tuple(bg), int(record_dtype))


def gs_autotune_batch(ctx: Context, g: dict, sh_degree: int, cams, outs, *, bg=(0.0, 0.0, 0.0),
                      record_dtype: int = 0, cache_path: str | None = None, stream=None):
    """Runs the C autotuner (tile shapes 16x16, 16x8, 8x8, 16x16 with 2x1 and
    2x2 blend clusters, 16x16 with 2x1, 2x2, 4x4 and 8x8 list tiles and, for
    the joint schedule, staging depths 256, 128, 64) and returns ((tile_w,
    tile_h), [ms per candidate], depth, cluster, list_tiles).
    With cache_path, results are kept in a JSON file keyed by GPU, scene
    size, view sizes and record precision."""
    import json
    import os
    import torch
    key = None
    if cache_path:
        sizes = ",".join(f"{c.width}x{c.height}" for c in cams)
        n = int(g["means"].shape[0])
        key = f"{torch.cuda.get_device_name()}|n{n}|d{sh_degree}|{sizes}|r{record_dtype}"
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache and "list_tiles" in cache[key]:
                return (tuple(cache[key]["tile"]), cache[key]["ms"], cache[key].get("depth", 256),
                        cache[key]["cluster"], cache[key]["list_tiles"])
    gs = gaussians_struct(g, sh_degree)
    o = options_struct((16, 16), bg, record_dtype)
    carr, farr = _cams_fbs(cams, outs)
    ms = (ctypes.c_float * 9)()
    ctx.check(_lib().gs_autotune_batch(ctx.handle, ctypes.byref(gs), carr, len(cams), ctypes.byref(o), farr,
                                       _stream(stream), ms))
    tile, times, depth = (int(o.tile_w), int(o.tile_h)), [float(x) for x in ms], int(o.batch_depth)
    cluster, list_tiles = int(o.cluster), int(o.list_tiles)
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[key] = {"tile": list(tile), "ms": times, "depth": depth, "cluster": cluster,
                      "list_tiles": list_tiles}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return tile, times, depth, cluster, list_tiles
