"""ctypes mirror of include/gs.h and loader of the in-tree libgs.so.

Nothing here computes: the structures copy the header's layouts and every
function forwards to the C entry point of the same name. Loading fails
loudly when the library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")

GS_OK = 0
GS_ERR_INVALID_ARG = 1
GS_ERR_CUDA = 2
GS_ERR_OOM = 3
GS_ERR_CAPACITY = 4
GS_ERR_TIMEOUT = 5
GS_ERR_UNSUPPORTED = 6
GS_RECORD_F32 = 0
GS_RECORD_F16 = 1
GS_RECORD_BF16 = 2
GS_BLEND_CULLED = 0
GS_BLEND_BASIC = 1
GS_BLEND_CULLED_WIDE = 2
GS_BLEND_CULLED_TILE = 3
GS_BLEND_CULLED_8X8 = 4
GS_BLEND_TMA = 5
GS_SYNC_FRAME = 0
GS_SYNC_DEFERRED = 1
GS_BATCH_AUTO = 0
GS_BATCH_JOINT = 1
GS_BATCH_PER_VIEW = 2
GS_CLUSTER_NONE = 0
GS_CLUSTER_2X1 = 2
GS_CLUSTER_2X2 = 4
GS_LISTS_1X1 = 0
GS_LISTS_2X1 = 2
GS_LISTS_2X2 = 4
GS_LISTS_4X4 = 16
GS_LISTS_8X8 = 64
GS_ORDER_LONGEST_FIRST = 0
GS_ORDER_GRID = 1
NOALLOC_SORT_MAX_PAIRS = 262144  # GS_NOALLOC_SORT_MAX_PAIRS in include/gs.h
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_OOM",
                4: "GS_ERR_CAPACITY", 5: "GS_ERR_TIMEOUT", 6: "GS_ERR_UNSUPPORTED"}

c_float_p = ctypes.POINTER(ctypes.c_float)
vp = ctypes.c_void_p


class gs_gaussians(ctypes.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp),
                ("sh", vp), ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32)]


class gs_camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_float * 12), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("near_z", ctypes.c_float)]


class gs_record(ctypes.Structure):
    _fields_ = [("mean2d", ctypes.c_float * 2), ("conic", ctypes.c_float * 3),
                ("opacity", ctypes.c_float), ("rgb", ctypes.c_float * 3),
                ("depth", ctypes.c_float), ("radius", ctypes.c_int32),
                ("tiles", ctypes.c_uint32)]


class gs_framebuffer(ctypes.Structure):
    _fields_ = [("rgb", vp), ("final_T", vp), ("n_contrib", vp), ("n_eval", vp)]


class gs_grads(ctypes.Structure):
    _fields_ = [("d_means", vp), ("d_log_scales", vp), ("d_quats", vp), ("d_opacity_logits", vp),
                ("d_sh", vp), ("d_records", vp)]


class gs_options(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("bg", ctypes.c_float * 3), ("record_dtype", ctypes.c_int32),
                ("blend_variant", ctypes.c_int32), ("direct_launch", ctypes.c_int32),
                ("sync_mode", ctypes.c_int32), ("temporal", ctypes.c_int32),
                ("batch_mode", ctypes.c_int32), ("batch_depth", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("list_tiles", ctypes.c_int32),
                ("tile_order", ctypes.c_int32)]


class gs_render_stats(ctypes.Structure):
    _fields_ = [("n_visible", ctypes.c_int64), ("n_keys", ctypes.c_int64),
                ("key_bits", ctypes.c_int32), ("n_tiles", ctypes.c_int32),
                ("n_moved", ctypes.c_int64), ("rebinned", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gs_stage_times(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("project_ms", "depth_sort_ms", "entry_scan_ms", "emit_ms",
                                              "tile_sort_ms", "ranges_ms", "blend_ms", "total_ms")]


assert ctypes.sizeof(gs_record) == 48

# name -> (restype, argtypes); every symbol include/gs.h declares.
SIGNATURES = {
    "gs_default_options": (None, [ctypes.POINTER(gs_options)]),
    "gs_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int]),
    "gs_destroy": (None, [vp]),
    "gs_last_error": (ctypes.c_char_p, [vp]),
    "gs_sync_status": (ctypes.c_int, [vp, vp]),
    "gs_workspace_bytes": (ctypes.c_size_t, [vp]),
    "gs_project": (ctypes.c_int, [vp, ctypes.POINTER(gs_gaussians), ctypes.POINTER(gs_camera),
                                  ctypes.POINTER(gs_options), vp, vp, vp]),
    "gs_bin": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(gs_camera),
                              ctypes.POINTER(gs_options), vp, vp, ctypes.c_int64, vp,
                              ctypes.POINTER(ctypes.c_int64), vp]),
    "gs_sort_pairs": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, ctypes.c_int32, vp]),
    "gs_sort_pairs_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_int64, ctypes.c_int32, vp]),
    "gs_tile_ranges": (ctypes.c_int, [vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp]),
    "gs_blend": (ctypes.c_int, [vp, vp, vp, vp, ctypes.POINTER(gs_camera),
                                ctypes.POINTER(gs_options), ctypes.POINTER(gs_framebuffer), vp]),
    "gs_render": (ctypes.c_int, [vp, ctypes.POINTER(gs_gaussians), ctypes.POINTER(gs_camera),
                                 ctypes.POINTER(gs_options), ctypes.POINTER(gs_framebuffer), vp]),
    "gs_last_render_stats": (ctypes.c_int, [vp, ctypes.POINTER(gs_render_stats)]),
    "gs_last_frame_id": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_uint64)]),
    "gs_reserve_keys": (ctypes.c_int, [vp, ctypes.c_int64]),
    "gs_render_batch_backward": (ctypes.c_int, [vp, ctypes.POINTER(gs_gaussians), ctypes.POINTER(gs_camera),
                                                ctypes.c_int32, ctypes.POINTER(gs_options),
                                                ctypes.POINTER(gs_framebuffer), ctypes.POINTER(vp),
                                                ctypes.POINTER(gs_grads), vp]),
    "gs_selftest_bounded_wait": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int64, vp]),
    "gs_render_batch": (ctypes.c_int, [vp, ctypes.POINTER(gs_gaussians), ctypes.POINTER(gs_camera),
                                       ctypes.c_int32, ctypes.POINTER(gs_options),
                                       ctypes.POINTER(gs_framebuffer), vp]),
    "gs_autotune_batch": (ctypes.c_int, [vp, ctypes.POINTER(gs_gaussians), ctypes.POINTER(gs_camera),
                                         ctypes.c_int32, ctypes.POINTER(gs_options),
                                         ctypes.POINTER(gs_framebuffer), vp,
                                         ctypes.POINTER(ctypes.c_float)]),
    "gs_render_backward": (ctypes.c_int, [vp, ctypes.POINTER(gs_gaussians), ctypes.POINTER(gs_camera),
                                          ctypes.POINTER(gs_options), ctypes.POINTER(gs_framebuffer),
                                          vp, ctypes.POINTER(gs_grads), vp]),
    "gs_set_stage_timing": (ctypes.c_int, [vp, ctypes.c_int]),
    "gs_last_stage_times": (ctypes.c_int, [vp, ctypes.POINTER(gs_stage_times)]),
}

_lib = None


def load(path: str | None = None):
    """Load libgs.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libgs.so not built at {p}; run paper_2607_15951_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def declared_symbols(header: str) -> list[str]:
    """Function names declared in a C header (used by the export test)."""
    import re
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_]+)\s*\(", src)))
