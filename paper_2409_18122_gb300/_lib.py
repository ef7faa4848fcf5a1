"""ctypes binding of libgs103.so (the C ABI declared in include/gs.h).

Argument marshalling only: struct layouts mirror include/gs.h field for field
and every function is bound with its exact prototype.  There is no fallback:
if the library is missing or fails to load, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_float, c_int32, c_int64, c_size_t, c_uint32, c_void_p, POINTER

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgs103.so")

# status codes and device flags (include/gs.h)
GS_OK, GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA, GS_ERR_DEVICE = range(7)
GS_FLAG_PAIR_OVERFLOW = 1 << 0
GS_FLAG_RANGE_OVERFLOW = 1 << 1
GS_FLAG_BAD_CAMERA = 1 << 2
GS_FLAG_NONFINITE = 1 << 3
GS_FLAG_RECORD_OVERFLOW = 1 << 4
GS_FLAG_BAD_RECORDS = 1 << 5
GS_FLAG_ERROR_MASK = (GS_FLAG_PAIR_OVERFLOW | GS_FLAG_RANGE_OVERFLOW | GS_FLAG_BAD_CAMERA | GS_FLAG_RECORD_OVERFLOW
                      | GS_FLAG_BAD_RECORDS)
GS_IG_RENDER_MEAN = 0
(GS_OP_PROJECT, GS_OP_BIN_SORT, GS_OP_RENDER_BWD, GS_OP_INFO_GAIN, GS_OP_IG_COMPOSITE, GS_OP_THRESHOLDS,
 GS_OP_VIEW_UTILITY, GS_OP_REGIONS, GS_OP_TRAJECTORY) = range(9)
GS_U_ABS, GS_U_SQ = 0, 1
GS_XI, GS_XI_SUM = 0, 1
GS_NOALLOC_MAX_RECORDS = 1 << 18
GS_SMALL_MAX_GAUSSIANS = 1 << 16
GS_SMALL_MAX_VIEWS = 64
GS_SMALL_MAX_LIST = 2048


class gs_camera(ctypes.Structure):
    _fields_ = [("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32), ("R", c_float * 9), ("T", c_float * 3),
                ("tile_w", c_int32), ("tile_h", c_int32)]


class gs_map(ctypes.Structure):
    _fields_ = [("mo", c_void_p), ("su", c_void_p), ("q", c_void_p), ("rgb", c_void_p), ("n", c_int64)]


class gs_params(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("eps2d", c_float), ("near_plane", c_float),
                ("guard", c_float), ("alpha_min", c_float), ("alpha_max", c_float), ("T_min", c_float),
                ("ig_batch", c_int32), ("fwd_batch", c_int32)]


class gs_proj(ctypes.Structure):
    _fields_ = [("capacity", c_int64), ("count", c_void_p), ("status", c_void_p), ("view_info", c_void_p),
                ("gid", c_void_p), ("view", c_void_p), ("splat", c_void_p), ("color_d", c_void_p),
                ("rect", c_void_p), ("depth_key", c_void_p), ("grp_mask", c_void_p), ("grp_base", c_void_p)]


class gs_bins(ctypes.Structure):
    _fields_ = [("pair_capacity", c_int64), ("tile_capacity", c_int64), ("count", c_void_p), ("tile", c_void_p),
                ("rec", c_void_p), ("ranges", c_void_p), ("item_order", c_void_p), ("item_capacity", c_int64)]


class gs_utility_params(ctypes.Structure):
    _fields_ = [("near_plane", c_float), ("range", c_float), ("lambda", c_float), ("ground_z", c_float)]


class gs_region_grid(ctypes.Structure):
    _fields_ = [("origin", c_float * 3), ("size", c_float), ("dims", c_int32 * 3)]


class gs_loss_weights(ctypes.Structure):
    _fields_ = [("w_depth", c_float), ("w_rgb", c_float), ("w_ssim", c_float)]


class gs_adam_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


GS_ADAM_MAX_TENSORS = 8


class gs_image(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("unc", c_void_p), ("T", c_void_p), ("last", c_void_p),
                ("n_contrib", c_void_p)]


class gs_image_grad(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p)]


class gs_map_grad(ctypes.Structure):
    _fields_ = [("dmo", c_void_p), ("dsu", c_void_p), ("dq", c_void_p), ("drgb", c_void_p)]


assert ctypes.sizeof(gs_camera) == 80
assert ctypes.sizeof(gs_params) == 40
assert ctypes.sizeof(gs_bins) == 64

# name -> (restype, argtypes); the exported C ABI
PROTOTYPES = {
    "gs_uncertainty_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    "gs_uncertainty_thresholds": (c_int32, [POINTER(gs_map), c_float, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_view_utility_batch": (c_int32, [POINTER(gs_map), c_void_p, c_int32, POINTER(gs_utility_params), c_int32,
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_region_uncertainty": (c_int32, [POINTER(gs_map), POINTER(gs_region_grid), c_void_p, c_void_p, c_void_p,
                                        c_size_t, c_void_p]),
    "gs_trajectory_utility": (c_int32, [POINTER(gs_map), c_void_p, c_int32, c_int32, POINTER(gs_utility_params),
                                        c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_collision_check": (c_int32, [POINTER(gs_map), c_void_p, c_int32, c_float, c_float, c_float, c_void_p,
                                     c_void_p, c_void_p]),
    "gs_image_loss": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(gs_loss_weights),
                                c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_image_loss_workspace_size": (c_int32, [c_void_p, c_int32, POINTER(c_size_t)]),
    "gs_adam_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, POINTER(gs_adam_params),
                               c_void_p, c_void_p]),
    "gs_project": (c_int32, [POINTER(gs_map), c_void_p, c_int32, POINTER(gs_params), POINTER(gs_proj), c_void_p,
                             c_size_t, c_void_p]),
    "gs_bin_sort": (c_int32, [POINTER(gs_proj), c_void_p, c_int32, POINTER(gs_params), POINTER(gs_bins), c_void_p,
                              c_size_t, c_void_p]),
    "gs_render_fwd": (c_int32, [POINTER(gs_map), POINTER(gs_proj), POINTER(gs_bins), c_void_p, c_int32,
                                POINTER(gs_params), POINTER(gs_image), c_void_p]),
    "gs_render_small": (c_int32, [POINTER(gs_map), c_void_p, c_int32, POINTER(gs_params), POINTER(gs_image),
                                  c_void_p, c_void_p]),
    "gs_render_bwd": (c_int32, [POINTER(gs_map), POINTER(gs_proj), POINTER(gs_bins), POINTER(gs_image),
                                POINTER(gs_image_grad), c_void_p, c_int32, POINTER(gs_params), POINTER(gs_map_grad),
                                c_void_p, c_size_t, c_void_p]),
    "gs_render_bwd_noalloc": (c_int32, [POINTER(gs_map), POINTER(gs_proj), POINTER(gs_bins), POINTER(gs_image),
                                        POINTER(gs_image_grad), c_void_p, c_int32, POINTER(gs_params),
                                        POINTER(gs_map_grad), c_void_p]),
    "gs_info_gain_batch": (c_int32, [POINTER(gs_map), c_void_p, c_int32, POINTER(gs_params), c_int32, c_void_p,
                                     c_void_p, c_int64, c_int64, c_int64, c_void_p, c_size_t, c_void_p]),
    "gs_info_gain_composite": (c_int32, [POINTER(gs_proj), POINTER(gs_bins), c_void_p, c_int32, POINTER(gs_params),
                                         c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_workspace_size": (c_int32, [c_int32, c_int64, c_int32, c_int64, c_int64, c_int64, POINTER(c_size_t)]),
    "gs_read_status": (c_int32, [c_void_p, POINTER(c_uint32)]),
    "gs_status_str": (ctypes.c_char_p, [c_int32]),
    "gs_version": (ctypes.c_char_p, []),
    "gs_kernel_launches": (ctypes.c_uint64, []),
}

_lib = None


class GSError(RuntimeError):
    pass


def lib():
    """Load libgs103.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GSError("libgs103.so is not built (expected at %s); run `python -c \"import __graft_entry__ as g; "
                          "g.build()\"`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str):
    if status != GS_OK:
        msg = lib().gs_status_str(status).decode()
        raise GSError("%s failed: %s" % (what, msg))


def workspace_size(op: int, n: int, n_views: int, rec_cap: int = 0, pair_cap: int = 0, tile_cap: int = 0) -> int:
    out = c_size_t(0)
    check(lib().gs_workspace_size(op, n, n_views, rec_cap, pair_cap, tile_cap, ctypes.byref(out)),
          "gs_workspace_size")
    return int(out.value)
