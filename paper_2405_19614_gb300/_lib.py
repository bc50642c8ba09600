"""ctypes view of the C ABI in include/gs.h (argument marshalling only).

Loading fails loudly when libgs.so has not been built: there is no CPU or
eager fallback for any step of the path.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgs.so")

c_f, c_i32, c_i64, c_p, c_sz = ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t

GS_MAX_VIEWS = 64
GS_TILE = 16  # default tile side
TILE_SIDES = (8, 16, 32, 64)
N_BAND_VARIANTS = 6
VARIANT_PPT = (1, 2, 2, 4, 4, 8)
VARIANT_BW = (8, 8, 16, 8, 16, 16)
GS_MAX_ADAM_GROUPS = 8
STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_CAPACITY", 4: "GS_ERR_TIMEOUT",
          5: "GS_ERR_UNSUPPORTED"}
ERR_CAPACITY, ERR_TIMEOUT = 3, 4
GS_OP_BIN_SORT, GS_OP_GRAD2D, GS_OP_SSIM, GS_OP_SELECT, GS_OP_SPATIAL_ORDER, GS_OP_CHECK_LOOKBACK = range(6)


class GsView(ctypes.Structure):
    _fields_ = [("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f), ("width", c_i32), ("height", c_i32),
                ("tile_w", c_i32), ("tile_h", c_i32)]


class GsParams(ctypes.Structure):
    _fields_ = [("means", c_p), ("log_scales", c_p), ("quats", c_p), ("opacity_logit", c_p), ("sh", c_p),
                ("n", c_i64), ("sh_degree", c_i32)]


class GsParamGrads(ctypes.Structure):
    _fields_ = [("means", c_p), ("log_scales", c_p), ("quats", c_p), ("opacity_logit", c_p), ("sh", c_p)]


class GsOptions(ctypes.Structure):
    _fields_ = [("near_z", c_f), ("blur", c_f), ("overwrite_grads", c_i32)]


class GsProjected(ctypes.Structure):
    _fields_ = [("rec", c_p), ("rect", c_p), ("radii", c_p), ("tiles_touched", c_p), ("tile_mask", c_p)]


class GsBins(ctypes.Structure):
    _fields_ = [("keys", c_p), ("vals", c_p), ("ranges", c_p), ("n_pairs", c_p), ("status", c_p),
                ("capacity", c_i64)]


class GsImage(ctypes.Structure):
    _fields_ = [("rgb", c_p), ("depth", c_p), ("alpha", c_p), ("final_T", c_p), ("n_contrib", c_p)]


class GsRows(ctypes.Structure):
    _fields_ = [("src", c_p), ("dst", c_p), ("row_floats", c_i32)]


class GsAdamGroup(ctypes.Structure):
    _fields_ = [("offset", c_i64), ("count", c_i64), ("lr", c_f)]


P = ctypes.POINTER
SIGNATURES = {
    "gs_version": ([], ctypes.c_char_p),
    "gs_status_string": ([c_i32], ctypes.c_char_p),
    "gs_layout": ([P(GsView), c_i32, P(c_i64), P(c_i64)], c_i32),
    "gs_project": ([P(GsParams), P(GsView), c_p, c_i32, P(GsOptions), P(GsProjected), c_p], c_i32),
    "gs_bin_sort_workspace_size": ([c_i64, c_i64, c_i64], c_sz),
    "gs_bin_sort": ([P(GsProjected), c_i64, P(GsView), c_i32, P(GsBins), c_p, c_sz, c_p], c_i32),
    "gs_bin_sort_noalloc": ([P(GsProjected), c_i64, P(GsView), c_i32, P(GsBins), c_p], c_i32),
    "gs_render_fwd": ([P(GsProjected), c_i64, P(GsBins), P(GsView), c_i32, P(GsImage), c_p, c_p], c_i32),
    "gs_render_fwd_l1": ([P(GsProjected), c_i64, P(GsBins), P(GsView), c_i32, P(GsImage), c_p, c_p, c_p, c_f, c_f,
                          c_i32, c_f, c_p, c_p, c_p, c_p], c_i32),
    "gs_render_stats": ([P(GsProjected), c_i64, P(GsBins), P(GsView), c_i32, c_p, c_p, c_p, c_p], c_i32),
    "gs_set_render_variants": ([c_i32, c_i32], c_i32),
    "gs_get_render_variants": ([P(c_i32), P(c_i32), P(c_i32), P(c_i32)], c_i32),
    "gs_decode_keyframes": ([c_p, c_p, c_i64, c_f, c_p, c_p, c_p], c_i32),
    "gs_loss_l1": ([c_p, c_p, c_p, c_p, c_p, c_i64, c_f, c_f, c_i32, c_f, c_p, c_p, c_p, c_p], c_i32),
    "gs_ssim_workspace_size": ([c_i64], c_sz),
    "gs_loss_ssim": ([c_p, c_p, P(GsView), c_i32, c_f, c_p, c_p, c_p, c_sz, c_p, c_p], c_i32),
    "gs_check_ssim_timeout": ([c_p, c_p, P(GsView), c_i32, c_p, c_p, c_p, c_sz, c_p, c_p], c_i32),
    "gs_grad2d_size": ([c_i64, c_i32], c_sz),
    "gs_render_bwd_splats": ([P(GsProjected), c_i64, P(GsBins), P(GsView), c_i32, P(GsImage), c_p, c_p, c_p,
                              c_p, c_p, c_p], c_i32),
    "gs_project_bwd": ([P(GsParams), P(GsView), c_p, c_i32, P(GsOptions), P(GsProjected), c_p, P(GsParamGrads),
                        c_p, c_p], c_i32),
    "gs_render_bwd": ([P(GsParams), P(GsView), c_p, c_i32, P(GsOptions), P(GsProjected), P(GsBins), P(GsImage),
                       c_p, c_p, c_p, c_p, P(GsParamGrads), c_p, c_p, c_p], c_i32),
    "gs_reproj_loss_grad": ([c_p, c_p, c_p, c_i64, P(GsView), c_p, c_i32, c_f, c_f, c_p, c_p, c_p], c_i32),
    "gs_adam_step": ([c_p, c_p, c_p, c_p, P(GsAdamGroup), c_i32, c_f, c_f, c_f, c_p, c_p], c_i32),
    "gs_pose_update": ([c_p, c_p, c_i32, c_p], c_i32),
    "gs_select_workspace_size": ([c_i64], c_sz),
    "gs_densify": ([c_p, c_p, c_p, P(GsView), c_p, c_i32, c_f, c_f, P(GsParamGrads), c_i32, c_i64, c_i64, c_p, c_p,
                    c_p, c_sz, c_p], c_i32),
    "gs_prune_select": ([c_p, c_i64, c_f, c_p, c_p, c_p, c_sz, c_p], c_i32),
    "gs_compact_rows": ([c_p, c_i64, P(GsRows), c_i32, c_p], c_i32),
    "gs_spatial_order_workspace_size": ([c_i64], c_sz),
    "gs_spatial_order": ([c_p, c_i64, c_p, c_p, c_sz, c_p, c_p], c_i32),
    "gs_select_views": ([c_p, c_p, c_i32, c_f, c_i32, c_p], c_i32),
    "gs_get_device_status": ([c_p, c_p, c_p], c_i32),
    "gs_workspace_size": ([c_i32, c_i64, c_i32, c_i64, c_i64], c_sz),
    "gs_check_lookback_timeout_workspace_size": ([], c_sz),
    "gs_check_lookback_timeout": ([ctypes.c_uint32, c_i32, c_p, c_p, c_sz, c_p], c_i32),
}

_lib = None


class GsError(RuntimeError):
    pass


def load():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GsError(f"{LIB_PATH} is missing: build it with paper_2405_19614_gb300.build.build() "
                          "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def check(code: int, what: str):
    if code != 0:
        raise GsError(f"{what}: {STATUS.get(code, code)}")
