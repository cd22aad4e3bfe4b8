"""ctypes binding of the C ABI in ``include/gs.h`` (argument marshalling only).

The library is loaded from the in-tree build (``_build/libgs_gb300.so``). If it
is missing, ``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

GS_OK = 0
GS_ERR_ARG = -1
GS_ERR_OOM = -2
GS_ERR_CAPACITY = -3
GS_ERR_CUDA = -4
GS_ERR_TIMEOUT = -5
GS_ERR_NONFINITE = -6
GS_ERR_STATE = -7
GS_ERR_IO = -8
GS_MAX_VIEWS = 16

ERR_NAMES = {GS_ERR_ARG: "GS_ERR_ARG", GS_ERR_OOM: "GS_ERR_OOM", GS_ERR_CAPACITY: "GS_ERR_CAPACITY",
             GS_ERR_CUDA: "GS_ERR_CUDA", GS_ERR_TIMEOUT: "GS_ERR_TIMEOUT", GS_ERR_NONFINITE: "GS_ERR_NONFINITE",
             GS_ERR_STATE: "GS_ERR_STATE", GS_ERR_IO: "GS_ERR_IO"}


class gs_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3)]


class gs_config(C.Structure):
    _fields_ = [("near_z", C.c_float), ("fov_clamp", C.c_float), ("dilation", C.c_float),
                ("lambda_floor", C.c_float), ("radius_sigma", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("T_min", C.c_float), ("lambda_color", C.c_float),
                ("lambda_reg", C.c_float), ("reg_floor", C.c_float), ("lambda_photo", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("lr", C.c_float * 5), ("split_thresh", C.c_float),
                ("split_factor", C.c_float), ("insert_opacity", C.c_float), ("insert_tau", C.c_float),
                ("clarity_sigma", C.c_float), ("tile_size", C.c_int32), ("pixels_per_thread", C.c_int32),
                ("capacity", C.c_int32), ("max_views", C.c_int32), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("pair_capacity", C.c_int64), ("seed", C.c_uint64),
                ("deterministic", C.c_int32)]


_P = C.c_void_p
_I = C.c_int
SIGNATURES = {
    "gs_default_config": (None, [C.POINTER(gs_config)]),
    "gs_create": (_I, [C.POINTER(gs_config), _I, C.POINTER(_P)]),
    "gs_destroy": (None, [_P]),
    "gs_last_error": (C.c_char_p, [_P]),
    "gs_num_gaussians": (_I, [_P]),
    "gs_set_params": (_I, [_P, _P, _I, _P]),
    "gs_get_params": (_I, [_P, _P, _P]),
    "gs_get_grads": (_I, [_P, _P, _P]),
    "gs_set_grads": (_I, [_P, _P, _P]),
    "gs_init_map": (_I, [_P, _P, _P, _I, _P]),
    "gs_render": (_I, [_P, C.POINTER(gs_camera), _I, _P, _P, _P, _P]),
    "gs_loss": (_I, [_P, _P, _P, _P]),
    "gs_backward": (_I, [_P, _P, _P]),
    "gs_step": (_I, [_P, _P]),
    "gs_iterate": (_I, [_P, C.POINTER(gs_camera), _I, _P, _P, _P, _P]),
    "gs_iterate_host": (_I, [_P, C.POINTER(gs_camera), _I, _P, _P, _P, _P]),
    "gs_count_dominant": (_I, [_P, C.POINTER(gs_camera), _I, _P]),
    "gs_timing_phases": (_I, [_P, C.c_uint32]),
    "gs_insert": (_I, [_P, C.POINTER(gs_camera), _P, _P, _I, C.POINTER(_I), _P, _P]),
    "gs_densify": (_I, [_P, _P, C.POINTER(_I), _P]),
    "gs_debug_projection": (_I, [_P, _I, _P]),
    "gs_debug_pairs": (_I, [_P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "gs_debug_grad2d": (_I, [_P, _P]),
    "gs_tile_size": (_I, [_P]),
    "gs_pixels_per_thread": (_I, [_P]),
    "gs_timing_enable": (_I, [_P, _I]),
    "gs_timing_read": (_I, [_P, _P, _P]),
    "gs_debug_work": (_I, [_P, _P]),
    "gs_launch_count": (C.c_int64, [_P]),
    "gs_sort_pairs_static": (_I, [_P, _P, _P, _P, C.c_int64, _I, _P]),
    "gs_save": (_I, [_P, C.c_char_p, _P]),
    "gs_load": (_I, [_P, C.c_char_p, _P]),
    "gs_checkpoint_info": (_I, [C.c_char_p, C.POINTER(_I), C.POINTER(_I)]),
    "gs_mlp_create": (_I, [_I, C.c_uint64, C.POINTER(_P)]),
    "gs_mlp_destroy": (None, [_P]),
    "gs_mlp_num_params": (_I, []),
    "gs_mlp_set_params": (_I, [_P, _P, _P]),
    "gs_mlp_get_params": (_I, [_P, _P, _P]),
    "gs_mlp_get_grads": (_I, [_P, _P, _P]),
    "gs_mlp_features": (_I, [C.POINTER(gs_camera), _P, _P, _I, _P, _P]),
    "gs_mlp_forward": (_I, [_P, _P, _I, _P, _P]),
    "gs_mlp_backward": (_I, [_P, _P, _P, _I, _P, _P]),
    "gs_mlp_step": (_I, [_P, C.c_float, _P]),
    "gs_set_initializer": (_I, [_P, _P]),
    "gs_mlp_targets": (_I, [_P, _I, _I, _P, _P]),
    "gs_psnr": (_I, [_P, _P, _P, C.c_int64, _P, _P]),
}
PHASES = ("project", "bin", "raster_fwd", "loss", "raster_bwd", "project_bwd", "adam", "raster_fused")

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class GSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, ctx=None):
    if code != GS_OK:
        msg = load().gs_last_error(ctx).decode() if ctx else ""
        raise GSError(code, msg)
