"""ctypes declarations of the C ABI in include/nrm.h (argument marshalling only).

``load()`` returns the shared library, building it in-tree first when a source
is newer than ``_build/libnrm.so``. There is no fallback: if the library cannot
be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

NRM_OK = 0
NRM_ERR_INVALID_ARG = 1
NRM_ERR_UNSUPPORTED = 2
NRM_ERR_CUDA = 3
NRM_ERR_OOM = 4
NRM_ERR_TIMEOUT = 5
NRM_ERR_NO_DEVICE = 6
NRM_ERR_BOUNDS = 7

NRM_IN_F32_M, NRM_IN_U16_MM = 0, 1
NRM_OUT_F32X4, NRM_OUT_F16X4, NRM_OUT_OCT16 = 0, 1, 2
NRM_MASK_RAW, NRM_MASK_SECANT = 0, 1
NRM_MAX_ALPHA = 16
NRM_NOALLOC_MAX_FRAMES = 256
NRM_MAX_PLANE_RADIUS = 4


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int), ("mask_mode", ctypes.c_int), ("tau", ctypes.c_float),
                ("depth_scale", ctypes.c_float), ("in_dtype", ctypes.c_int),
                ("out_dtype", ctypes.c_int), ("orient_to_camera", ctypes.c_int)]


class Frame(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_void_p), ("normals", ctypes.c_void_p),
                ("valid", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("depth_pitch", ctypes.c_longlong), ("out_pitch", ctypes.c_longlong),
                ("K", Intrinsics), ("in_dtype", ctypes.c_int), ("points", ctypes.c_void_p)]


class GradFrame(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_void_p), ("grad_normals", ctypes.c_void_p),
                ("valid", ctypes.c_void_p), ("grad_depth", ctypes.c_void_p),
                ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("depth_pitch", ctypes.c_longlong), ("out_pitch", ctypes.c_longlong),
                ("K", Intrinsics)]


class TileConfig(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("threads", ctypes.c_int),
                ("stages", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


NRM_MAX_SCALES = 8
NRM_MS_PAIR, NRM_MS_QUAD = 0, 1


class Scales(ctypes.Structure):
    _fields_ = [("n_scales", ctypes.c_int), ("alpha", ctypes.c_int * NRM_MAX_SCALES), ("form", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("kernel_ms", ctypes.c_double),
                ("tiles", ctypes.c_longlong)]


# (name, restype, argtypes) of every function declared in include/nrm.h.
_H = ctypes.c_void_p
_S = ctypes.c_void_p  # cudaStream_t
SIGNATURES = [
    ("nrm_default_params", None, [ctypes.POINTER(Params)]),
    ("nrm_create", ctypes.c_int, [ctypes.POINTER(Intrinsics), ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(Params), ctypes.POINTER(_H)]),
    ("nrm_destroy", None, [_H]),
    ("nrm_estimate", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _S]),
    ("nrm_estimate_points", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, _S]),
    ("nrm_estimate_batched", ctypes.c_int, [_H, ctypes.POINTER(Frame), ctypes.c_int, _S]),
    ("nrm_backward", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, _S]),
    ("nrm_backward_batched", ctypes.c_int, [_H, ctypes.POINTER(GradFrame), ctypes.c_int, _S]),
    ("nrm_backward_batched_scaled", ctypes.c_int, [_H, ctypes.POINTER(GradFrame), ctypes.c_int, ctypes.c_void_p,
                                                   _S]),
    ("nrm_cosine_loss_scale", ctypes.c_int, [_H, ctypes.POINTER(GradFrame), ctypes.c_int, ctypes.c_void_p, _S]),
    ("nrm_spherical", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, _S]),
    ("nrm_angle_mse", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, _S]),
    ("nrm_estimate_multiscale", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(Scales), _S]),
    ("nrm_estimate_batched_host", ctypes.c_int, [_H, ctypes.POINTER(Frame), ctypes.c_int, _S]),
    ("nrm_estimate_batched_multiscale", ctypes.c_int, [_H, ctypes.POINTER(Frame), ctypes.c_int,
                                                       ctypes.POINTER(Scales), _S]),
    ("nrm_plane_fit", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _S]),
    ("nrm_selftest_wait_expiry", ctypes.c_int, [ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_float)]),
    ("nrm_selftest_bounds", ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    ("nrm_sync_status", ctypes.c_int, [_H]),
    ("nrm_get_config", ctypes.c_int, [_H, ctypes.POINTER(TileConfig)]),
    ("nrm_set_config", ctypes.c_int, [_H, ctypes.POINTER(TileConfig)]),
    ("nrm_autotune", ctypes.c_int, [_H, ctypes.POINTER(Frame), ctypes.c_int, _S, ctypes.c_char_p]),
    ("nrm_set_autotune_cache", ctypes.c_int, [ctypes.c_char_p]),
    ("nrm_autotune_key", ctypes.c_int, [_H, ctypes.c_char_p, ctypes.c_int]),
    ("nrm_autotune_cache_get", ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(TileConfig)]),
    ("nrm_autotune_cache_put", ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(TileConfig)]),
    ("nrm_enable_timing", ctypes.c_int, [_H, ctypes.c_int]),
    ("nrm_get_stats", ctypes.c_int, [_H, ctypes.POINTER(Stats)]),
    ("nrm_reset_stats", ctypes.c_int, [_H]),
    ("nrm_estimate_batched_noalloc", ctypes.c_int, [ctypes.POINTER(Frame), ctypes.c_int,
                                                    ctypes.POINTER(Params), ctypes.c_void_p, _S]),
    ("nrm_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("nrm_last_error", ctypes.c_char_p, []),
    ("nrm_version", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


class NrmError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {message} ({status_name(status)})")


def status_name(code: int) -> str:
    names = {0: "NRM_OK", 1: "NRM_ERR_INVALID_ARG", 2: "NRM_ERR_UNSUPPORTED", 3: "NRM_ERR_CUDA",
             4: "NRM_ERR_OOM", 5: "NRM_ERR_TIMEOUT", 6: "NRM_ERR_NO_DEVICE", 7: "NRM_ERR_BOUNDS"}
    return names.get(code, f"status {code}")


def load():
    """The loaded libnrm.so with argument types set (built first if stale)."""
    global _lib
    with _lock:
        if _lib is None:
            # NRM_LIB_VARIANT=debug selects the range-checking build.
            path = _build.build(debug=os.environ.get("NRM_LIB_VARIANT", "") == "debug")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int, where: str) -> None:
    if rc != NRM_OK:
        msg = load().nrm_last_error().decode(errors="replace")
        raise NrmError(rc, where, msg)
