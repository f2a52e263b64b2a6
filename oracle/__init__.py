"""FP64 CPU oracle for boundary-aware surface normals (arXiv 2209.08241).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(``paper_2209_08241_gb300``) never imports it, and it imports nothing from the
product path.

The arithmetic lives in ``nrm_oracle.cpp`` (plain C++17, FP64, no CUDA). This
module builds it with g++ and marshals numpy arrays through ctypes; it adds no
arithmetic of its own.

Paper passages followed (see the header of ``nrm_oracle.cpp`` for the steps):
Section 2 (definitions below Eq. 3), Section 3.1 (Fig. 2, the first two lines of
the "proof of efficiency" equation, the s24/s35 vectors), Section 3.2 (Eq.
"veclength", the threshold on r) and Section 4 (Fig. 8, mask applied to the
normal map).

Parity unpinned: the threshold value tau and the convention that masked pixels
carry the zero normal are stated conventions, not facts from the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrm_oracle.cpp")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libnrm_oracle.so")

DEPTH_F32, DEPTH_U16, DEPTH_F64 = 0, 1, 2
STAT_RAW, STAT_SECANT = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (no CUDA). Returns its path.

    ``-ffp-contract=off`` keeps the arithmetic identical on x86_64 and aarch64
    (GCC contracts a*b+c into an FMA by default on aarch64).
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declares the C signatures on a loaded oracle library; returns it."""
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.nrm_oracle_forward.restype = ctypes.c_int
    lib.nrm_oracle_forward.argtypes = [
        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_longlong, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        dp, dp, dp, dp, u8p, ctypes.c_int]
    lib.nrm_oracle_vjp.restype = ctypes.c_int
    lib.nrm_oracle_vjp.argtypes = [
        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_longlong, dp, ctypes.c_int, ctypes.c_int, dp, u8p,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
        ctypes.c_double, ctypes.c_int]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.float32:
        return DEPTH_F32
    if a.dtype == np.uint16:
        return DEPTH_U16
    if a.dtype == np.float64:
        return DEPTH_F64
    raise TypeError(f"unsupported depth dtype {a.dtype}")


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class OracleResult:
    n_raw: np.ndarray   # (H, W, 3) unnormalised normal
    n_hat: np.ndarray   # (H, W, 3) unit normal, zero where masked
    r: np.ndarray       # (H, W) ||n||, NaN where the stencil is invalid
    stat: np.ndarray    # (H, W) thresholded statistic, NaN where the stencil is invalid
    valid: np.ndarray   # (H, W) uint8 mask


def forward(depth: np.ndarray, K, alpha: int = 2, stat_mode: int = STAT_SECANT,
            tau: float = 12.0, depth_scale: float = 0.001, orient: int = 0,
            rows: tuple[int, int] | None = None, nthreads: int = 1) -> OracleResult:
    """Normals, statistic and mask of one depth map (H x W, float32/uint16/float64).

    ``K`` = (fx, fy, cx, cy). ``rows`` restricts the work to a row range; the
    outputs of the other rows are left at zero.
    """
    depth = np.ascontiguousarray(depth)
    if depth.ndim != 2:
        raise ValueError("depth must be 2-D")
    H, W = depth.shape
    K4 = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(4))
    n_raw = np.zeros((H, W, 3), np.float64)
    n_hat = np.zeros((H, W, 3), np.float64)
    r = np.zeros((H, W), np.float64)
    stat = np.zeros((H, W), np.float64)
    valid = np.zeros((H, W), np.uint8)
    r0, r1 = (0, H) if rows is None else rows
    rc = _load().nrm_oracle_forward(
        depth.ctypes.data_as(ctypes.c_void_p), _dtype_code(depth), H, W, W,
        _ptr(K4, ctypes.c_double), int(alpha), int(stat_mode), float(tau),
        float(depth_scale), int(orient), int(r0), int(r1),
        _ptr(n_raw, ctypes.c_double), _ptr(n_hat, ctypes.c_double),
        _ptr(r, ctypes.c_double), _ptr(stat, ctypes.c_double),
        _ptr(valid, ctypes.c_uint8), int(nthreads))
    if rc != 0:
        raise ValueError("nrm_oracle_forward rejected its arguments")
    return OracleResult(n_raw, n_hat, r, stat, valid)


def vjp(depth: np.ndarray, K, g: np.ndarray, valid: np.ndarray, alpha: int = 2,
        orient: int = 0, crop: tuple[int, int, int, int] | None = None,
        step: float = 1e-30, nthreads: int = 1) -> np.ndarray:
    """dL/d(depth) on a crop (y0, x0, h, w) for upstream g = dL/d(n_hat) (H x W x 3),
    mask held fixed, by complex-step differentiation of the direct form."""
    depth = np.ascontiguousarray(depth)
    if depth.dtype not in (np.float32, np.float64):
        raise TypeError("vjp needs float32 or float64 depth")
    H, W = depth.shape
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(H, W, 3)
    valid = np.ascontiguousarray(valid, dtype=np.uint8).reshape(H, W)
    y0, x0, h, w = (0, 0, H, W) if crop is None else crop
    K4 = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(4))
    out = np.zeros((h, w), np.float64)
    rc = _load().nrm_oracle_vjp(
        depth.ctypes.data_as(ctypes.c_void_p), _dtype_code(depth), H, W, W,
        _ptr(K4, ctypes.c_double), int(alpha), int(orient), _ptr(g, ctypes.c_double),
        _ptr(valid, ctypes.c_uint8), int(y0), int(x0), int(h), int(w),
        _ptr(out, ctypes.c_double), float(step), int(nthreads))
    if rc != 0:
        raise ValueError("nrm_oracle_vjp rejected its arguments")
    return out
