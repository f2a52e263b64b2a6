"""GB300-native boundary-aware surface normals from depth maps (arXiv 2209.08241).

A thin Python layer over the C ABI of ``libnrm.so`` (include/nrm.h). Every
step of the method runs in the library's CUDA kernels; this module only
allocates output tensors with torch, passes device pointers and the current
CUDA stream, and raises on a non-zero status. There is no CPU fallback: on a
machine without the built library or a GPU every call raises.

    est = NormalEstimator((fx, fy, cx, cy), H, W, alpha=2)
    normals, mask = est(depth)              # depth: (H, W) float32 or uint16 CUDA tensor

    batch = BatchedEstimator(alpha=2)
    outs = batch([(depth0, K0), (depth1, K1), ...])    # one persistent launch

    n = estimate_normals(depth, K)          # differentiable (float32 depth)
"""
from __future__ import annotations

import ctypes
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Sequence

import torch

from . import _lib
from ._lib import (NRM_IN_F32_M, NRM_IN_U16_MM, NRM_MASK_RAW, NRM_MASK_SECANT, NRM_MAX_ALPHA,
                   NRM_OUT_F16X4, NRM_OUT_F32X4, NRM_OUT_OCT16, NrmError)

__all__ = ["NormalEstimator", "BatchedEstimator", "NormalParams", "NrmError", "estimate_normals",
           "estimate_normals_batch", "NormalsFunction", "NormalsBatchFunction", "MASK_RAW", "MASK_SECANT",
           "decode_oct16", "spherical_images", "angle_mse", "version"]

MASK_RAW = NRM_MASK_RAW
MASK_SECANT = NRM_MASK_SECANT


@dataclass
class NormalParams:
    """Mirror of ``nrm_params``. mask_mode: "secant" (default) or "raw"."""
    alpha: int = 2
    mask_mode: str = "secant"
    tau: float = 12.0
    depth_scale: float = 0.001
    out_dtype: str = "f32"          # "f32" (float4 per pixel), "f16" (half4) or "oct16" (2 x int16)
    orient_to_camera: bool = False

    def to_c(self, in_dtype: int) -> _lib.Params:
        """The C ``nrm_params`` struct for these parameters and an input dtype."""
        p = _lib.Params()
        p.alpha = int(self.alpha)
        p.mask_mode = {"secant": NRM_MASK_SECANT, "raw": NRM_MASK_RAW}[self.mask_mode]
        p.tau = float(self.tau)
        p.depth_scale = float(self.depth_scale)
        p.in_dtype = int(in_dtype)
        p.out_dtype = {"f32": NRM_OUT_F32X4, "f16": NRM_OUT_F16X4, "oct16": NRM_OUT_OCT16}[self.out_dtype]
        p.orient_to_camera = int(bool(self.orient_to_camera))
        return p

    @property
    def torch_out_dtype(self) -> torch.dtype:
        return {"f32": torch.float32, "f16": torch.float16, "oct16": torch.int16}[self.out_dtype]

    @property
    def out_channels(self) -> int:
        """Elements per pixel of the normal map: 4 (x, y, z, 0) or 2 (octahedral code)."""
        return 2 if self.out_dtype == "oct16" else 4


def decode_oct16(codes: torch.Tensor) -> torch.Tensor:
    """Unit normals (..., 3) float32 from octahedral codes (..., 2) int16 (the
    NRM_OUT_OCT16 encoding). Masked pixels decode to (0, 0, 1); use the mask."""
    q = codes.to(torch.float32) / 32767.0
    x, y = q[..., 0], q[..., 1]
    z = 1.0 - x.abs() - y.abs()
    neg = z < 0
    fx = torch.where(neg, (1.0 - y.abs()) * torch.where(x >= 0, 1.0, -1.0), x)
    fy = torch.where(neg, (1.0 - x.abs()) * torch.where(y >= 0, 1.0, -1.0), y)
    v = torch.stack([fx, fy, z], dim=-1)
    return v / v.norm(dim=-1, keepdim=True)


def version() -> str:
    """The library's version string (with the architecture it was built for)."""
    return _lib.load().nrm_version().decode()


def set_autotune_cache(path: str | None) -> None:
    """Sets the process-wide autotune cache file (``nrm_set_autotune_cache``):
    handles created afterwards start from the tuned geometry recorded for their
    key, and ``autotune`` without a path reads and records there. None clears it."""
    _lib.check(_lib.load().nrm_set_autotune_cache(path.encode() if path else None), "nrm_set_autotune_cache")


def autotune_cache_get(path: str, key: str) -> dict | None:
    """The configuration recorded for ``key`` in the cache file, or None."""
    c = _lib.TileConfig()
    lib = _lib.load()
    if lib.nrm_autotune_cache_get(path.encode(), key.encode(), ctypes.byref(c)) != _lib.NRM_OK:
        return None
    return {"tile_x": c.tile_x, "tile_y": c.tile_y, "threads": c.threads, "stages": c.stages,
            "ctas_per_sm": c.ctas_per_sm}


def autotune_cache_put(path: str, key: str, tile_x: int, tile_y: int, threads: int, stages: int,
                       ctas_per_sm: int = 0) -> None:
    """Adds or replaces the entry of ``key`` in the cache file."""
    c = _lib.TileConfig(tile_x, tile_y, threads, stages, ctas_per_sm)
    _lib.check(_lib.load().nrm_autotune_cache_put(path.encode(), key.encode(), ctypes.byref(c)),
               "nrm_autotune_cache_put")


def _in_dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return NRM_IN_F32_M
    if t.dtype == torch.uint16:
        return NRM_IN_U16_MM
    raise TypeError(f"depth must be float32 (metres) or uint16 (depth_scale units), got {t.dtype}")


def _stream_ptr(stream: torch.cuda.Stream | None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _intr(K) -> _lib.Intrinsics:
    fx, fy, cx, cy = (float(v) for v in K)
    return _lib.Intrinsics(fx, fy, cx, cy)


def _check_cuda(t: torch.Tensor, name: str, device: torch.device | None = None):
    if device is None:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    elif t.device != device:  # device is a CUDA device, so this also refuses host tensors
        raise ValueError(f"{name} must be a CUDA tensor on {device}, got one on {t.device}")


def _check_dense(t: torch.Tensor, shape, dtype: torch.dtype, device: torch.device, name: str):
    """t must be a contiguous CUDA tensor of exactly this shape and dtype on
    ``device``: the library writes through its raw pointer."""
    _check_cuda(t, name, device)
    if t.shape != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {tuple(shape)} {dtype} tensor, got "
                         f"{tuple(t.shape)} {t.dtype}{'' if t.is_contiguous() else ' (not contiguous)'}")


class _Handle:
    def __init__(self, K, H: int, W: int, params: NormalParams, in_dtype: int, device=None):
        self.lib = _lib.load()
        self.params = params
        self.in_dtype = in_dtype
        self.H, self.W = int(H), int(W)
        index = None if device is None else torch.device(device).index
        self.device = torch.device("cuda", torch.cuda.current_device() if index is None else index)
        h = ctypes.c_void_p()
        c_params = params.to_c(in_dtype)
        with torch.cuda.device(self.device):
            kp = ctypes.byref(_intr(K)) if K is not None else None
            _lib.check(self.lib.nrm_create(kp, self.H, self.W, ctypes.byref(c_params),
                                           ctypes.byref(h)), "nrm_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.nrm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # Introspection and tuning ------------------------------------------
    def config(self) -> dict:
        c = _lib.TileConfig()
        _lib.check(self.lib.nrm_get_config(self.h, ctypes.byref(c)), "nrm_get_config")
        return {k: getattr(c, k) for k, _ in c._fields_}

    def autotune_key(self) -> str:
        """This handle's key in the autotune cache (``nrm_autotune_key``)."""
        buf = ctypes.create_string_buffer(512)
        _lib.check(self.lib.nrm_autotune_key(self.h, buf, len(buf)), "nrm_autotune_key")
        return buf.value.decode()

    def set_config(self, tile_x=128, tile_y=16, threads=256, stages=3, ctas_per_sm=0):
        c = _lib.TileConfig(tile_x, tile_y, threads, stages, ctas_per_sm)
        _lib.check(self.lib.nrm_set_config(self.h, ctypes.byref(c)), "nrm_set_config")

    def sync_status(self):
        _lib.check(self.lib.nrm_sync_status(self.h), "nrm_sync_status")

    def enable_timing(self, on: bool = True):
        _lib.check(self.lib.nrm_enable_timing(self.h, int(on)), "nrm_enable_timing")

    def stats(self) -> dict:
        s = _lib.Stats()
        _lib.check(self.lib.nrm_get_stats(self.h, ctypes.byref(s)), "nrm_get_stats")
        return {"launches": s.launches, "kernel_ms": s.kernel_ms, "tiles": s.tiles}

    def reset_stats(self):
        _lib.check(self.lib.nrm_reset_stats(self.h), "nrm_reset_stats")


class NormalEstimator(_Handle):
    """Fixed-size single-frame estimator (one plain launch per call).

    ``in_dtype`` is "f32" (metres) or "u16" (units of ``depth_scale``)."""

    def __init__(self, K, H: int, W: int, params: NormalParams | None = None,
                 in_dtype: str = "f32", device=None, **kw):
        params = params or NormalParams(**kw)
        super().__init__(K, H, W, params, {"f32": NRM_IN_F32_M, "u16": NRM_IN_U16_MM}[in_dtype], device)
        self.K = tuple(float(v) for v in K)
        # What every call checks, formed once (the per-frame call is host-bound).
        self._dev_index = self.device.index
        self._depth_dtype = torch.float32 if self.in_dtype == NRM_IN_F32_M else torch.uint16
        self._hw = (self.H, self.W)
        self._nshape = (self.H, self.W, self.params.out_channels)
        self._ndtype = self.params.torch_out_dtype

    def new_outputs(self):
        """A new (normals, valid) pair of this estimator's size and output dtype."""
        n = torch.empty((self.H, self.W, self.params.out_channels), dtype=self.params.torch_out_dtype,
                        device=self.device)
        m = torch.empty((self.H, self.W), dtype=torch.uint8, device=self.device)
        return n, m

    def _check_depth(self, depth: torch.Tensor):
        if depth.get_device() != self._dev_index:  # -1 for host tensors
            _check_cuda(depth, "depth", self.device)
        if depth.shape != self._hw or not depth.is_contiguous():
            raise ValueError(f"depth must be a contiguous ({self.H}, {self.W}) tensor")
        if depth.dtype != self._depth_dtype:
            _in_dtype(depth)  # raises for a dtype the library does not take
            raise TypeError("depth dtype does not match the estimator's in_dtype")

    def _outputs(self, normals: torch.Tensor | None, valid: torch.Tensor | None):
        """The caller's (normals, valid), checked, or new ones."""
        if normals is None or valid is None:
            return self.new_outputs()
        # The common case in a few attribute reads; anything off goes through
        # the full check, which raises with the details.
        if not (normals.get_device() == self._dev_index and valid.get_device() == self._dev_index
                and normals.shape == self._nshape and valid.shape == self._hw and normals.dtype == self._ndtype
                and valid.dtype == torch.uint8 and normals.is_contiguous() and valid.is_contiguous()):
            _check_dense(normals, self._nshape, self._ndtype, self.device, "normals")
            _check_dense(valid, self._hw, torch.uint8, self.device, "valid")
        return normals, valid

    def estimate(self, depth: torch.Tensor, normals: torch.Tensor | None = None,
                 valid: torch.Tensor | None = None, stream=None, points: torch.Tensor | None = None):
        """Writes the (H, W, 4) normal map and (H, W) uint8 mask; returns both.
        With ``points`` ((H, W, 4) float32) the organised point cloud is written
        in the same pass."""
        self._check_depth(depth)
        normals, valid = self._outputs(normals, valid)
        if points is not None:
            _check_dense(points, (self.H, self.W, 4), torch.float32, self.device, "points")
            _lib.check(self.lib.nrm_estimate_points(self.h, depth.data_ptr(), normals.data_ptr(), valid.data_ptr(),
                                                    points.data_ptr(), _stream_ptr(stream)), "nrm_estimate_points")
            return normals, valid
        _lib.check(self.lib.nrm_estimate(self.h, depth.data_ptr(), normals.data_ptr(),
                                         valid.data_ptr(), _stream_ptr(stream)), "nrm_estimate")
        return normals, valid

    __call__ = estimate

    def backward(self, depth: torch.Tensor, grad_normals: torch.Tensor, valid: torch.Tensor,
                 grad_depth: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """dL/d(depth) for upstream dL/d(normals) (H, W, 4) float32, mask fixed."""
        # (A uint16 handle passes here; the library refuses it: NRM_ERR_UNSUPPORTED.)
        _check_dense(depth, (self.H, self.W), torch.float32 if self.in_dtype == NRM_IN_F32_M else torch.uint16,
                     self.device, "depth")
        _check_dense(grad_normals, (self.H, self.W, 4), torch.float32, self.device, "grad_normals")
        _check_dense(valid, (self.H, self.W), torch.uint8, self.device, "valid")
        if grad_depth is None:
            grad_depth = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
        _check_dense(grad_depth, (self.H, self.W), torch.float32, self.device, "grad_depth")
        _lib.check(self.lib.nrm_backward(self.h, depth.data_ptr(), grad_normals.data_ptr(),
                                         valid.data_ptr(), grad_depth.data_ptr(),
                                         _stream_ptr(stream)), "nrm_backward")
        return grad_depth

    def estimate_multiscale(self, depth: torch.Tensor, alphas=(1, 2, 3, 4), form: str = "pair",
                            normals: torch.Tensor | None = None, valid: torch.Tensor | None = None, stream=None):
        """Multi-scale variant (Section 2): the average of the per-scale
        unnormalised normals over pixel distances ``alphas`` (at most 8),
        each scale the previous method's single pair (``form="pair"``, Eq. 1-3)
        or the four-direction form (``form="quad"``, Eq. 4-6); mask, dtypes and
        orientation as for ``estimate``."""
        self._check_depth(depth)
        sc = _scales(alphas, form)
        normals, valid = self._outputs(normals, valid)
        _lib.check(self.lib.nrm_estimate_multiscale(self.h, depth.data_ptr(), normals.data_ptr(), valid.data_ptr(),
                                                    ctypes.byref(sc), _stream_ptr(stream)), "nrm_estimate_multiscale")
        return normals, valid

    def plane_fit(self, depth: torch.Tensor, radius: int = 2, normals: torch.Tensor | None = None,
                  valid: torch.Tensor | None = None, stream=None):
        """Plane-fitting ground truth (Sections 1 and 4; radius 2 = 25 points):
        (H, W, 4) float32 normals (w = 0) and (H, W) uint8 mask of the
        (2 radius + 1)^2 window fit, oriented like the method's normals."""
        self._check_depth(depth)
        if normals is None:
            normals = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        if valid is None:
            valid = torch.empty((self.H, self.W), dtype=torch.uint8, device=self.device)
        _check_dense(normals, (self.H, self.W, 4), torch.float32, self.device, "normals")
        _check_dense(valid, (self.H, self.W), torch.uint8, self.device, "valid")
        _lib.check(self.lib.nrm_plane_fit(self.h, depth.data_ptr(), normals.data_ptr(), valid.data_ptr(),
                                          int(radius), _stream_ptr(stream)), "nrm_plane_fit")
        return normals, valid


def _scales(alphas, form: str) -> _lib.Scales:
    alphas = [int(a) for a in alphas]
    if not 1 <= len(alphas) <= _lib.NRM_MAX_SCALES:
        raise ValueError(f"between 1 and {_lib.NRM_MAX_SCALES} scales")
    forms = {"pair": _lib.NRM_MS_PAIR, "quad": _lib.NRM_MS_QUAD}
    if form not in forms:
        raise ValueError(f"form must be one of {tuple(forms)}")
    sc = _lib.Scales()
    sc.n_scales = len(alphas)
    for i, a in enumerate(alphas):
        sc.alpha[i] = a
    sc.form = forms[form]
    return sc


def _check_points(points: torch.Tensor, H: int, W: int, out_pitch: int):
    _check_cuda(points, "points")
    if points.dtype != torch.float32 or tuple(points.shape) != (H, W, 4) or points.stride(2) != 1 \
            or points.stride(1) != 4 or (H * W and points.stride(0) != 4 * out_pitch):
        raise ValueError("points must be (H, W, 4) float32 with the normals' pixel pitch")


def _frame(depth: torch.Tensor, K, normals: torch.Tensor, valid: torch.Tensor,
           points: torch.Tensor | None = None) -> _lib.Frame:
    f = _lib.Frame()
    f.depth = depth.data_ptr()
    f.normals = normals.data_ptr()
    f.valid = valid.data_ptr()
    f.H, f.W = int(depth.shape[0]), int(depth.shape[1])
    if depth.numel():
        f.depth_pitch = int(depth.stride(0))
        f.out_pitch = int(normals.stride(0) // normals.shape[2])
    else:
        f.depth_pitch = f.out_pitch = f.W
    f.K = _intr(K)
    f.in_dtype = _in_dtype(depth)
    if points is not None:
        _check_points(points, f.H, f.W, f.out_pitch)
        f.points = points.data_ptr()
    return f


class BatchedEstimator(_Handle):
    """Any number of frames of any sizes, intrinsics and input dtypes per call,
    processed by one persistent launch replayed from a CUDA graph."""

    def __init__(self, params: NormalParams | None = None, device=None, **kw):
        params = params or NormalParams(**kw)
        super().__init__(None, 0, 0, params, NRM_IN_F32_M, device)
        self._frames = None

    def make_frames(self, items: Sequence, outputs: Sequence | None = None, points: bool = False):
        """ctypes frame array for [(depth, K), ...] with outputs [(normals, valid), ...]
        or [(normals, valid, points), ...] (allocated when None; ``points`` asks for
        the organised point cloud, (H, W, 4) float32). Returns (frames_array, outputs)."""
        n = len(items)
        arr = (_lib.Frame * max(n, 1))()
        outs = []
        for i, (depth, K) in enumerate(items):
            _check_cuda(depth, "depth", self.device)
            if depth.dim() != 2 or depth.stride(1) != 1:
                raise ValueError("each depth must be a 2-D tensor with unit column stride")
            H, W = depth.shape
            C = self.params.out_channels
            pm = None
            if outputs is None:
                nm = torch.empty((H, W, C), dtype=self.params.torch_out_dtype, device=depth.device)
                vm = torch.empty((H, W), dtype=torch.uint8, device=depth.device)
                if points:
                    pm = torch.empty((H, W, 4), dtype=torch.float32, device=depth.device)
            elif len(outputs[i]) == 3:
                nm, vm, pm = outputs[i]
            else:
                nm, vm = outputs[i]
            for t, name in ((nm, "normals"), (vm, "valid")) + (((pm, "points"),) if pm is not None else ()):
                _check_cuda(t, name, self.device)
            if tuple(nm.shape) != (H, W, C) or tuple(vm.shape) != (H, W):
                raise ValueError(f"outputs must be (H, W, {C}) normals and (H, W) valid")
            if depth.numel() and (nm.stride(2) != 1 or nm.stride(1) != C or nm.stride(0) % C
                                  or vm.stride(1) != 1 or vm.stride(0) * C != nm.stride(0)):
                raise ValueError(f"normals (H, W, {C}) and valid (H, W) must share the pixel pitch")
            if nm.dtype != self.params.torch_out_dtype or vm.dtype != torch.uint8:
                raise TypeError("output dtypes do not match the estimator's out_dtype / uint8")
            arr[i] = _frame(depth, K, nm, vm, pm)
            outs.append((nm, vm) if pm is None else (nm, vm, pm))
        return arr, outs

    def run(self, frames_array, n: int, stream=None):
        """One batched launch over the first n frames of a ``make_frames`` array."""
        _lib.check(self.lib.nrm_estimate_batched(self.h, frames_array, int(n), _stream_ptr(stream)),
                   "nrm_estimate_batched")

    def __call__(self, items: Sequence, outputs: Sequence | None = None, stream=None, points: bool = False):
        arr, outs = self.make_frames(items, outputs, points)
        self.run(arr, len(items), stream)
        return outs

    def run_multiscale(self, frames_array, n: int, alphas=(1, 2, 3, 4), form: str = "pair", stream=None):
        """Multi-scale variant (Section 2's scale average; see
        ``NormalEstimator.estimate_multiscale``) of a batch in one launch."""
        sc = _scales(alphas, form)
        _lib.check(self.lib.nrm_estimate_batched_multiscale(self.h, frames_array, int(n), ctypes.byref(sc),
                                                            _stream_ptr(stream)), "nrm_estimate_batched_multiscale")

    def multiscale(self, items: Sequence, alphas=(1, 2, 3, 4), form: str = "pair", outputs: Sequence | None = None,
                   stream=None):
        """``run_multiscale`` on [(depth, K), ...]; returns the (normals, valid) outputs."""
        arr, outs = self.make_frames(items, outputs)
        self.run_multiscale(arr, len(items), alphas, form, stream)
        return outs

    def make_host_frames(self, depth_host: torch.Tensor, Ks: Sequence, normals_host: torch.Tensor,
                         valid_host: torch.Tensor, points_host: torch.Tensor | None = None):
        """ctypes frame array with HOST pointers for ``run_host``: a stack of n
        equal-size frames, depth (n, H, W) float32/uint16, normals
        (n, H, W, C), valid (n, H, W) uint8 and optional points (n, H, W, 4)
        float32, contiguous CPU tensors (page-locked for asynchronous copies)."""
        n, H, W = depth_host.shape
        C = self.params.out_channels
        tensors = [depth_host, normals_host, valid_host] + ([points_host] if points_host is not None else [])
        for t in tensors:
            if t.device.type != "cpu" or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors")
        if tuple(normals_host.shape) != (n, H, W, C) or normals_host.dtype != self.params.torch_out_dtype \
                or tuple(valid_host.shape) != (n, H, W) or valid_host.dtype != torch.uint8:
            raise ValueError(f"normals must be (n, H, W, {C}) {self.params.torch_out_dtype}, valid (n, H, W) uint8")
        if points_host is not None and (tuple(points_host.shape) != (n, H, W, 4)
                                        or points_host.dtype != torch.float32):
            raise ValueError("points must be (n, H, W, 4) float32")
        arr = (_lib.Frame * max(n, 1))()
        for i in range(n):
            f = arr[i]
            f.depth = depth_host[i].data_ptr()
            f.normals = normals_host[i].data_ptr()
            f.valid = valid_host[i].data_ptr()
            f.H, f.W = int(H), int(W)
            f.depth_pitch = f.out_pitch = int(W)
            f.K = _intr(Ks[i])
            f.in_dtype = _in_dtype(depth_host)
            if points_host is not None:
                f.points = points_host[i].data_ptr()
        return arr

    def run_host(self, depth_host: torch.Tensor, Ks: Sequence, normals_host: torch.Tensor,
                 valid_host: torch.Tensor, frames=None, stream=None, points_host: torch.Tensor | None = None):
        """End-to-end call on HOST buffers (``nrm_estimate_batched_host``): the
        library uploads, computes and downloads in overlapped chunks on its own
        streams, after everything already queued on ``stream``, which waits for
        it; synchronise ``stream`` before reading the outputs. Returns the frame
        array (pass it back as ``frames`` to skip rebuilding it)."""
        n = depth_host.shape[0]
        if frames is None:
            frames = self.make_host_frames(depth_host, Ks, normals_host, valid_host, points_host)
        _lib.check(self.lib.nrm_estimate_batched_host(self.h, frames, int(n), _stream_ptr(stream)),
                   "nrm_estimate_batched_host")
        return frames

    def make_grad_frames(self, items: Sequence, grad_normals: Sequence, valids: Sequence,
                         grad_depths: Sequence | None = None):
        """ctypes adjoint frame array for items [(depth float32 (H, W), K)],
        grad_normals [(H, W, 4) float32], valids [(H, W) uint8 masks from the
        forward] and depth gradients [(H, W) float32] (allocated when None).
        Returns (frames_array, grad_depths)."""
        n = len(items)
        arr = (_lib.GradFrame * max(n, 1))()
        outs = []
        for i, (depth, K) in enumerate(items):
            g, v = grad_normals[i], valids[i]
            for t, name in ((depth, "depth"), (g, "grad_normals"), (v, "valid")):
                _check_cuda(t, name, self.device)
            if depth.dtype != torch.float32 or g.dtype != torch.float32:
                raise TypeError("the adjoint needs float32 depth and float32 grad_normals")
            H, W = depth.shape
            gd = (torch.empty((H, W), dtype=torch.float32, device=depth.device) if grad_depths is None
                  else grad_depths[i])
            _check_cuda(gd, "grad_depth", self.device)
            if tuple(g.shape) != (H, W, 4) or tuple(v.shape) != (H, W) or tuple(gd.shape) != (H, W):
                raise ValueError("shape mismatch in the adjoint batch")
            if v.dtype != torch.uint8 or gd.dtype != torch.float32:
                raise TypeError("the adjoint needs a uint8 mask and a float32 grad_depth")
            if depth.numel() and (depth.stride(1) != 1 or gd.stride(1) != 1 or gd.stride(0) != depth.stride(0)
                                  or g.stride(2) != 1 or g.stride(1) != 4 or v.stride(1) != 1
                                  or v.stride(0) * 4 != g.stride(0)):
                raise ValueError("depth/grad_depth and grad_normals/valid must each share a row pitch")
            f = arr[i]
            f.depth, f.grad_normals, f.valid, f.grad_depth = (depth.data_ptr(), g.data_ptr(), v.data_ptr(),
                                                              gd.data_ptr())
            f.H, f.W = int(H), int(W)
            f.depth_pitch = int(depth.stride(0)) if depth.numel() else f.W
            f.out_pitch = int(g.stride(0) // 4) if depth.numel() else f.W
            f.K = _intr(K)
            outs.append(gd)
        return arr, outs

    def run_backward(self, grad_frames_array, n: int, stream=None):
        """One batched adjoint launch over the first n frames of a ``make_grad_frames`` array."""
        _lib.check(self.lib.nrm_backward_batched(self.h, grad_frames_array, int(n), _stream_ptr(stream)),
                   "nrm_backward_batched")

    def run_backward_scaled(self, grad_frames_array, n: int, scale: torch.Tensor, stream=None):
        """``nrm_backward_batched_scaled``: the upstream gradient of frame i is
        scale[i] times its grad_normals buffer (a float32 device tensor of n
        values, e.g. -1 / N_valid with target normals for the cosine loss)."""
        _check_dense(scale, (int(n),), torch.float32, self.device, "scale")
        _lib.check(self.lib.nrm_backward_batched_scaled(self.h, grad_frames_array, int(n), scale.data_ptr(),
                                                        _stream_ptr(stream)), "nrm_backward_batched_scaled")

    def cosine_loss_scale(self, grad_frames_array, n: int, scale: torch.Tensor | None = None, stream=None):
        """``nrm_cosine_loss_scale``: the (n,) float32 device tensor of
        -1 / max(N_valid, 1) per frame of a grad-frame array (its masks), for
        ``run_backward_scaled``; written asynchronously on the stream."""
        if scale is None:
            scale = torch.empty(int(n), dtype=torch.float32, device=self.device)
        _check_dense(scale, (int(n),), torch.float32, self.device, "scale")
        _lib.check(self.lib.nrm_cosine_loss_scale(self.h, grad_frames_array, int(n), scale.data_ptr(),
                                                  _stream_ptr(stream)), "nrm_cosine_loss_scale")
        return scale

    def cosine_loss_backward(self, items: Sequence, targets: Sequence, valids: Sequence,
                             grad_depths: Sequence | None = None, stream=None):
        """Depth gradients of L_i = mean over the valid pixels of frame i of
        (1 - n_hat . t) for each frame i of a batch: the per-frame factor
        -1 / max(N_valid, 1) (``nrm_cosine_loss_scale``), then one adjoint
        launch with no dL/dn_hat buffer: targets [(H, W, 4) float32 unit
        normals, 4th component ignored], valids the forward's masks. Returns
        the gradients and the per-frame scale it used."""
        arr, outs = self.make_grad_frames(items, targets, valids, grad_depths)
        scale = self.cosine_loss_scale(arr, len(items), stream=stream)
        self.run_backward_scaled(arr, len(items), scale, stream)
        return outs, scale

    def backward(self, items: Sequence, grad_normals: Sequence, valids: Sequence,
                 grad_depths: Sequence | None = None, stream=None) -> list:
        """Adjoint of a batch in one launch (see ``make_grad_frames``); returns
        (or fills) the [(H, W) float32] depth gradients."""
        arr, outs = self.make_grad_frames(items, grad_normals, valids, grad_depths)
        self.run_backward(arr, len(items), stream)
        return outs

    def autotune(self, items: Sequence, outputs: Sequence | None = None, cache_path: str | None = None,
                 stream=None) -> dict:
        """Times the compiled launch geometries (tile shape, pipeline depth,
        CTAs per SM) on these frames and keeps the fastest (``nrm_autotune``;
        cached in ``cache_path``, or in the process-wide file of
        ``set_autotune_cache`` when None); returns the chosen configuration."""
        arr, _ = self.make_frames(items, outputs)
        cp = cache_path.encode() if cache_path else None
        _lib.check(self.lib.nrm_autotune(self.h, arr, len(items), _stream_ptr(stream), cp), "nrm_autotune")
        return self.config()


class NormalsFunction(torch.autograd.Function):
    """Differentiable normal map of float32 depth: forward = nrm_estimate,
    backward = nrm_backward (mask held fixed; the mask output has no gradient)."""

    @staticmethod
    def forward(ctx, depth: torch.Tensor, est: NormalEstimator):
        depth = depth.contiguous()
        normals, valid = est.estimate(depth)
        ctx.est = est
        ctx.save_for_backward(depth, valid)
        ctx.mark_non_differentiable(valid)
        return normals, valid

    @staticmethod
    def backward(ctx, grad_normals, grad_valid):
        depth, valid = ctx.saved_tensors
        if grad_normals is None:
            return None, None
        g = grad_normals.contiguous().to(torch.float32)
        return ctx.est.backward(depth, g, valid), None


class NormalsBatchFunction(torch.autograd.Function):
    """Differentiable normals of a stack of float32 depth maps (B, H, W) with
    per-frame intrinsics: forward = one nrm_estimate_batched launch, backward =
    one nrm_backward_batched launch (masks held fixed)."""

    @staticmethod
    def forward(ctx, depth: torch.Tensor, Ks: tuple, est: "BatchedEstimator"):
        depth = depth.contiguous()
        B, H, W = depth.shape
        normals = torch.empty((B, H, W, 4), dtype=est.params.torch_out_dtype, device=depth.device)
        valid = torch.empty((B, H, W), dtype=torch.uint8, device=depth.device)
        est([(depth[i], Ks[i]) for i in range(B)], [(normals[i], valid[i]) for i in range(B)])
        ctx.est, ctx.Ks = est, Ks
        ctx.save_for_backward(depth, valid)
        ctx.mark_non_differentiable(valid)
        return normals, valid

    @staticmethod
    def backward(ctx, grad_normals, grad_valid):
        depth, valid = ctx.saved_tensors
        if grad_normals is None:
            return None, None, None
        g = grad_normals.contiguous().to(torch.float32)
        B = depth.shape[0]
        grad = torch.empty_like(depth)
        ctx.est.backward([(depth[i], ctx.Ks[i]) for i in range(B)], [g[i] for i in range(B)],
                         [valid[i] for i in range(B)], [grad[i] for i in range(B)])
        return grad, None, None


def _check_map(n: torch.Tensor, v: torch.Tensor, name: str, device: torch.device | None = None):
    _check_cuda(n, name, device)
    _check_cuda(v, name + " mask", n.device)
    if n.dtype != torch.float32 or n.dim() != 3 or n.shape[2] != 4 or v.dtype != torch.uint8:
        raise TypeError(f"{name}: expected (H, W, 4) float32 normals and an (H, W) uint8 mask")
    if tuple(v.shape) != tuple(n.shape[:2]) or n.stride(2) != 1 or n.stride(1) != 4 or v.stride(1) != 1 \
            or v.stride(0) * 4 != n.stride(0):
        raise ValueError(f"{name}: normals and mask must share one pixel pitch")


def spherical_images(normals: torch.Tensor, valid: torch.Tensor, stream=None):
    """(phi, theta) images (Section 4: I_phi in [0, 2 pi), I_theta in [0, pi]) of a
    float4 normal map; masked pixels get 0."""
    _check_map(normals, valid, "normals")
    H, W = valid.shape
    phi = torch.empty((H, W), dtype=torch.float32, device=normals.device)
    theta = torch.empty_like(phi)
    if H * W:
        if phi.stride(0) != valid.stride(0):
            raise ValueError("dense (H, W) outputs need a dense mask")
        _lib.check(_lib.load().nrm_spherical(normals.data_ptr(), valid.data_ptr(), H, W, valid.stride(0),
                                             phi.data_ptr(), theta.data_ptr(), _stream_ptr(stream)),
                   "nrm_spherical")
    return phi, theta


def angle_mse(est, normals, valid, ref_normals, ref_valid, stream=None) -> torch.Tensor:
    """(MSE of I_theta, MSE of I_phi, count) as a float64 CUDA tensor of 3, over
    the pixels valid in both maps (Tables 2-5); ``est`` provides the scratch."""
    _check_map(normals, valid, "normals", est.device)
    _check_map(ref_normals, ref_valid, "ref_normals", est.device)
    if valid.shape != ref_valid.shape or valid.stride(0) != ref_valid.stride(0):
        raise ValueError("the two maps must have one shape and pitch")
    out = torch.zeros(3, dtype=torch.float64, device=normals.device)
    H, W = valid.shape
    _lib.check(est.lib.nrm_angle_mse(est.h, normals.data_ptr(), valid.data_ptr(), ref_normals.data_ptr(),
                                     ref_valid.data_ptr(), H, W, valid.stride(0), out.data_ptr(),
                                     _stream_ptr(stream)), "nrm_angle_mse")
    return out


# Handles made by the functional calls below, most recently used last; at most
# _CACHE_MAX per cache (an evicted handle is released once nothing refers to
# it, e.g. after the backward pass of a graph that saved it).
_CACHE_MAX = 32
_batch_estimators: "OrderedDict" = OrderedDict()


def _cached(cache: "OrderedDict", key, make):
    est = cache.get(key)
    if est is None:
        est = make()
        cache[key] = est
        while len(cache) > _CACHE_MAX:
            cache.popitem(last=False)
    else:
        cache.move_to_end(key)
    return est


def estimate_normals_batch(depth: torch.Tensor, K, params: NormalParams | None = None):
    """Differentiable (B, H, W) float32 depth -> ((B, H, W, 4) normals, (B, H, W)
    masks). K: one (fx, fy, cx, cy) for all frames or a sequence of B of them."""
    params = params or NormalParams()
    B = depth.shape[0]
    Ks = tuple(tuple(float(v) for v in k) for k in K) if len(K) == B and hasattr(K[0], "__len__") \
        else tuple(tuple(float(v) for v in K) for _ in range(B))
    key = (repr(params), depth.device.index)

    def make():
        with torch.cuda.device(depth.device):
            return BatchedEstimator(params, device=depth.device)

    return NormalsBatchFunction.apply(depth, Ks, _cached(_batch_estimators, key, make))


def estimate(depth: torch.Tensor, K, params: NormalParams | None = None):
    """Normals and mask of a depth map: ``(H, W)`` -> ((H, W, 4), (H, W)) through
    ``estimate_normals``, or a stack ``(B, H, W)`` -> ((B, H, W, 4), (B, H, W))
    through ``estimate_normals_batch`` (K: one for all frames or one per
    frame). Differentiable with respect to float32 depth, masks held fixed."""
    if depth.dim() == 3:
        return estimate_normals_batch(depth, K, params)
    return estimate_normals(depth, K, params)


_estimators: "OrderedDict" = OrderedDict()


def estimate_normals(depth: torch.Tensor, K, params: NormalParams | None = None):
    """Differentiable (H, W) float32 depth -> ((H, W, 4) normals, (H, W) mask).
    Handles are cached per (shape, K, params, device)."""
    params = params or NormalParams()
    key = (tuple(depth.shape), tuple(float(v) for v in K), repr(params), depth.device.index)

    def make():
        with torch.cuda.device(depth.device):
            return NormalEstimator(K, depth.shape[0], depth.shape[1], params,
                                   in_dtype="f32" if depth.dtype == torch.float32 else "u16")

    return NormalsFunction.apply(depth, _cached(_estimators, key, make))
