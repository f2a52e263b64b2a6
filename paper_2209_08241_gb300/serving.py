"""Continuous-batching server for depth frames (the served form).

Requests (one depth frame each, any size, float32 metres or uint16 units, own
intrinsics) arrive in host memory. The server

  * admits a waiting request when a device buffer set for its frame size is
    free or can be created within the device-memory budget (buffers stay
    resident and are reused by later requests of the same size), and, when it
    delivers results, a pinned host buffer set for them within the host budget;
  * copies the admitted frames to the device and launches everything admitted
    so far as ONE batched persistent launch (``nrm_estimate_batched``) on the
    next free stream, followed by the copies of every result (normals and
    mask) back to the request's pinned host buffers, so a batch's uploads,
    kernel and downloads overlap those of the batches before and after it;
  * retires batches as their completion events fire (after the downloads), and
    hands each finished request to the ``on_done`` callback with its results
    in host memory (``Request.normals`` / ``Request.valid``, valid until the
    callback returns; copy them to keep them) before recycling the buffers.

Per-request latency is completion time minus arrival time, both on the host
clock, so it includes the result's delivery to host memory. ``PlainServer``
is the baseline: one plain per-frame launch per request, in arrival order, on
one stream, with the same upload and delivery. With ``deliver=False`` results
stay on the device (``Request.buffers`` during the callback).

All normal arithmetic runs in the library's CUDA kernels; this module only
schedules, copies and keeps books.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import torch

from . import BatchedEstimator, NormalEstimator, NormalParams, _cached, _lib


def _device(device) -> torch.device:
    """The CUDA device a server runs on: ``device``, else the current one."""
    index = None if device is None else torch.device(device).index
    return torch.device("cuda", torch.cuda.current_device() if index is None else index)


@dataclass
class Request:
    rid: int
    depth: torch.Tensor          # (H, W) float32 or uint16, host (pinned for async copies)
    K: tuple                     # (fx, fy, cx, cy)
    t_arrival: float = 0.0       # host clock (time.perf_counter)
    t_launch: float = 0.0
    t_done: float = 0.0
    buffers: Optional["BufferSet"] = None       # device buffers while on the GPU
    host: Optional["BufferSet"] = None          # pinned result buffers while delivering
    normals: Optional[torch.Tensor] = None      # delivered results (host), during on_done
    valid: Optional[torch.Tensor] = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival

    @property
    def pixels(self) -> int:
        return int(self.depth.shape[0] * self.depth.shape[1])


@dataclass
class BufferSet:
    """Resident device buffers for one frame: depth in, normals and mask out."""
    key: tuple
    depth: torch.Tensor
    normals: torch.Tensor
    valid: torch.Tensor
    nbytes: int


class BufferPool:
    """Buffer sets per (H, W, depth dtype), bounded by a byte budget: device
    sets (depth, normals, mask) or, with ``host=True``, pinned host sets for
    delivered results (normals, mask; the depth field is an empty tensor).

    acquire() returns a free set of the right size, or creates one if the
    budget allows, else None (the request waits). Free sets of other sizes are
    evicted (their memory returned to the allocator) when that makes room."""

    def __init__(self, budget_bytes: int, out_dtype: torch.dtype, device, host: bool = False):
        self.budget = int(budget_bytes)
        self.out_dtype = out_dtype
        self.device = device
        self.host = bool(host)
        self.free: dict = collections.defaultdict(list)
        self.reserved = 0   # bytes of all sets, free or in use
        self.in_use = 0

    @staticmethod
    def set_bytes(H: int, W: int, depth_dtype: torch.dtype, out_dtype: torch.dtype, host: bool = False) -> int:
        """Bytes of one buffer set of an H x W frame: depth (device sets only),
        normals and mask."""
        eb = 0 if host else (2 if depth_dtype == torch.uint16 else 4)
        ob = {torch.float32: 16, torch.float16: 8, torch.int16: 4}[out_dtype]
        return H * W * (eb + ob + 1)

    def acquire(self, H: int, W: int, depth_dtype: torch.dtype) -> Optional[BufferSet]:
        """A free buffer set for this frame size, a new one within the budget, or None."""
        key = (H, W, None if self.host else depth_dtype)  # host sets hold no depth
        if self.free[key]:
            b = self.free[key].pop()
            self.in_use += b.nbytes
            return b
        need = self.set_bytes(H, W, depth_dtype, self.out_dtype, self.host)
        if need > self.budget:
            raise ValueError(f"a {H}x{W} frame needs {need} bytes, more than the whole budget")
        # Evict free sets of other sizes until the new one fits.
        while self.reserved + need > self.budget:
            victim = next((k for k, v in self.free.items() if v), None)
            if victim is None:
                return None
            b = self.free[victim].pop()
            self.reserved -= b.nbytes
            del b
        channels = 2 if self.out_dtype == torch.int16 else 4
        if self.host:
            b = BufferSet(key, torch.empty(0, dtype=depth_dtype),
                          torch.empty((H, W, channels), dtype=self.out_dtype, pin_memory=True),
                          torch.empty((H, W), dtype=torch.uint8, pin_memory=True), need)
        else:
            b = BufferSet(key,
                          torch.empty((H, W), dtype=depth_dtype, device=self.device),
                          torch.empty((H, W, channels), dtype=self.out_dtype, device=self.device),
                          torch.empty((H, W), dtype=torch.uint8, device=self.device),
                          need)
        self.reserved += need
        self.in_use += need
        return b

    def release(self, b: BufferSet):
        """Returns a set to the free list (it stays allocated for reuse)."""
        self.in_use -= b.nbytes
        self.free[b.key].append(b)


@dataclass
class _Batch:
    event: torch.cuda.Event
    requests: list
    stream_index: int


class NormalServer:
    """Continuous batching over ``streams`` CUDA streams (one batched handle,
    with its own CUDA-graph slots, per stream)."""

    def __init__(self, params: NormalParams | None = None, budget_bytes: int = 40 << 30,
                 streams: int = 3, max_batch: int = 256, device=None,
                 on_done: Callable[[Request], None] | None = None, deliver: bool = True,
                 host_budget_bytes: int = 8 << 30):
        self.params = params or NormalParams()
        self.device = _device(device)
        self.pool = BufferPool(budget_bytes, self.params.torch_out_dtype, self.device)
        self.deliver = bool(deliver)
        self.host_pool = BufferPool(host_budget_bytes, self.params.torch_out_dtype, None, host=True)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.handles = [BatchedEstimator(self.params, device=self.device) for _ in range(streams)]
        self.free_streams = list(range(streams))
        self.max_batch = int(max_batch)
        self.waiting: collections.deque = collections.deque()
        self.inflight: collections.deque = collections.deque()
        self.on_done = on_done
        self.completed = 0
        self.batches = 0
        self._frames = (_lib.Frame * self.max_batch)()

    def submit(self, req: Request):
        """Queues a request; it is admitted and launched by a later poll()."""
        self.waiting.append(req)

    def busy(self) -> bool:
        """True while requests are waiting or on the GPU."""
        return bool(self.waiting or self.inflight)

    def _retire(self):
        now = None
        while self.inflight and self.inflight[0].event.query():
            b = self.inflight.popleft()
            now = time.perf_counter() if now is None else now
            for r in b.requests:
                _finish(r, now, self.on_done, self.pool, self.host_pool)
                self.completed += 1
            self.free_streams.append(b.stream_index)

    def _launch(self):
        if not self.free_streams or not self.waiting:
            return
        batch = []
        while self.waiting and len(batch) < self.max_batch:
            r = self.waiting[0]
            if not _admit(r, self.pool, self.host_pool if self.deliver else None):
                break
            self.waiting.popleft()
            batch.append(r)
        if not batch:
            return
        si = self.free_streams.pop(0)
        stream = self.streams[si]
        arr = self._frames
        t = time.perf_counter()
        with torch.cuda.stream(stream):
            for i, r in enumerate(batch):
                b = r.buffers
                b.depth.copy_(r.depth, non_blocking=True)
                f = arr[i]
                f.depth = b.depth.data_ptr()
                f.normals = b.normals.data_ptr()
                f.valid = b.valid.data_ptr()
                f.H, f.W = int(b.depth.shape[0]), int(b.depth.shape[1])
                f.depth_pitch = f.W
                f.out_pitch = f.W  # resident buffers are dense
                fx, fy, cx, cy = r.K
                f.K.fx, f.K.fy, f.K.cx, f.K.cy = float(fx), float(fy), float(cx), float(cy)
                f.in_dtype = _lib.NRM_IN_U16_MM if b.depth.dtype == torch.uint16 else _lib.NRM_IN_F32_M
                r.t_launch = t
            self.handles[si].run(arr, len(batch), stream)
            if self.deliver:
                for r in batch:
                    r.host.normals.copy_(r.buffers.normals, non_blocking=True)
                    r.host.valid.copy_(r.buffers.valid, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.append(_Batch(ev, batch, si))
        self.batches += 1

    def poll(self):
        """Retire finished batches, then admit and launch what is waiting."""
        self._retire()
        self._launch()

    def drain(self):
        """Polls until every submitted request has completed."""
        while self.busy():
            self.poll()

    def sync_status(self):
        """Raises the first device-side error any of the server's handles recorded."""
        for h in self.handles:
            h.sync_status()


def _admit(r: Request, pool: BufferPool, host_pool: Optional[BufferPool]) -> bool:
    """Device (and, when delivering, pinned host) buffers for r, or False."""
    H, W = r.depth.shape
    buf = pool.acquire(H, W, r.depth.dtype)
    if buf is None:
        return False
    if host_pool is not None:
        hb = host_pool.acquire(H, W, r.depth.dtype)
        if hb is None:
            pool.release(buf)
            return False
        r.host = hb
    r.buffers = buf
    return True


def _finish(r: Request, now: float, on_done, pool: BufferPool, host_pool: BufferPool):
    """Completes r at host time now: results to the callback, buffers back."""
    r.t_done = now
    if r.host is not None:
        r.normals, r.valid = r.host.normals, r.host.valid
    if on_done is not None:
        on_done(r)
    pool.release(r.buffers)
    r.buffers = None
    if r.host is not None:
        host_pool.release(r.host)
        r.host = None
        r.normals = r.valid = None


class PlainServer:
    """Baseline: one plain per-frame launch per request, in arrival order, on
    one stream, with the same resident-buffer pools and result delivery."""

    def __init__(self, params: NormalParams | None = None, budget_bytes: int = 40 << 30, device=None,
                 on_done: Callable[[Request], None] | None = None, deliver: bool = True,
                 host_budget_bytes: int = 8 << 30):
        self.params = params or NormalParams()
        self.device = _device(device)
        self.pool = BufferPool(budget_bytes, self.params.torch_out_dtype, self.device)
        self.deliver = bool(deliver)
        self.host_pool = BufferPool(host_budget_bytes, self.params.torch_out_dtype, None, host=True)
        self.stream = torch.cuda.Stream(self.device)
        self.estimators: collections.OrderedDict = collections.OrderedDict()
        self.waiting: collections.deque = collections.deque()
        self.inflight: collections.deque = collections.deque()
        self.on_done = on_done
        self.completed = 0

    def submit(self, req: Request):
        """Queues a request; it is admitted and launched by a later poll()."""
        self.waiting.append(req)

    def busy(self) -> bool:
        """True while requests are waiting or on the GPU."""
        return bool(self.waiting or self.inflight)

    def _estimator(self, r: Request) -> NormalEstimator:
        H, W = r.depth.shape
        key = (H, W, r.depth.dtype, tuple(r.K))
        return _cached(self.estimators, key,
                       lambda: NormalEstimator(r.K, H, W, self.params,
                                               in_dtype="u16" if r.depth.dtype == torch.uint16 else "f32",
                                               device=self.device))

    def poll(self):
        """Retire finished requests, then launch waiting ones whose buffers fit."""
        now = None
        while self.inflight and self.inflight[0][0].query():
            ev, r = self.inflight.popleft()
            now = time.perf_counter() if now is None else now
            _finish(r, now, self.on_done, self.pool, self.host_pool)
            self.completed += 1
        while self.waiting:
            r = self.waiting[0]
            if not _admit(r, self.pool, self.host_pool if self.deliver else None):
                break
            self.waiting.popleft()
            buf = r.buffers
            r.t_launch = time.perf_counter()
            with torch.cuda.stream(self.stream):
                buf.depth.copy_(r.depth, non_blocking=True)
                self._estimator(r).estimate(buf.depth, buf.normals, buf.valid, self.stream)
                if self.deliver:
                    r.host.normals.copy_(buf.normals, non_blocking=True)
                    r.host.valid.copy_(buf.valid, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.stream)
            self.inflight.append((ev, r))

    def drain(self):
        """Polls until every submitted request has completed."""
        while self.busy():
            self.poll()

    def sync_status(self):
        """Raises the first device-side error any of the server's handles recorded."""
        for est in self.estimators.values():
            est.sync_status()


def run_arrivals(server, requests: list, t0: float | None = None):
    """Feeds requests whose ``t_arrival`` holds an offset (seconds) from t0 into
    the server in real time, polling continuously; returns the wall duration.
    ``t_arrival`` is rewritten to the absolute host time of the arrival."""
    offsets = [r.t_arrival for r in requests]
    t0 = time.perf_counter() if t0 is None else t0
    i, n = 0, len(requests)
    while i < n or server.busy():
        now = time.perf_counter()
        while i < n and t0 + offsets[i] <= now:
            requests[i].t_arrival = t0 + offsets[i]
            server.submit(requests[i])
            i += 1
        server.poll()
    return time.perf_counter() - t0


def latency_summary(requests: list, duration: float) -> dict:
    """Served Mpx/s and p50 / p99 / max latency (ms) of completed requests."""
    lat = sorted(r.latency for r in requests)
    n = len(lat)
    px = sum(r.pixels for r in requests)

    def pct(q):
        return lat[min(n - 1, int(q * n))] * 1e3 if n else None

    return {"requests": n, "duration_s": round(duration, 3), "mpx_s": round(px / duration / 1e6, 1) if duration else None,
            "p50_ms": round(pct(0.50), 3) if n else None, "p99_ms": round(pct(0.99), 3) if n else None,
            "max_ms": round(lat[-1] * 1e3, 3) if n else None}
