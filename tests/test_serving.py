"""Served form: continuous batching with admission by a device-memory budget.

CPU tests cover the buffer pool's budget and reuse rules. GPU tests show that
each request's result is the same alone and in the mix (bit for bit: the same
per-pixel arithmetic runs whatever batch a frame lands in), that admission
never exceeds the budget, and that the per-request plain baseline agrees."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2209_08241_gb300 as nrm
from paper_2209_08241_gb300.serving import (BufferPool, NormalServer, PlainServer, Request,
                                            latency_summary, run_arrivals)
from parity import compare
from synth import scenes


def test_pool_reuses_and_respects_budget():
    per = BufferPool.set_bytes(10, 20, torch.float32, torch.float32)
    pool = BufferPool(3 * per, torch.float32, "cpu")
    a = pool.acquire(10, 20, torch.float32)
    b = pool.acquire(10, 20, torch.float32)
    c = pool.acquire(10, 20, torch.float32)
    assert pool.acquire(10, 20, torch.float32) is None      # budget full
    assert pool.reserved == 3 * per and pool.in_use == 3 * per
    pool.release(b)
    again = pool.acquire(10, 20, torch.float32)
    assert again is b                                         # resident buffer reused
    pool.release(a)
    pool.release(c)
    # A different size evicts free sets of other sizes to make room.
    small = BufferPool.set_bytes(4, 4, torch.uint16, torch.float32)
    d = pool.acquire(4, 4, torch.uint16)
    assert d is not None and pool.reserved <= 3 * per
    assert pool.reserved == 2 * per + small
    with pytest.raises(ValueError):
        pool.acquire(1000, 1000, torch.float32)               # larger than the whole budget


def test_pool_set_bytes():
    assert BufferPool.set_bytes(2, 3, torch.uint16, torch.float32) == 6 * (2 + 16 + 1)
    assert BufferPool.set_bytes(2, 3, torch.float32, torch.float16) == 6 * (4 + 8 + 1)
    # Host sets hold the delivered results only (normals and mask).
    assert BufferPool.set_bytes(2, 3, torch.uint16, torch.float32, host=True) == 6 * (16 + 1)


def _requests(n, seed=0):
    """Mixed sizes and dtypes in pinned host memory."""
    sizes = [(320, 240), (640, 480), (1280, 720), (333, 197), (1920, 1080)]
    reqs = []
    for i in range(n):
        W, H = sizes[i % len(sizes)]
        kind = "u16" if (i + seed) % 2 else "f32"
        d, K = scenes.random_frame(9000 + 31 * i + seed, W, H, "cuda", kind=kind)
        reqs.append(Request(i, d.cpu().pin_memory(), K))
    return reqs


def _collect(store):
    """Keeps each request's results as delivered to host memory, after checking
    that they are the device results."""
    def on_done(r):
        assert r.normals is not None and r.normals.device.type == "cpu" and r.normals.is_pinned()
        n, v = r.normals.clone(), r.valid.clone()
        assert torch.equal(n, r.buffers.normals.cpu()) and torch.equal(v, r.buffers.valid.cpu())
        store[r.rid] = (n, v)
    return on_done


@pytest.mark.gpu
def test_same_result_alone_and_in_the_mix():
    reqs = _requests(14)
    alone = {}
    for r in reqs:
        srv = NormalServer(streams=2, on_done=_collect(alone))
        srv.submit(Request(r.rid, r.depth, r.K))
        srv.drain()
        srv.sync_status()
    mix = {}
    srv = NormalServer(streams=3, on_done=_collect(mix))
    rng = np.random.default_rng(1)
    offsets = np.cumsum(rng.exponential(1 / 2000.0, size=len(reqs)))  # Poisson, 2000 frames/s
    mixed = [Request(r.rid, r.depth, r.K, t_arrival=float(o)) for r, o in zip(reqs, offsets)]
    run_arrivals(srv, mixed)
    srv.sync_status()
    assert srv.completed == len(reqs)
    for r in reqs:
        na, ma = alone[r.rid]
        nb, mb = mix[r.rid]
        assert torch.equal(na, nb) and torch.equal(ma, mb), r.rid
    # And the mix against the oracle on a few frames.
    p = nrm.NormalParams()
    for r in reqs[:3]:
        ref = oracle.forward(r.depth.numpy(), r.K, alpha=p.alpha, stat_mode=oracle.STAT_SECANT, tau=p.tau,
                             depth_scale=p.depth_scale, nthreads=8)
        compare(mix[r.rid][0], mix[r.rid][1], ref, p.tau, what=f"served #{r.rid}")
    s = latency_summary(mixed, 1.0)
    assert s["requests"] == len(reqs) and s["p50_ms"] > 0


@pytest.mark.gpu
def test_admission_is_bounded_by_the_budget():
    reqs = _requests(10, seed=1)
    largest = max(BufferPool.set_bytes(r.depth.shape[0], r.depth.shape[1], r.depth.dtype, torch.float32)
                  for r in reqs)
    budget = 2 * largest
    peak = {"reserved": 0}
    out = {}

    def on_done(r):
        peak["reserved"] = max(peak["reserved"], srv.pool.reserved)
        out[r.rid] = r.buffers.valid.sum().item()

    srv = NormalServer(budget_bytes=budget, streams=3, on_done=on_done)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    srv.sync_status()
    assert srv.completed == len(reqs) and len(out) == len(reqs)
    assert peak["reserved"] <= budget
    assert srv.batches >= 2   # the budget forced the requests into more than one batch


@pytest.mark.gpu
def test_plain_baseline_agrees_with_batched_server():
    reqs = _requests(6, seed=2)
    a, b = {}, {}
    srv = NormalServer(on_done=_collect(a))
    for r in reqs:
        srv.submit(Request(r.rid, r.depth, r.K))
    srv.drain()
    base = PlainServer(on_done=_collect(b))
    for r in reqs:
        base.submit(Request(r.rid, r.depth, r.K))
    base.drain()
    base.sync_status()
    for r in reqs:
        assert torch.equal(a[r.rid][0], b[r.rid][0]) and torch.equal(a[r.rid][1], b[r.rid][1])


@pytest.mark.gpu
def test_results_stay_on_the_device_without_delivery():
    reqs = _requests(4, seed=3)
    got = {}

    def on_done(r):
        assert r.normals is None and r.host is None
        got[r.rid] = (r.buffers.normals.clone(), r.buffers.valid.clone())

    srv = NormalServer(on_done=on_done, deliver=False)
    for r in reqs:
        srv.submit(Request(r.rid, r.depth, r.K))
    srv.drain()
    srv.sync_status()
    ref = {}
    srv2 = NormalServer(on_done=_collect(ref))
    for r in reqs:
        srv2.submit(Request(r.rid, r.depth, r.K))
    srv2.drain()
    for r in reqs:
        assert torch.equal(got[r.rid][0].cpu(), ref[r.rid][0]) and torch.equal(got[r.rid][1].cpu(), ref[r.rid][1])
    assert srv2.host_pool.in_use == 0 and srv2.pool.in_use == 0
