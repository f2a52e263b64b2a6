"""CUDA stream capture: the plain single-frame launch and the batched launch
(which switches to a single kernel node with its descriptors as a kernel
parameter while the stream is capturing) are recorded into a CUDA graph, and
replays write exactly what the ordinary calls write."""
import pytest
import torch

import paper_2209_08241_gb300 as nrm
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("mode", ["global", "thread_local", "relaxed"])
@pytest.mark.parametrize("out", ["f32", "f16"])
def test_batched_call_captures_and_replays(mode, out):
    specs = [(1920, 1080, "u16"), (333, 197, "f32"), (640, 480, "u16"), (64, 64, "f32")]
    items = [scenes.random_frame(2200 + i, W, H, DEV, kind=k) for i, (W, H, k) in enumerate(specs)]
    b = nrm.BatchedEstimator(nrm.NormalParams(out_dtype=out))
    ref = [(n.clone(), m.clone()) for n, m in b(items)]
    outs = b(items)
    arr, _ = b.make_frames(items, outs)
    torch.cuda.synchronize()
    for n, m in outs:
        n.zero_()
        m.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream(), capture_error_mode=mode):
        b.run(arr, len(items), torch.cuda.current_stream())
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    b.sync_status()
    for (n, m), (rn, rm) in zip(outs, ref):
        assert torch.equal(m, rm)
        assert torch.equal(n, rn)


def test_plain_call_captures_and_replays():
    d, K = scenes.random_frame(2300, 640, 480, DEV, kind="f32")
    est = nrm.NormalEstimator(K, 480, 640)
    n0, m0 = est(d)
    n1, m1 = torch.zeros_like(n0), torch.zeros_like(m0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        est.estimate(d, n1, m1, torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(n0, n1) and torch.equal(m0, m1)


def test_capture_limits_are_reported():
    items = [scenes.random_frame(2400, 64, 48, DEV, kind="f32")] * 101
    b = nrm.BatchedEstimator()
    b(items[:2])
    arr, _ = b.make_frames(items)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(nrm._lib.NrmError):
        with torch.cuda.graph(g, stream=torch.cuda.Stream()):
            b.run(arr, len(items), torch.cuda.current_stream())
    torch.cuda.synchronize()
    # The same limit for the batched multi-scale forward (100 frames) ...
    outs = b.multiscale(items, (1, 2), "pair")
    marr, _ = b.make_frames(items, outs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(nrm._lib.NrmError):
        with torch.cuda.graph(g, stream=torch.cuda.Stream()):
            b.run_multiscale(marr, len(items), (1, 2), "pair", torch.cuda.current_stream())
    torch.cuda.synchronize()
    # ... and for the batched adjoint (60 frames).
    gitems = items[:61]
    gs = [torch.zeros_like(n) for n, _ in outs[:61]]
    grads = [torch.empty_like(d) for d, _ in gitems]
    garr, _ = b.make_grad_frames(gitems, gs, [m for _, m in outs[:61]], grads)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(nrm._lib.NrmError):
        with torch.cuda.graph(g, stream=torch.cuda.Stream()):
            b.run_backward(garr, len(gitems), torch.cuda.current_stream())
    torch.cuda.synchronize()


def test_batched_adjoint_captures_and_replays():
    W, H, n = 320, 240, 6
    items = [scenes.random_frame(2500 + i, W, H, DEV, kind="f32", holes=False, clip_range=False) for i in range(n)]
    b = nrm.BatchedEstimator()
    outs = b(items)
    gs = []
    for nm, m in outs:
        g = torch.zeros_like(nm)
        g[..., 2] = m.float()
        gs.append(g)
    ref = [x.clone() for x in b.backward(items, gs, [m for _, m in outs])]
    grads = [torch.full_like(d, 7.0) for d, _ in items]
    arr, _ = b.make_grad_frames(items, gs, [m for _, m in outs], grads)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        b.run_backward(arr, n, torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    b.sync_status()
    for x, r in zip(grads, ref):
        assert torch.equal(x, r)


def test_batched_multiscale_captures_and_replays():
    items = [scenes.random_frame(2600 + i, 320 + 64 * i, 240, DEV, kind="u16") for i in range(3)]
    b = nrm.BatchedEstimator()
    ref = [(n.clone(), m.clone()) for n, m in b.multiscale(items, (1, 2, 3), "quad")]
    outs = b.multiscale(items, (1, 2, 3), "quad")
    arr, _ = b.make_frames(items, outs)
    torch.cuda.synchronize()
    for n, m in outs:
        n.zero_()
        m.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        b.run_multiscale(arr, len(items), (1, 2, 3), "quad", torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    for (n, m), (rn, rm) in zip(outs, ref):
        assert torch.equal(m, rm) and torch.equal(n, rn)
