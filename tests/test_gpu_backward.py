"""GPU adjoint parity: nrm_backward against the oracle's complex-step VJP on
crops, against central finite differences of the GPU forward, and through the
torch.autograd.Function, for the loss L = mean over valid pixels of
(1 - n_hat . t) with random unit targets t (the differentiation workload:
640 x 480 float32 depth without holes)."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2209_08241_gb300 as nrm
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"
NT = max(1, min(16, os.cpu_count() or 1))


def frame(seed=4, W=640, H=480):
    return scenes.random_frame(4000 + seed, W, H, DEV, kind="f32", holes=False, clip_range=False)


def loss_grad(n, m, t):
    """dL/d(n_hat) of L = mean over valid of (1 - n_hat . t): -t / N_valid on valid."""
    nv = m.sum().clamp(min=1).to(torch.float32)
    g = torch.zeros_like(n)
    g[..., :3] = -t * m[..., None].float() / nv
    return g


@pytest.mark.parametrize("alpha", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("orient", [False, True])
def test_adjoint_matches_complex_step_oracle(alpha, orient):
    d, K = frame(alpha)
    H, W = d.shape
    p = nrm.NormalParams(alpha=alpha, orient_to_camera=orient)
    est = nrm.NormalEstimator(K, H, W, p)
    n, m = est(d)
    t = scenes.unit_targets(1, H, W, seed=4, device=DEV)[0]
    g = loss_grad(n, m, t)
    grad = est.backward(d, g, m)
    est.sync_status()
    dn = d.cpu().numpy()
    gn = g[..., :3].double().cpu().numpy()
    mv = m.cpu().numpy()
    for (y0, x0) in ((0, 0), (200, 300), (H - 64, W - 64), (100, 17)):
        ref = oracle.vjp(dn, K, gn, mv, alpha=alpha, orient=int(orient), crop=(y0, x0, 64, 64), nthreads=NT)
        got = grad[y0:y0 + 64, x0:x0 + 64].double().cpu().numpy()
        scale = np.abs(ref).max()
        big = np.abs(ref) > 1e-3 * scale
        rel = np.abs(got - ref)[big] / np.abs(ref)[big]
        assert rel.max() <= 1e-3, (y0, x0, rel.max())
        assert np.abs(got - ref)[~big].max(initial=0) <= 1e-3 * scale


def test_adjoint_matches_central_differences_of_gpu_forward():
    """64 random pixels with a stable mask; the FD step is the exact float32
    difference of the perturbed depths (h = 1e-4 m requested)."""
    d, K = frame(9)
    H, W = d.shape
    alpha = 2
    est = nrm.NormalEstimator(K, H, W, nrm.NormalParams(alpha=alpha))
    n, m = est(d)
    t = scenes.unit_targets(1, H, W, seed=5, device=DEV)[0]
    g = loss_grad(n, m, t)
    grad = est.backward(d, g, m).cpu().numpy()
    rng = np.random.default_rng(0)
    checked = 0
    gd = g[..., :3].double()
    while checked < 64:
        y = int(rng.integers(2 * alpha, H - 2 * alpha))
        x = int(rng.integers(2 * alpha, W - 2 * alpha))
        dp, dm = d.clone(), d.clone()
        dp[y, x] += 1e-4
        dm[y, x] -= 1e-4
        h2 = float(dp[y, x].double() - dm[y, x].double())
        n_p, m_p = est(dp)
        n_m, m_m = est(dm)
        if not (torch.equal(m_p, m) and torch.equal(m_m, m)):
            continue
        ys, xs = slice(y - alpha, y + alpha + 1), slice(x - alpha, x + alpha + 1)
        Lp = float((n_p[ys, xs, :3].double() * gd[ys, xs]).sum())
        Lm = float((n_m[ys, xs, :3].double() * gd[ys, xs]).sum())
        fd = (Lp - Lm) / h2
        a = grad[y, x]
        assert abs(a - fd) <= 2e-2 * abs(fd) + 1e-9, (y, x, a, fd)
        checked += 1


def test_autograd_function_and_determinism():
    d, K = frame(11)
    H, W = d.shape
    t = scenes.unit_targets(1, H, W, seed=6, device=DEV)[0]
    x = d.clone().requires_grad_(True)
    n, m = nrm.estimate_normals(x, K)
    assert not m.requires_grad
    valid = m.bool()
    loss = (1.0 - (n[..., :3] * t).sum(-1))[valid].mean()
    loss.backward()
    est = nrm.NormalEstimator(K, H, W)
    n2, m2 = est(d)
    g = loss_grad(n2, m2, t)
    direct = est.backward(d, g, m2)
    direct2 = est.backward(d, g, m2)
    assert torch.equal(direct, direct2)
    torch.testing.assert_close(x.grad, direct, rtol=1e-5, atol=1e-6 * direct.abs().max().item())


def test_backward_rejects_uint16_handles():
    est = nrm.NormalEstimator((100.0, 100.0, 10.0, 10.0), 20, 20, in_dtype="u16")
    d = torch.ones((20, 20), dtype=torch.uint16, device=DEV)
    n, m = est(d)
    with pytest.raises(nrm.NrmError):
        est.backward(d, torch.zeros((20, 20, 4), device=DEV), m)


def test_batch_of_32_losses():
    """The differentiation workload: 32 frames of 640 x 480, forward + adjoint
    per frame; gradients finite and zero outside the stencils of valid pixels."""
    est = nrm.NormalEstimator(scenes.intrinsics_for(640, 480), 480, 640)
    for i in range(32):
        d, K = frame(100 + i)
        n, m = est(d)
        t = scenes.unit_targets(1, 480, 640, seed=100 + i, device=DEV)[0]
        grad = est.backward(d, loss_grad(n, m, t), m)
        assert torch.isfinite(grad).all()
    est.sync_status()


@pytest.mark.parametrize("repeat", [1, 14])
def test_batched_adjoint_equals_per_frame_adjoint(repeat):
    """One nrm_backward_batched launch over frames of different sizes and
    intrinsics (ragged tails included) gives the per-frame results bit for bit:
    5 frames (descriptors as a kernel parameter) and 70 frames (descriptor ring
    in device memory)."""
    sizes = [(640, 480), (333, 197), (64, 16), (1280, 720), (100, 300)] * repeat
    frames = [scenes.random_frame(4100 + i, W, H, DEV, kind="f32", holes=True, clip_range=False)
              for i, (W, H) in enumerate(sizes)]
    b = nrm.BatchedEstimator()
    outs = b(frames)
    gs = []
    for i, ((d, K), (n, m)) in enumerate(zip(frames, outs)):
        t = scenes.unit_targets(1, d.shape[0], d.shape[1], seed=50 + i, device=DEV)[0]
        gs.append(loss_grad(n, m, t))
    grads = b.backward(frames, gs, [m for _, m in outs])
    b.sync_status()
    for (d, K), g, (n, m), gb in zip(frames, gs, outs, grads):
        est = nrm.NormalEstimator(K, d.shape[0], d.shape[1])
        ref = est.backward(d, g, m)
        est.sync_status()
        assert torch.equal(gb, ref)


def test_batch_autograd_matches_per_frame_autograd():
    B, H, W = 4, 120, 160
    frames = [frame(200 + i, W, H) for i in range(B)]
    depth = torch.stack([d for d, _ in frames])
    K = frames[0][1]
    t = scenes.unit_targets(B, H, W, seed=9, device=DEV)
    x = depth.clone().requires_grad_(True)
    n, m = nrm.estimate_normals_batch(x, K)
    valid = m.bool()
    loss = (1.0 - (n[..., :3] * t).sum(-1))[valid].mean()
    loss.backward()
    y = depth.clone().requires_grad_(True)
    total = 0.0
    nv = 0
    outs = []
    for i in range(B):
        ni, mi = nrm.estimate_normals(y[i], K)
        outs.append((ni, mi))
        nv += int(mi.sum())
    for i, (ni, mi) in enumerate(outs):
        total = total + (1.0 - (ni[..., :3] * t[i]).sum(-1))[mi.bool()].sum()
    (total / nv).backward()
    torch.testing.assert_close(x.grad, y.grad, rtol=1e-5, atol=1e-6 * y.grad.abs().max().item())


def test_scaled_adjoint_equals_adjoint_of_scaled_gradient():
    """nrm_backward_batched_scaled(t, s) is nrm_backward_batched(s * t) bit for
    bit (the kernel forms the same float32 product), for a parameter-block
    batch and a descriptor-ring batch (70 frames), with per-frame scales."""
    b = nrm.BatchedEstimator(nrm.NormalParams())
    for nfr in (3, 70):
        items = [frame(30 + i, W, H) for i, (W, H) in enumerate([(160, 120), (97, 61), (640, 480)] * 24)][:nfr]
        outs = b(items)
        ts = [scenes.unit_targets(1, d.shape[0], d.shape[1], seed=40 + i, device=DEV)[0] for i, (d, _) in enumerate(items)]
        t4 = []
        for t in ts:
            x = torch.zeros((*t.shape[:2], 4), device=DEV)
            x[..., :3] = t
            t4.append(x)
        scale = (-1.0 / torch.arange(1, nfr + 1, device=DEV, dtype=torch.float32) * 0.37).contiguous()
        arr, got = b.make_grad_frames(items, t4, [m for _, m in outs])
        b.run_backward_scaled(arr, nfr, scale)
        g4 = [t * scale[i] for i, t in enumerate(t4)]
        ref = b.backward(items, g4, [m for _, m in outs])
        torch.cuda.synchronize()
        for a, r in zip(got, ref):
            assert torch.equal(a, r)
    b.sync_status()


def test_cosine_loss_backward_matches_complex_step_oracle():
    """The fused loss entry against the oracle's VJP of L = mean over valid
    pixels of (1 - n_hat . t), per frame, on crops of two frames."""
    b = nrm.BatchedEstimator(nrm.NormalParams())
    items = [frame(50 + i) for i in range(2)]
    outs = b(items)
    t4 = []
    for i, (d, _) in enumerate(items):
        t = scenes.unit_targets(1, d.shape[0], d.shape[1], seed=60 + i, device=DEV)[0]
        x = torch.zeros((t.shape[0], t.shape[1], 4), device=DEV)
        x[..., :3] = t
        t4.append(x)
    grads, scale = b.cosine_loss_backward(items, t4, [m for _, m in outs])
    torch.cuda.synchronize()
    b.sync_status()
    for i, ((d, K), (n, m)) in enumerate(zip(items, outs)):
        assert float(scale[i]) == pytest.approx(-1.0 / float(m.sum()), rel=1e-6)
        gn = (t4[i][..., :3].double() * (-1.0 / float(m.sum())) * m[..., None].double()).cpu().numpy()
        for (y0, x0) in ((0, 0), (210, 290)):
            ref = oracle.vjp(d.cpu().numpy(), K, gn, m.cpu().numpy(), alpha=2, crop=(y0, x0, 64, 64), nthreads=NT)
            got = grads[i][y0:y0 + 64, x0:x0 + 64].double().cpu().numpy()
            sc = np.abs(ref).max()
            big = np.abs(ref) > 1e-3 * sc
            rel = np.abs(got - ref)[big] / np.abs(ref)[big]
            assert rel.max() <= 1e-3, (i, y0, x0, rel.max())
            assert np.abs(got - ref)[~big].max(initial=0) <= 1e-3 * sc


def test_scaled_adjoint_rejects_missing_scale():
    from paper_2209_08241_gb300 import _lib
    b = nrm.BatchedEstimator(nrm.NormalParams())
    items = [frame(70, 64, 48)]
    outs = b(items)
    arr, _ = b.make_grad_frames(items, [torch.zeros((48, 64, 4), device=DEV)], [outs[0][1]])
    rc = b.lib.nrm_backward_batched_scaled(b.h, arr, 1, None, None)
    assert rc == _lib.NRM_ERR_INVALID_ARG
    b.sync_status()


def test_cosine_loss_scale_counts_every_mask():
    """-1 / max(N_valid, 1) per frame from the masks, equal bit for bit to the
    same expression in float32: mixed sizes and pitches, an empty frame, an
    all-invalid frame, more than one launch's 128 frames, and repeated calls
    (the handle's counters return to zero)."""
    b = nrm.BatchedEstimator(nrm.NormalParams())
    for n in (3, 140, 5):
        items, gs, ms = [], [], []
        for i in range(n):
            W, H = [(97, 61), (640, 480), (0, 0), (130, 64), (5, 9)][i % 5]
            d = torch.rand((H, W), device=DEV) + 1.0
            K = (100.0, 100.0, W / 2, H / 2)
            items.append((d, K))
            gs.append(torch.zeros((H, W + 3, 4), device=DEV)[:, :W])  # grad_normals and mask share a pitch
            mw = torch.zeros((H, W + 3), dtype=torch.uint8, device=DEV)
            if i % 7 != 3:
                mw[:, :W] = (torch.rand((H, W), device=DEV) > 0.3).to(torch.uint8) * (1 + i % 3)
            ms.append(mw[:, :W])
        arr, _ = b.make_grad_frames(items, gs, ms)
        for _ in range(2):
            scale = b.cosine_loss_scale(arr, n)
            torch.cuda.synchronize()
            counts = torch.stack([(m != 0).sum(dtype=torch.float32) for m in ms])
            ref = -1.0 / counts.clamp(min=1.0)
            assert torch.equal(scale, ref.to(torch.float32)), n
    b.sync_status()
