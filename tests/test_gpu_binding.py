"""The Python binding refuses output and input tensors the library could not
write or read safely (wrong shape, dtype, layout or device), before any
launch: the C ABI takes raw pointers and cannot check them itself."""
import pytest
import torch

import paper_2209_08241_gb300 as nrm

pytestmark = pytest.mark.gpu
DEV = "cuda"
H, W = 48, 64
K = (60.0, 60.0, (W - 1) / 2, (H - 1) / 2)


def depth():
    g = torch.Generator(device="cpu").manual_seed(3)
    return (1.0 + 0.1 * torch.rand((H, W), generator=g)).to(DEV)


def bad_maps(n, m):
    """(normals, valid) pairs that must be refused, each with its reason."""
    return [
        ((torch.empty((H, W - 1, 4), device=DEV), m), "normals shape"),
        ((n.to(torch.float16), m), "normals dtype"),
        ((n, m.float()), "mask dtype"),
        ((n, m[:, : W // 2]), "mask shape"),
        ((torch.empty((W, H, 4), device=DEV).transpose(0, 1), m), "normals layout"),
        ((n.cpu(), m), "normals on the host"),
        ((n, m.cpu()), "mask on the host"),
    ]


def test_single_frame_outputs_are_checked():
    est = nrm.NormalEstimator(K, H, W)
    d = depth()
    n, m = est.new_outputs()
    for (bn, bm), why in bad_maps(n, m):
        with pytest.raises((ValueError, TypeError)):
            est(d, bn, bm)
        with pytest.raises((ValueError, TypeError)):
            est.estimate_multiscale(d, (1, 2), "pair", bn, bm)
    for bd in (d.cpu(), d[:, : W // 2], d.double()):
        with pytest.raises((ValueError, TypeError)):
            est(bd, n, m)
    with pytest.raises(ValueError):
        est(d, n, m, points=torch.empty((H, W, 3), device=DEV))
    with pytest.raises(ValueError):
        est.plane_fit(d, 2, n.cpu(), m)
    est(d, n, m)
    est.sync_status()


def test_adjoint_arguments_are_checked():
    est = nrm.NormalEstimator(K, H, W)
    d = depth()
    n, m = est(d)
    g = torch.zeros_like(n)
    with pytest.raises(ValueError):
        est.backward(d, g, m, torch.empty((H, W - 1), device=DEV))
    with pytest.raises(ValueError):
        est.backward(d, g, m, torch.empty((H, W), device="cpu"))
    with pytest.raises(ValueError):
        est.backward(d, g[..., :3].contiguous(), m)
    with pytest.raises(ValueError):
        est.backward(d, g, m.float())
    b = nrm.BatchedEstimator()
    with pytest.raises((ValueError, TypeError)):
        b.make_grad_frames([(d, K)], [g], [m], [torch.empty((H, W), dtype=torch.float64, device=DEV)])
    with pytest.raises(ValueError):
        b.make_grad_frames([(d, K)], [g.cpu()], [m])
    grad = est.backward(d, g, m)
    est.sync_status()
    assert grad.shape == (H, W)


def test_batched_outputs_are_checked():
    b = nrm.BatchedEstimator()
    d = depth()
    (n, m), = b([(d, K)])
    for (bn, bm), why in bad_maps(n, m):
        with pytest.raises((ValueError, TypeError)):
            b([(d, K)], [(bn, bm)])
    with pytest.raises(ValueError):
        b([(d.cpu(), K)])
    b.sync_status()


def test_functional_estimate_single_and_stack():
    """nrm.estimate: a (H, W) map through the single-frame handle, a (B, H, W)
    stack through one batched launch; both equal the estimator classes."""
    d = depth()
    n, m = nrm.estimate(d, K)
    ref_n, ref_m = nrm.NormalEstimator(K, H, W)(d)
    assert torch.equal(n, ref_n) and torch.equal(m, ref_m)
    stack = torch.stack([d, d.flip(0).contiguous()])
    ns, ms = nrm.estimate(stack, K)
    assert ns.shape == (2, H, W, 4) and ms.shape == (2, H, W)
    assert torch.equal(ns[0], ref_n) and torch.equal(ms[0], ref_m)
