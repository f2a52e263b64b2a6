"""GPU organised point-cloud output (Section 2 back-projection, written in the
same pass as the normals) against the FP64 point-cloud oracle.

Tolerance: each coordinate is z u1 (or z v1, z) with z = d times the depth
scale (one rounding) and u1 = (col - cx) / fx formed in FP32 (two roundings),
so a point differs from the FP64 one by at most a few ulp of its length:
5e-7 |P| per pixel. Invalid depth gives exactly (0, 0, 0, 0). Writing points
must not change the normal map or the mask: they are compared bit for bit with
the same call without points."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2209_08241_gb300 as nrm
from oracle.pointcloud import points as oracle_points
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"
REL = 5e-7


def check_points(P, depth, K, scale=0.001, what=""):
    P = P.cpu().numpy().astype(np.float64)
    ref = oracle_points(depth.cpu().numpy(), K, scale)
    assert (P[..., 3] == 0).all(), what
    err = np.linalg.norm(P[..., :3] - ref, axis=-1)
    bound = REL * np.linalg.norm(ref, axis=-1)
    assert (err <= bound).all(), f"{what}: {int((err > bound).sum())} points off, worst {float(err.max()):.3g}"
    invalid = np.linalg.norm(ref, axis=-1) == 0
    assert (P[invalid] == 0).all(), f"{what}: invalid depth must give the origin"


@pytest.mark.parametrize("kind", ["f32", "u16"])
@pytest.mark.parametrize("shape", [(197, 333), (480, 640), (7, 5)])
@pytest.mark.parametrize("out", ["f32", "f16", "oct16"])
def test_plain_points(kind, shape, out):
    H, W = shape
    d, K = scenes.random_frame(1300 + H, W, H, DEV, kind=kind)
    p = nrm.NormalParams(out_dtype=out)
    est = nrm.NormalEstimator(K, H, W, p, in_dtype=kind)
    n0, m0 = est.estimate(d)
    P = torch.full((H, W, 4), 7.0, device=DEV)
    n1, m1 = est.estimate(d, points=P)
    est.sync_status()
    assert torch.equal(m0, m1) and torch.equal(n0, n1)
    check_points(P, d, K, what=f"{kind} {shape} {out}")


def test_batched_points_mixed_with_frames_without():
    specs = [(1920, 1080, "u16", True), (333, 197, "f32", False), (640, 480, "u16", True), (64, 64, "f32", True)]
    items = [scenes.random_frame(1400 + i, W, H, DEV, kind=k) for i, (W, H, k, _) in enumerate(specs)]
    b = nrm.BatchedEstimator()
    ref_outs = b(items)
    outs = []
    for (d, K), (W, H, k, want) in zip(items, specs):
        nm = torch.empty((H, W, 4), device=DEV)
        vm = torch.empty((H, W), dtype=torch.uint8, device=DEV)
        outs.append((nm, vm, torch.full((H, W, 4), 3.0, device=DEV)) if want else (nm, vm))
    got = b(items, outs)
    b.sync_status()
    for (d, K), o, r, (W, H, k, want) in zip(items, got, ref_outs, specs):
        assert torch.equal(o[0], r[0]) and torch.equal(o[1], r[1])
        if want:
            check_points(o[2], d, K, what=f"batched {W}x{H} {k}")
    # The next batch without points reuses the slot with the normal-only kernel.
    again = b(items, [(o[0], o[1]) for o in got])
    b.sync_status()
    for o, r in zip(again, ref_outs):
        assert torch.equal(o[0], r[0]) and torch.equal(o[1], r[1])


def test_points_argument_checks():
    d, K = scenes.random_frame(1500, 64, 48, DEV, kind="f32")
    est = nrm.NormalEstimator(K, 48, 64)
    n, m = est.new_outputs()
    buf = torch.empty(48 * 64 * 4 + 4, device=DEV)
    lib = est.lib
    rc = lib.nrm_estimate_points(est.h, d.data_ptr(), n.data_ptr(), m.data_ptr(), buf.data_ptr() + 4, None)
    assert rc == nrm._lib.NRM_ERR_INVALID_ARG
    rc = lib.nrm_estimate_points(est.h, d.data_ptr(), n.data_ptr(), m.data_ptr(), None, None)
    assert rc == nrm._lib.NRM_ERR_INVALID_ARG
    # The allocation-free entry point writes no point clouds and says so.
    f = nrm._lib.Frame()
    f.depth, f.normals, f.valid = d.data_ptr(), n.data_ptr(), m.data_ptr()
    f.H, f.W, f.depth_pitch, f.out_pitch = 48, 64, 64, 64
    f.K = nrm._lib.Intrinsics(*K)
    f.in_dtype = nrm._lib.NRM_IN_F32_M
    P = torch.empty((48, 64, 4), device=DEV)
    f.points = P.data_ptr()
    arr = (nrm._lib.Frame * 1)(f)
    assert lib.nrm_estimate_batched_noalloc(arr, 1, None, None, None) == nrm._lib.NRM_ERR_UNSUPPORTED


def test_host_buffer_entry_point_matches_device_batch():
    """nrm_estimate_batched_host (host buffers, chunked on internal streams)
    returns what the device batch returns, bit for bit, including points.
    Nine 1280 x 720 frames make three chunks on the two internal streams."""
    n, H, W = 9, 720, 1280
    items = [scenes.random_frame(1900 + i, W, H, DEV, kind="u16") for i in range(n)]
    depth = torch.stack([d for d, _ in items])
    Ks = [K for _, K in items]
    b = nrm.BatchedEstimator()
    P = torch.empty((n, H, W, 4), device=DEV)
    ref = b([(depth[i], Ks[i]) for i in range(n)],
            [(torch.empty((H, W, 4), device=DEV), torch.empty((H, W), dtype=torch.uint8, device=DEV), P[i])
             for i in range(n)])
    hd = depth.cpu().pin_memory()
    hn = torch.empty((n, H, W, 4), pin_memory=True)
    hv = torch.empty((n, H, W), dtype=torch.uint8, pin_memory=True)
    hp = torch.empty((n, H, W, 4), pin_memory=True)
    s = torch.cuda.Stream()
    frames = b.run_host(hd, Ks, hn, hv, stream=s, points_host=hp)
    s.synchronize()
    for i in range(n):
        assert torch.equal(hn[i], ref[i][0].cpu())
        assert torch.equal(hv[i], ref[i][1].cpu())
        assert torch.equal(hp[i], ref[i][2].cpu())
    # Reusing the frame array on the default stream gives the same again.
    hn.zero_()
    b.run_host(hd, Ks, hn, hv, frames=frames)
    torch.cuda.synchronize()
    assert torch.equal(hn[n - 1], ref[n - 1][0].cpu())
