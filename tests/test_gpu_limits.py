"""Frames at the size limits, against the FP64 oracle: long thin frames (many
tiles along one axis, ragged tails on both), and frames with more tile rows
than one launch grid holds (65535), which the single-frame calls run as
one-frame batches."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2209_08241_gb300 as nrm
from oracle.multiscale import multiscale as oracle_multiscale
from parity import compare, compare_ms, ms_kappa

pytestmark = pytest.mark.gpu
DEV = "cuda"
NT = max(1, min(16, os.cpu_count() or 1))


def axis_term(n, seed):
    """Depth variation along an axis of n pixels: three slow periods on a long
    axis (surface slopes up to ~2 when the focal length is n pixels), a 1 mm
    per pixel ramp on a short one."""
    i = torch.arange(n, dtype=torch.float64)
    if n > 1000:
        return 0.2 * torch.sin(2 * np.pi * (3 * i / n + 0.1 * seed))
    return 0.001 * i


def smooth_depth(H, W, seed, kind="f32"):
    d = 2.0 + axis_term(H, seed)[:, None] + axis_term(W, seed)[None, :]
    if kind == "u16":
        return (d * 1000.0).round().to(torch.int32).to(torch.uint16)
    return d.float()


def run_oracle(d, K, p: nrm.NormalParams):
    mode = oracle.STAT_SECANT if p.mask_mode == "secant" else oracle.STAT_RAW
    return oracle.forward(d.numpy(), K, alpha=p.alpha, stat_mode=mode, tau=p.tau, depth_scale=p.depth_scale,
                          orient=int(p.orient_to_camera), nthreads=NT)


@pytest.mark.parametrize("shape,kind,alpha", [((3, 150001), "f32", 1), ((200003, 5), "u16", 2)])
def test_long_thin_frames(shape, kind, alpha):
    H, W = shape
    d = smooth_depth(H, W, 31 + W, kind)
    K = (float(max(W, 100)), float(max(H, 100)), (W - 1) / 2, (H - 1) / 2)
    p = nrm.NormalParams(alpha=alpha)
    est = nrm.NormalEstimator(K, H, W, p, in_dtype=kind)
    n, m = est(d.to(DEV))
    est.sync_status()
    near, _, n_valid = compare(n, m, run_oracle(d, K, p), p.tau, what=f"thin {shape}")
    assert n_valid > 0
    b = nrm.BatchedEstimator(p)
    (nb, mb), = b([(d.to(DEV), K)])
    b.sync_status()
    assert torch.equal(nb, n) and torch.equal(mb, m)


def test_forward_beyond_one_launch_grid_of_tile_rows():
    """65535 x 16 + 40 rows with 16-row tiles: nrm_estimate runs the frame as
    a one-frame batch; results equal the oracle and the batched call."""
    H, W = 65535 * 16 + 40, 4
    d = smooth_depth(H, W, 7)
    K = (500.0, float(H), (W - 1) / 2, (H - 1) / 2)
    p = nrm.NormalParams(alpha=1)
    est = nrm.NormalEstimator(K, H, W, p)
    est.set_config(128, 16, 256)
    n, m = est(d.to(DEV))
    est.sync_status()
    _, _, n_valid = compare(n, m, run_oracle(d, K, p), p.tau, what="tall forward")
    assert n_valid > H
    b = nrm.BatchedEstimator(p)
    (nb, mb), = b([(d.to(DEV), K)])
    b.sync_status()
    assert torch.equal(nb, n) and torch.equal(mb, m)


def test_adjoint_beyond_one_launch_grid_of_tile_rows():
    """More than 65535 adjoint tile rows: nrm_backward runs the frame as a
    one-frame batched adjoint; the gradient equals the batched call's, and on
    the interior it is nonzero."""
    H, W = 65535 * 32 + 40, 6
    d = smooth_depth(H, W, 8).to(DEV)
    K = (500.0, float(H), (W - 1) / 2, (H - 1) / 2)
    p = nrm.NormalParams(alpha=1)
    est = nrm.NormalEstimator(K, H, W, p)
    n, m = est(d)
    g = torch.zeros_like(n)
    g[..., 2] = m.float()
    grad = est.backward(d, g, m)
    est.sync_status()
    b = nrm.BatchedEstimator(p)
    gb, = b.backward([(d, K)], [g], [m])
    b.sync_status()
    assert torch.equal(grad, gb)
    assert torch.isfinite(grad).all() and (grad[2:-2, 2:-2] != 0).any()


def test_multiscale_beyond_one_launch_grid_of_tile_rows():
    H, W = 65535 * 16 + 40, 7
    d = smooth_depth(H, W, 9)
    K = (500.0, float(H), (W - 1) / 2, (H - 1) / 2)
    p = nrm.NormalParams()
    est = nrm.NormalEstimator(K, H, W, p)
    n, m = est.estimate_multiscale(d.to(DEV), (1, 2), "pair")
    est.sync_status()
    dn = d.numpy()
    ref = oracle_multiscale(dn, K, (1, 2), "pair", oracle.STAT_SECANT, p.tau)
    _, _, n_valid, _ = compare_ms(n, m, ref, p.tau, ms_kappa(dn, K, (1, 2), "pair"), what="tall multiscale")
    assert n_valid > H


def test_plane_fit_rejects_too_many_tile_rows():
    H, W = 65535 * 8 + 8, 4
    d = torch.ones((H, W), device=DEV)
    est = nrm.NormalEstimator((500.0, float(H), 1.5, (H - 1) / 2), H, W)
    with pytest.raises(nrm._lib.NrmError):
        est.plane_fit(d, 1)
    est.sync_status()


@pytest.mark.parametrize("k", [2.0 ** -18, 2.0 ** 33])
def test_numerical_domain_ends_match_oracle(k):
    """Depths at both ends of the documented FP32 domain (2^-28 <= alpha d / f
    <= 2^28): a float32 scene scaled to about 1.5e-6 .. 2.3e-5 m and to
    3.4e9 .. 5.2e10 m against the FP64 oracle, for alpha = 1 and 2."""
    from synth import scenes
    d0, K = scenes.random_frame(91, 640, 480, "cpu", kind="f32")
    d = (d0.double() * k).float()
    for alpha in (1, 2):
        p = nrm.NormalParams(alpha=alpha)
        est = nrm.NormalEstimator(K, 480, 640, p)
        n, m = est(d.cuda())
        est.sync_status()
        ref = oracle.forward(d.numpy(), K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=p.tau, nthreads=8)
        near, ang, nv = compare(n, m, ref, p.tau, what=f"k={k} alpha={alpha}")
        assert nv > 100000
