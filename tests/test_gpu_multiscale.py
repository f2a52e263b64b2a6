"""GPU multi-scale variant (Section 2's average over pixel distances, with the
previous method's single-pair stencil of Eq. 1-3 or the four-direction stencil
of Eq. 4-6) against the FP64 multi-scale oracle, element by element.

Tolerances: normals 1e-4 rad (FP32 output) / 5e-3 rad (half), masks bit-exact
except pixels whose oracle statistic lies within 1e-6 kappa relative of tau,
kappa being the per-pixel cancellation factor of the scale average (see
parity.compare_ms). With one scale the four-direction variant must equal the
single-scale kernel bit for bit."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2209_08241_gb300 as nrm
from oracle.multiscale import multiscale
from parity import ANG_TOL_OCT16, angles, compare_ms, decode_oct16, ms_kappa
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


def stat_mode(p):
    return oracle.STAT_SECANT if p.mask_mode == "secant" else oracle.STAT_RAW


def run(depth, K, p, alphas, form):
    in_dtype = "u16" if depth.dtype == torch.uint16 else "f32"
    H, W = depth.shape
    est = nrm.NormalEstimator(K, H, W, p, in_dtype=in_dtype)
    n, m = est.estimate_multiscale(depth, alphas, form)
    est.sync_status()
    D = depth.cpu().numpy()
    ref = multiscale(D, K, alphas, form, stat_mode(p), p.tau, p.depth_scale, int(p.orient_to_camera))
    kappa = ms_kappa(D, K, alphas, form, p.depth_scale)
    return n, m, ref, kappa


@pytest.fixture(scope="module")
def cfg1():
    return scenes.cfg1_depth(DEV)


@pytest.mark.parametrize("form", ["pair", "quad"])
@pytest.mark.parametrize("alphas", [(1, 2, 3, 4), (2,), (1, 3, 8)])
@pytest.mark.parametrize("mode", ["secant", "raw"])
def test_cfg1_parity(cfg1, form, alphas, mode):
    d, K = cfg1
    tau = 12.0
    if mode == "raw":
        # Split the valid pixels: tau at the median length of the averaged n.
        r = multiscale(d.cpu().numpy(), K, alphas, form, oracle.STAT_RAW, np.inf).r
        tau = float(np.nanmedian(r))
    p = nrm.NormalParams(mask_mode=mode, tau=tau)
    n, m, ref, kappa = run(d, K, p, list(alphas), form)
    near, ang, nv, mk = compare_ms(n, m, ref, tau, kappa, what=f"cfg1 {form} {alphas} {mode}")
    assert nv > 0.3 * d.numel()
    print(f"{form} {alphas} {mode}: max angle {ang:.2e} rad, near-tau {near}, max kappa {mk:.3g}")


@pytest.mark.parametrize("form", ["pair", "quad"])
def test_cfg1_half_output(cfg1, form):
    d, K = cfg1
    p = nrm.NormalParams(out_dtype="f16")
    n, m, ref, kappa = run(d, K, p, [1, 2, 3, 4], form)
    compare_ms(n, m, ref, p.tau, kappa, half=True, what=f"cfg1 {form} f16")


@pytest.mark.parametrize("shape", [(197, 333), (481, 641), (37, 70)])
@pytest.mark.parametrize("form,alphas", [("pair", (1, 2, 3, 4)), ("quad", (1, 2)), ("pair", (16,)), ("quad", (1, 16))])
@pytest.mark.parametrize("orient", [False, True])
def test_u16_ragged_with_holes(shape, form, alphas, orient):
    H, W = shape
    d, K = scenes.random_frame(700 + H + W, W, H, DEV, kind="u16")
    p = nrm.NormalParams(orient_to_camera=orient)
    n, m, ref, kappa = run(d, K, p, list(alphas), form)
    compare_ms(n, m, ref, p.tau, kappa, what=f"u16 {shape} {form} {alphas} orient={orient}")


@pytest.mark.parametrize("alpha", [1, 2, 5])
@pytest.mark.parametrize("kind", ["f32", "u16"])
@pytest.mark.parametrize("out", ["f32", "oct16"])
def test_one_quad_scale_equals_the_single_scale_kernel(alpha, kind, out):
    """K = 1 with the four-direction stencil is the method itself: same
    constants, same operations, so the outputs are identical bit for bit."""
    d, K = scenes.random_frame(900 + alpha, 641, 479, DEV, kind=kind)
    p = nrm.NormalParams(alpha=alpha, out_dtype=out)
    est = nrm.NormalEstimator(K, 479, 641, p, in_dtype=kind)
    n1, m1 = est.estimate(d)
    n2, m2 = est.estimate_multiscale(d, [alpha], "quad")
    est.sync_status()
    assert torch.equal(m1, m2)
    assert torch.equal(n1, n2)


@pytest.mark.parametrize("out", ["f32", "f16", "oct16"])
@pytest.mark.parametrize("form", ["pair", "quad"])
def test_pitched_outputs_give_the_same_bits(out, form):
    """The same frames written to contiguous outputs and to outputs with an
    odd row pitch (mask bytes then stored one by one instead of four at a
    time) give the same bits, for several scale sets."""
    b = nrm.BatchedEstimator(nrm.NormalParams(out_dtype=out))
    C = 2 if out == "oct16" else 4
    dt = {"f32": torch.float32, "f16": torch.float16, "oct16": torch.int16}[out]
    items = [scenes.random_frame(950 + i, W, H, DEV, kind=kind)
             for i, (W, H, kind) in enumerate([(640, 480, "u16"), (517, 300, "f32"), (1920, 1080, "u16")])]
    for alphas in [(1, 2, 3, 4), (3,), (2, 4), (1,), (4, 1), (1, 5)]:
        vec = b.multiscale(items, alphas, form)
        outs = []
        for d, _ in items:
            H, W = d.shape
            nb = torch.zeros((H, W + 1, C), dtype=dt, device=DEV)
            vb = torch.zeros((H, W + 1), dtype=torch.uint8, device=DEV)
            outs.append((nb[:, :W], vb[:, :W]))
        sca = b.multiscale(items, alphas, form, outputs=outs)
        b.sync_status()
        for (n1, m1), (n2, m2) in zip(vec, sca):
            assert torch.equal(m1, m2), (out, form, alphas)
            assert torch.equal(n1, n2), (out, form, alphas)


def test_oct16_output_matches_float_output():
    d, K = scenes.random_frame(77, 640, 480, DEV, kind="u16")
    ef = nrm.NormalEstimator(K, 480, 640, nrm.NormalParams(), in_dtype="u16")
    eo = nrm.NormalEstimator(K, 480, 640, nrm.NormalParams(out_dtype="oct16"), in_dtype="u16")
    nf, mf = ef.estimate_multiscale(d, [1, 2, 3, 4], "pair")
    no, mo = eo.estimate_multiscale(d, [1, 2, 3, 4], "pair")
    ef.sync_status()
    eo.sync_status()
    assert torch.equal(mf, mo)
    v = mf.cpu().numpy() == 1
    codes = no.cpu().numpy()
    assert (codes[~v] == 0).all()
    ang = angles(decode_oct16(codes[v]), nf.cpu().numpy()[v][:, :3])
    assert ang.max() <= ANG_TOL_OCT16


def test_fullsize_1080p_u16():
    """The bench's frame size and input type, compared pixel by pixel."""
    d, K = scenes.random_frame(1000, 1920, 1080, DEV, kind="u16")
    p = nrm.NormalParams()
    n, m, ref, kappa = run(d, K, p, [1, 2, 3, 4], "pair")
    near, ang, nv, mk = compare_ms(n, m, ref, p.tau, kappa, what="1080p u16 pair 1-4")
    assert nv > 0.5 * 1920 * 1080


def test_bad_scales_are_rejected():
    est = nrm.NormalEstimator((100.0, 100.0, 10.0, 10.0), 20, 20)
    d = torch.ones((20, 20), device=DEV)
    for alphas in ([], [1] * 9, [0], [17], [1, -2]):
        with pytest.raises((nrm._lib.NrmError, ValueError)):
            est.estimate_multiscale(d, alphas)
    n, m = est.new_outputs()
    sc = nrm._lib.Scales()
    sc.n_scales = 1
    sc.alpha[0] = 1
    sc.form = 2
    rc = est.lib.nrm_estimate_multiscale(est.h, d.data_ptr(), n.data_ptr(), m.data_ptr(), ctypes.byref(sc), None)
    assert rc == nrm._lib.NRM_ERR_INVALID_ARG
    assert est.lib.nrm_estimate_multiscale(est.h, d.data_ptr(), n.data_ptr(), m.data_ptr(), None, None) \
        == nrm._lib.NRM_ERR_INVALID_ARG


@pytest.mark.parametrize("form,alphas", [("pair", (1, 2, 3, 4)), ("quad", (1, 2, 3, 4)), ("pair", (1, 16)),
                                         ("quad", (3,))])
def test_batched_mixed_sizes_dtypes_and_intrinsics(form, alphas):
    specs = [(1920, 1080, "u16"), (333, 197, "f32"), (640, 480, "u16"), (64, 64, "f32"), (17, 9, "f32")]
    items = [scenes.random_frame(1600 + i, W, H, DEV, kind=k) for i, (W, H, k) in enumerate(specs)]
    b = nrm.BatchedEstimator()
    outs = b.multiscale(items, alphas, form)
    b.sync_status()
    p = nrm.NormalParams()
    for (d, K), (n, m), (W, H, k) in zip(items, outs, specs):
        D = d.cpu().numpy()
        ref = multiscale(D, K, list(alphas), form, stat_mode(p), p.tau, p.depth_scale, 0)
        kappa = ms_kappa(D, K, list(alphas), form, p.depth_scale)
        compare_ms(n, m, ref, p.tau, kappa, what=f"batched {form} {alphas} {W}x{H} {k}")


def test_batched_half_and_orientation():
    items = [scenes.random_frame(1700 + i, 320, 240, DEV, kind="u16") for i in range(3)]
    b = nrm.BatchedEstimator(nrm.NormalParams(out_dtype="f16", orient_to_camera=True))
    outs = b.multiscale(items, (1, 2), "pair")
    b.sync_status()
    p = nrm.NormalParams()
    for (d, K), (n, m) in zip(items, outs):
        D = d.cpu().numpy()
        ref = multiscale(D, K, [1, 2], "pair", stat_mode(p), p.tau, p.depth_scale, 1)
        compare_ms(n, m, ref, p.tau, ms_kappa(D, K, [1, 2], "pair"), half=True, what="batched f16 orient")


def test_batched_multiscale_rejects_point_buffers():
    d, K = scenes.random_frame(1800, 64, 48, DEV, kind="f32")
    b = nrm.BatchedEstimator()
    n = torch.empty((48, 64, 4), device=DEV)
    m = torch.empty((48, 64), dtype=torch.uint8, device=DEV)
    P = torch.empty((48, 64, 4), device=DEV)
    arr, _ = b.make_frames([(d, K)], [(n, m, P)])
    with pytest.raises(nrm._lib.NrmError):
        b.run_multiscale(arr, 1)


def test_batched_multiscale_ring_path_for_large_batches():
    """More than 100 frames take the device descriptor ring; the results equal
    those of the same frames in small (parameter-path) batches."""
    items = [scenes.random_frame(1750 + (i % 7), 96, 64, DEV, kind="u16") for i in range(105)]
    b = nrm.BatchedEstimator()
    big = b.multiscale(items, (1, 2), "pair")
    small = []
    for k in range(0, 105, 35):
        small += b.multiscale(items[k:k + 35], (1, 2), "pair")
    b.sync_status()
    for (n1, m1), (n2, m2) in zip(big, small):
        assert torch.equal(m1, m2) and torch.equal(n1, n2)
