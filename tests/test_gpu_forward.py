"""GPU forward parity: the CUDA kernels (through the C ABI) against the FP64
oracle on the same seeded inputs, element by element, at sizes that span
several tiles with ragged tails, plus edge cases."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2209_08241_gb300 as nrm
from parity import compare, compare_oct16, decode_oct16
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"
NT = max(1, min(16, os.cpu_count() or 1))

# Every compiled (tile_x, tile_y, threads) configuration.
CONFIGS = [(128, 16, 256), (128, 8, 256), (128, 32, 256), (128, 8, 128), (128, 16, 128),
           (128, 32, 512), (128, 64, 512), (64, 16, 128), (64, 32, 256), (64, 64, 256)]


def run_oracle(depth, K, p: nrm.NormalParams):
    d = depth.cpu().numpy() if isinstance(depth, torch.Tensor) else depth
    mode = oracle.STAT_SECANT if p.mask_mode == "secant" else oracle.STAT_RAW
    return oracle.forward(d, K, alpha=p.alpha, stat_mode=mode, tau=p.tau, depth_scale=p.depth_scale,
                          orient=int(p.orient_to_camera), nthreads=NT)


def plain(depth, K, p, in_dtype=None):
    in_dtype = in_dtype or ("u16" if depth.dtype == torch.uint16 else "f32")
    est = nrm.NormalEstimator(K, depth.shape[0], depth.shape[1], p, in_dtype=in_dtype)
    n, m = est(depth)
    est.sync_status()
    return n, m


@pytest.fixture(scope="module")
def cfg1():
    d, K = scenes.cfg1_depth(DEV)
    return d, K


@pytest.mark.parametrize("alpha", [1, 2, 3])
@pytest.mark.parametrize("mode,tau", [("secant", 12.0), ("secant", 1.5), ("raw", 2e-4)])
@pytest.mark.parametrize("out", ["f32", "f16"])
def test_cfg1_plain_parity(cfg1, alpha, mode, tau, out):
    d, K = cfg1
    p = nrm.NormalParams(alpha=alpha, mask_mode=mode, tau=tau, out_dtype=out)
    n, m = plain(d, K, p)
    ref = run_oracle(d, K, p)
    near, ang, nv = compare(n, m, ref, tau, half=(out == "f16"), what=f"cfg1 a{alpha} {mode} {out}")
    # A tight secant threshold with alpha = 1 masks most noisy pixels; the
    # default one keeps the smooth surfaces.
    assert nv > (0.5 if tau == 12.0 else 0.05) * d.numel()
    print(f"alpha={alpha} {mode} tau={tau} {out}: max angle {ang:.2e} rad, near-tau excluded {near}")


def test_cfg1_masks_discontinuities(cfg1):
    """The sphere and the patch produce depth steps: the secant mask removes a
    band along them and keeps the smooth surfaces."""
    d, K = cfg1
    p = nrm.NormalParams()
    _, m = plain(d, K, p)
    frac = 1.0 - m.float().mean().item()
    assert 0.005 < frac < 0.2


@pytest.mark.parametrize("shape", [(197, 333), (240, 320), (481, 641), (1080, 1920)])
@pytest.mark.parametrize("out", ["f32", "f16"])
def test_u16_plain_parity_ragged(shape, out):
    H, W = shape
    d, K = scenes.random_frame(77 + W, W, H, DEV, kind="u16")
    p = nrm.NormalParams(alpha=2, out_dtype=out)
    n, m = plain(d, K, p)
    ref = run_oracle(d, K, p)
    compare(n, m, ref, p.tau, half=(out == "f16"), what=f"u16 {shape} {out}")


@pytest.mark.parametrize("shape", [(0, 0), (1, 1), (3, 7), (5, 5), (4, 129), (130, 3), (17, 200), (2, 300)])
@pytest.mark.parametrize("alpha", [1, 2])
def test_tiny_and_degenerate_maps(shape, alpha):
    H, W = shape
    if H == 0:
        b = nrm.BatchedEstimator(alpha=alpha)
        d = torch.zeros((0, 0), device=DEV)
        assert b([(d, (1.0, 1.0, 0.0, 0.0))]) is not None
        b.sync_status()
        return
    g = torch.Generator(device="cpu").manual_seed(H * 1000 + W)
    d = (1.0 + 0.3 * torch.rand((H, W), generator=g)).to(DEV)
    K = (40.0, 42.0, (W - 1) / 2, (H - 1) / 2)
    p = nrm.NormalParams(alpha=alpha)
    n, m = plain(d, K, p)
    compare(n, m, run_oracle(d, K, p), p.tau, what=f"tiny {shape}")
    b = nrm.BatchedEstimator(alpha=alpha)
    (nb, mb), = b([(d, K)])
    b.sync_status()
    assert torch.equal(nb, n) and torch.equal(mb, m)


def test_special_depth_values():
    """0, negative, NaN and infinite depths invalidate exactly the pixels whose
    stencil holds them."""
    H, W = 70, 150
    g = torch.Generator(device="cpu").manual_seed(5)
    d = 1.0 + 0.5 * torch.rand((H, W), generator=g)
    idx = torch.randint(0, H * W, (200,), generator=g)
    vals = torch.tensor([0.0, -1.0, float("nan"), float("inf"), -float("inf")])
    d.view(-1)[idx] = vals[torch.arange(200) % 5]
    d = d.to(DEV)
    K = (100.0, 100.0, 74.5, 34.5)
    for alpha in (1, 2, 5):
        p = nrm.NormalParams(alpha=alpha)
        n, m = plain(d, K, p)
        compare(n, m, run_oracle(d, K, p), p.tau, what=f"special a{alpha}")


def test_alpha_limits(cfg1):
    d, K = cfg1
    for alpha in (8, 16):
        p = nrm.NormalParams(alpha=alpha)
        n, m = plain(d, K, p)
        compare(n, m, run_oracle(d, K, p), p.tau, what=f"alpha {alpha}")
    with pytest.raises(nrm.NrmError):
        nrm.NormalEstimator(K, 480, 640, nrm.NormalParams(alpha=17))


def test_orientation_flag(cfg1):
    d, K = cfg1
    n0, m0 = plain(d, K, nrm.NormalParams())
    n1, m1 = plain(d, K, nrm.NormalParams(orient_to_camera=True))
    assert torch.equal(m0, m1)
    assert torch.equal(n1[..., :3], -n0[..., :3])
    ref = run_oracle(d, K, nrm.NormalParams(orient_to_camera=True))
    compare(n1, m1, ref, 12.0, what="orient")


@pytest.mark.parametrize("cfg", CONFIGS)
def test_every_tile_config_is_bitwise_identical(cfg1, cfg):
    """All compiled tile shapes compute the same per-pixel arithmetic."""
    d, K = cfg1
    p = nrm.NormalParams()
    base_n, base_m = plain(d, K, p)
    est = nrm.NormalEstimator(K, 480, 640, p)
    est.set_config(*cfg, stages=3)
    n, m = est(d)
    b = nrm.BatchedEstimator(p)
    for stages in (2, 3, 4):
        b.set_config(*cfg, stages=stages)
        (nb, mb), = b([(d, K)])
        assert torch.equal(nb, base_n) and torch.equal(mb, base_m), (cfg, stages)
    est.sync_status()
    b.sync_status()
    assert torch.equal(n, base_n) and torch.equal(m, base_m)


def test_batched_equals_plain_bitwise():
    frames = [scenes.random_frame(500 + i, W, H, DEV, kind=k)
              for i, (W, H, k) in enumerate([(320, 240, "f32"), (641, 479, "u16"), (200, 900, "f32"),
                                             (1280, 720, "u16"), (64, 64, "f32"), (127, 33, "u16")])]
    for out in ("f32", "f16"):
        p = nrm.NormalParams(out_dtype=out)
        b = nrm.BatchedEstimator(p)
        outs = b(frames)
        b.sync_status()
        for (d, K), (nb, mb) in zip(frames, outs):
            n, m = plain(d, K, p)
            assert torch.equal(nb, n) and torch.equal(mb, m)


def test_unaligned_pitches_use_plain_loads_and_byte_stores():
    """Depth rows whose pitch is not a multiple of 16 bytes cannot be TMA-mapped;
    masks whose pitch is not a multiple of 4 need byte stores. Results must not
    change."""
    H, W = 123, 301
    d0, K = scenes.random_frame(9, W, H, DEV, kind="f32")
    wide = torch.zeros((H, W + 2), device=DEV)
    wide[:, 1:W + 1] = d0                       # pitch W + 2 = 303, base offset 4 bytes
    view = wide[:, 1:W + 1]
    n_wide = torch.full((H, W + 1, 4), 7.0, device=DEV)
    m_wide = torch.full((H, W + 1), 9, dtype=torch.uint8, device=DEV)
    p = nrm.NormalParams()
    b = nrm.BatchedEstimator(p)
    b([(view, K)], outputs=[(n_wide[:, :W], m_wide[:, :W])])
    b.sync_status()
    ref = run_oracle(d0, K, p)
    compare(n_wide[:, :W], m_wide[:, :W], ref, p.tau, what="unaligned")
    # Padding columns are untouched.
    assert (n_wide[:, W] == 7.0).all() and (m_wide[:, W] == 9).all()
    n, m = plain(d0.contiguous(), K, p)
    assert torch.equal(n_wide[:, :W], n) and torch.equal(m_wide[:, :W], m)


@pytest.mark.parametrize("out", ["f16", "oct16"])
@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_vector_and_scalar_tile_loops_give_the_same_bits(out, alpha):
    """half4 and octahedral outputs of full tiles take the vector tile loop
    (alpha 1 or 2, aligned outputs); an odd row pitch (mask stores not
    aligned) sends the same frames through the scalar loop, and alpha 3 takes
    it everywhere. Every compiled tile shape, uint16 and float32 input: both
    loops give the same bits."""
    items = [scenes.random_frame(930 + i, W, H, DEV, kind=kind)
             for i, (W, H, kind) in enumerate([(640, 480, "u16"), (517, 300, "f32"), (1920, 1080, "u16")])]
    C = 2 if out == "oct16" else 4
    dt = torch.int16 if out == "oct16" else torch.float16
    b = nrm.BatchedEstimator(nrm.NormalParams(alpha=alpha, out_dtype=out))
    for cfg in [(128, 16, 256), (64, 64, 256), (128, 64, 512), (64, 16, 128)]:
        b.set_config(*cfg, stages=3)
        vec = b(items)
        outs = []
        for d, _ in items:
            H, W = d.shape
            nb = torch.zeros((H, W + 1, C), dtype=dt, device=DEV)
            vb = torch.zeros((H, W + 1), dtype=torch.uint8, device=DEV)
            outs.append((nb[:, :W], vb[:, :W]))
        sca = b(items, outputs=outs)
        b.sync_status()
        for (n1, m1), (n2, m2) in zip(vec, sca):
            assert torch.equal(m1, m2), (out, alpha, cfg)
            assert torch.equal(n1, n2), (out, alpha, cfg)


@pytest.mark.parametrize("out", ["f32", "f16"])
def test_mixed_size_batch_parity(out):
    """A batch drawn from the uneven size mix (with a 4096 x 3072 frame), float32
    and uint16 frames mixed, in one persistent launch."""
    sizes = [(320, 240), (640, 480), (1280, 720), (1920, 1080), (4096, 3072), (320, 240), (640, 480)]
    frames = [scenes.random_frame(3000 + i, W, H, DEV, kind=("f32" if i % 2 == 0 else "u16"))
              for i, (W, H) in enumerate(sizes)]
    p = nrm.NormalParams(out_dtype=out)
    b = nrm.BatchedEstimator(p)
    outs = b(frames)
    b.sync_status()
    total_near = 0
    for i, ((d, K), (n, m)) in enumerate(zip(frames, outs)):
        near, _, _ = compare(n, m, run_oracle(d, K, p), p.tau, half=(out == "f16"), what=f"mixed #{i}")
        total_near += near
    print(f"mixed batch {out}: near-tau excluded {total_near}")


def test_repeated_batched_calls_reuse_slots():
    """More calls than descriptor slots, alternating batch shapes, stay exact."""
    p = nrm.NormalParams()
    b = nrm.BatchedEstimator(p)
    a = [scenes.random_frame(40 + i, 320, 240, DEV, kind="f32") for i in range(3)]
    c = [scenes.random_frame(60 + i, 640, 480, DEV, kind="u16") for i in range(2)]
    ref_a = b(a)
    ref_c = b(c)
    for it in range(8):
        out = b(a if it % 2 == 0 else c)
        ref = ref_a if it % 2 == 0 else ref_c
        for (n, m), (rn, rm) in zip(out, ref):
            assert torch.equal(n, rn) and torch.equal(m, rm)
    b.sync_status()


def test_timing_stats_count_launches():
    b = nrm.BatchedEstimator()
    frames = [scenes.random_frame(7, 640, 480, DEV, kind="f32")]
    b.enable_timing(True)
    b.reset_stats()
    for _ in range(5):
        b(frames)
    s = b.stats()
    assert s["launches"] == 5
    assert s["kernel_ms"] > 0
    assert s["tiles"] == 5 * 5 * 30


def test_autotune_picks_a_config_and_caches_it(tmp_path):
    frames = [scenes.random_frame(8 + i, 640, 480, DEV, kind="f32") for i in range(4)]
    cache = str(tmp_path / "tune.json")
    b = nrm.BatchedEstimator()
    cfg = b.autotune(frames, cache_path=cache)
    assert (cfg["tile_x"], cfg["tile_y"], cfg["threads"]) in CONFIGS
    text = open(cache).read()
    assert str(cfg["tile_y"]) in text
    b2 = nrm.BatchedEstimator()
    assert b2.autotune(frames, cache_path=cache) == cfg
    outs = b2(frames)
    for (d, K), (n, m) in zip(frames, outs):
        compare(n, m, run_oracle(d, K, nrm.NormalParams()), 12.0, what="tuned")


@pytest.mark.parametrize("alpha", [1, 2])
@pytest.mark.parametrize("orient", [False, True])
def test_oct16_output_parity(cfg1, alpha, orient):
    """2 x int16 octahedral normals (4 B/px) against the oracle, plain and
    batched, float32 and uint16 input."""
    d, K = cfg1
    p = nrm.NormalParams(alpha=alpha, out_dtype="oct16", orient_to_camera=orient)
    n, m = plain(d, K, p)
    assert n.dtype == torch.int16 and tuple(n.shape) == (480, 640, 2)
    near, ang, nv = compare_oct16(n, m, run_oracle(d, K, p), p.tau, what=f"oct16 a{alpha}")
    assert nv > 0.5 * d.numel()
    print(f"oct16 alpha={alpha} orient={orient}: max angle {ang:.2e} rad")
    frames = [scenes.random_frame(600 + i, W, H, DEV, kind=k)
              for i, (W, H, k) in enumerate([(1920, 1080, "u16"), (333, 197, "f32"), (640, 480, "u16")])]
    b = nrm.BatchedEstimator(p)
    outs = b(frames)
    b.sync_status()
    for i, ((fd, fK), (fn, fm)) in enumerate(zip(frames, outs)):
        compare_oct16(fn, fm, run_oracle(fd, fK, p), p.tau, what=f"oct16 batched #{i}")
        pn, pm = plain(fd, fK, p)
        assert torch.equal(pn, fn) and torch.equal(pm, fm)


def test_oct16_decoder_round_trip_against_float_output(cfg1):
    """The library's torch decoder and the float32 output agree within the
    quantisation bound."""
    d, K = cfg1
    n32, m = plain(d, K, nrm.NormalParams())
    n16, m16 = plain(d, K, nrm.NormalParams(out_dtype="oct16"))
    assert torch.equal(m, m16)
    v = m.bool()
    dec = nrm.decode_oct16(n16)[v].double()
    ref = n32[..., :3][v].double()
    ang = torch.atan2(torch.linalg.cross(dec, ref).norm(dim=-1), (dec * ref).sum(-1))
    assert float(ang.max()) <= 1e-4
