"""Parity at full size in the benchmark's launch configuration: the batch of
64 full-HD uint16 frames through one persistent launch (graph replay), every
frame compared with the oracle (masks bit-exact outside the near-tau band,
normals within 1e-4 rad), and the uneven batch of 256 float32 frames with
float4 and half4 output."""
import os

import pytest
import torch

import oracle
import paper_2209_08241_gb300 as nrm
from parity import compare
from synth import scenes

pytestmark = pytest.mark.gpu
NT = max(1, min(16, os.cpu_count() or 1))


@pytest.mark.parametrize("config", ["default", "autotuned", (128, 16, 128, 2, 3)])
def test_u16_full_hd_batch_of_64(config):
    """The default launch geometry, the one the autotuner picks for this batch
    (as bench.py does before timing), and the geometry it has been picking."""
    frames = scenes.u16_batch(64, 1920, 1080, device="cuda")
    p = nrm.NormalParams()
    b = nrm.BatchedEstimator(p)
    if config == "autotuned":
        b.autotune(frames)
    elif config != "default":
        b.set_config(*config)
    outs = b(frames)
    outs = b(frames, outputs=outs)  # second replay of the same graph slot ring
    b.sync_status()
    near_total = 0
    for i, ((d, K), (n, m)) in enumerate(zip(frames, outs)):
        ref = oracle.forward(d.cpu().numpy(), K, alpha=p.alpha, stat_mode=oracle.STAT_SECANT, tau=p.tau,
                             depth_scale=p.depth_scale, nthreads=NT)
        near, _, _ = compare(n, m, ref, p.tau, what=f"frame {i}")
        near_total += near
    print(f"64 x 1080p u16 {config} {b.config()}: near-tau pixels excluded {near_total}")


@pytest.mark.parametrize("out,every", [("f32", 1), ("f16", 4)])
def test_f32_mixed_batch_of_256(out, every):
    """The uneven batch at full size (256 float32 frames from the size mix,
    262 Mpx) in the launch geometry the autotuner picks for it, as bench.py
    times it; float4 output compared frame by frame with the oracle, half4
    output on every fourth frame."""
    frames = scenes.mixed_batch(256, device="cuda", kind="f32")
    p = nrm.NormalParams(out_dtype=out)
    b = nrm.BatchedEstimator(p)
    outs = [(torch.empty((*d.shape, 4), dtype=p.torch_out_dtype, device="cuda"),
             torch.empty(d.shape, dtype=torch.uint8, device="cuda")) for d, _ in frames]
    b.autotune(frames, outs)
    b(frames, outputs=outs)
    b.sync_status()
    near_total = 0
    for i in range(0, len(frames), every):
        (d, K), (n, m) = frames[i], outs[i]
        ref = oracle.forward(d.cpu().numpy(), K, alpha=p.alpha, stat_mode=oracle.STAT_SECANT, tau=p.tau,
                             nthreads=NT)
        near, _, _ = compare(n, m, ref, p.tau, half=(out == "f16"), what=f"frame {i} {tuple(d.shape)}")
        near_total += near
    print(f"256 mixed f32 -> {out} {b.config()}: near-tau pixels excluded {near_total}")
