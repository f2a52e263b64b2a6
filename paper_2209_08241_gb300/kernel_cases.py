"""Run one kernel on synthetic input, for timing and profiling.

    python -m paper_2209_08241_gb300.kernel_cases CASE [--reps N] [--frames N]

Cases:
  forward        batched forward on N full-HD uint16 frames (default 8), normals
                 stored as --out (f32, f16 or oct16)
  adjoint        single-frame adjoint on a 4096 x 3072 float32 frame
  adjoint_batch  batched adjoint on N 640 x 480 float32 frames (default 32)
  plane_fit      plane-fitting ground truth, radius --radius (default 2), on a
                 4096 x 3072 float32 frame
  multiscale     multi-scale variant, scales 1..4, stencil --form (pair or
                 quad), on a 4096 x 3072 float32 frame
  multiscale_batch  the same, batched, on N full-HD uint16 frames (default 8)
  spherical      I_phi / I_theta images of a 4096 x 3072 normal map
  angle_mse      angle-image MSE of two 4096 x 3072 normal maps

Each case runs the kernel ``--reps`` times after one untimed call and prints the
mean time per call (CUDA events) and the algorithmic bandwidth.
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2209_08241_gb300 as nrm  # noqa: E402
from synth import scenes  # noqa: E402


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


OUT_BYTES = {"f32": 16, "f16": 8, "oct16": 4}


def case_forward(frames: int, reps: int, out: str = "f32"):
    items = [scenes.random_frame(1000 + i, 1920, 1080, "cuda", kind="u16") for i in range(frames)]
    b = nrm.BatchedEstimator(nrm.NormalParams(out_dtype=out))
    outs = b(items)
    ms = _time(lambda: b(items, outs), reps)
    px = frames * 1920 * 1080
    return ms, px, px * (2 + OUT_BYTES[out] + 1)


def case_adjoint(reps: int):
    d, K = scenes.random_frame(4999, 4096, 3072, "cuda", kind="f32", holes=False, clip_range=False)
    est = nrm.NormalEstimator(K, 3072, 4096)
    n, m = est(d)
    g = torch.zeros_like(n)
    g[..., 2] = m.float()
    grad = torch.empty_like(d)
    ms = _time(lambda: est.backward(d, g, m, grad), reps)
    px = 4096 * 3072
    return ms, px, px * 25


def case_adjoint_batch(frames: int, reps: int):
    items = [scenes.random_frame(4000 + i, 640, 480, "cuda", kind="f32", holes=False, clip_range=False)
             for i in range(frames)]
    b = nrm.BatchedEstimator()
    outs = b(items)
    gs = []
    for n, m in outs:
        g = torch.zeros_like(n)
        g[..., 2] = m.float()
        gs.append(g)
    grads = [torch.empty_like(d) for d, _ in items]
    arr, _ = b.make_grad_frames(items, gs, [m for _, m in outs], grads)
    ms = _time(lambda: b.run_backward(arr, frames), reps)
    px = frames * 640 * 480
    return ms, px, px * 25


def case_plane_fit(radius: int, reps: int):
    d, K = scenes.random_frame(4999, 4096, 3072, "cuda", kind="f32", holes=False, clip_range=False)
    est = nrm.NormalEstimator(K, 3072, 4096)
    n, m = est.plane_fit(d, radius)
    ms = _time(lambda: est.plane_fit(d, radius, n, m), reps)
    px = 4096 * 3072
    return ms, px, px * 21


def case_spherical(reps: int):
    d, K = scenes.random_frame(4999, 4096, 3072, "cuda", kind="f32", holes=False, clip_range=False)
    n, m = nrm.NormalEstimator(K, 3072, 4096)(d)
    ms = _time(lambda: nrm.spherical_images(n, m), reps)
    px = 4096 * 3072
    return ms, px, px * 25


def case_angle_mse(reps: int):
    d, K = scenes.random_frame(4999, 4096, 3072, "cuda", kind="f32", holes=False, clip_range=False)
    est = nrm.NormalEstimator(K, 3072, 4096)
    n, m = est(d)
    rn, rm = est(torch.roll(d, 1, dims=0).contiguous())
    ms = _time(lambda: nrm.angle_mse(est, n, m, rn, rm), reps)
    px = 4096 * 3072
    return ms, px, px * 34


def case_multiscale(form: str, reps: int):
    d, K = scenes.random_frame(4999, 4096, 3072, "cuda", kind="f32", holes=False, clip_range=False)
    est = nrm.NormalEstimator(K, 3072, 4096)
    n, m = est.estimate_multiscale(d, (1, 2, 3, 4), form)
    ms = _time(lambda: est.estimate_multiscale(d, (1, 2, 3, 4), form, n, m), reps)
    px = 4096 * 3072
    return ms, px, px * 21


def case_multiscale_batch(form: str, frames: int, reps: int):
    items = [scenes.random_frame(1000 + i, 1920, 1080, "cuda", kind="u16") for i in range(frames)]
    b = nrm.BatchedEstimator()
    outs = b.multiscale(items, (1, 2, 3, 4), form)
    arr, _ = b.make_frames(items, outs)
    ms = _time(lambda: b.run_multiscale(arr, frames, (1, 2, 3, 4), form), reps)
    px = frames * 1920 * 1080
    return ms, px, px * 19


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["forward", "adjoint", "adjoint_batch", "plane_fit", "multiscale",
                                     "multiscale_batch", "spherical", "angle_mse"])
    ap.add_argument("--radius", type=int, default=2)
    ap.add_argument("--form", choices=["pair", "quad"], default="pair")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--frames", type=int, default=0)
    ap.add_argument("--out", choices=sorted(OUT_BYTES), default="f32")
    a = ap.parse_args(argv)
    if a.case == "forward":
        ms, px, nbytes = case_forward(a.frames or 8, a.reps, a.out)
    elif a.case == "adjoint":
        ms, px, nbytes = case_adjoint(a.reps)
    elif a.case == "plane_fit":
        ms, px, nbytes = case_plane_fit(a.radius, a.reps)
    elif a.case == "multiscale":
        ms, px, nbytes = case_multiscale(a.form, a.reps)
    elif a.case == "spherical":
        ms, px, nbytes = case_spherical(a.reps)
    elif a.case == "angle_mse":
        ms, px, nbytes = case_angle_mse(a.reps)
    elif a.case == "multiscale_batch":
        ms, px, nbytes = case_multiscale_batch(a.form, a.frames or 8, a.reps)
    else:
        ms, px, nbytes = case_adjoint_batch(a.frames or 32, a.reps)
    print(f"{a.case}: {ms:.4f} ms/call, {px / ms / 1e3:.1f} Mpx/s, {nbytes / ms / 1e6:.1f} GB/s algorithmic")


if __name__ == "__main__":
    main()
