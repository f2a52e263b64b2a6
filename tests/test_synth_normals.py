"""The analytic ground-truth normals of the synthetic scenes (scene geometry,
used to score estimates as in Section 4): the same nearest hits as the depth
caster, unit length, oriented away from the camera, radial on spheres, the
plane's normal on planes, and in agreement with the oracle's estimates on
noise-free surfaces away from depth steps."""
import math

import numpy as np
import torch

import oracle
from synth import scenes


def angle(a, b):
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1))


def rays(H, W, K):
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    return np.stack([uu, vv, np.ones_like(uu)], -1)


def test_cfg1_normals_match_the_caster_and_the_primitives():
    K = scenes.CFG1_K
    d0 = scenes.cast(scenes.cfg1_scene(), 640, 480, K, "cpu")
    d1, n = scenes.cast_normals(scenes.cfg1_scene(), 640, 480, K, "cpu")
    assert torch.equal(d0, d1)
    n = n.numpy()
    hit = np.isfinite(d1.numpy())
    assert np.allclose(np.linalg.norm(n[hit], axis=-1), 1.0, atol=1e-12)
    assert (n[~hit] == 0).all()
    assert ((n[hit] * rays(480, 640, K)[hit]).sum(-1) > 0).all()
    # Background plane (top-left corner) and the sphere's centre pixel.
    n_bg = scenes.cfg1_scene().prims[0].normal
    assert angle(n[5, 5], n_bg) < 1e-12
    C = np.array([-0.35, 0.0, 1.8])
    col = int(round(C[0] / C[2] * K[0] + K[2]))
    row = int(round(C[1] / C[2] * K[1] + K[3]))
    P = d1.numpy()[row, col] * rays(480, 640, K)[row, col]
    assert angle(n[row, col], (C - P) / 0.4) < 1e-12


def test_method_agrees_with_analytic_normals_on_noise_free_surfaces():
    d, K = scenes.cfg1_depth("cpu", noise=False)
    gt = scenes.cfg1_normals("cpu").numpy()
    ref = oracle.forward(d.numpy(), K, alpha=1)
    v = ref.valid == 1
    a = angle(ref.n_hat[v], gt[v])
    assert np.median(a) < 1e-3
    assert np.quantile(a, 0.95) < 2e-2


def test_box_and_cylinder_normals_agree_with_estimates():
    for seed in (3, 8):
        K = scenes.intrinsics_for(320, 240)
        scene = scenes.random_scene(np.random.default_rng(seed), 320, 240, K)
        d, n = scenes.cast_normals(scene, 320, 240, K, "cpu")
        D = torch.where(torch.isfinite(d), d, torch.zeros_like(d)).numpy()
        ref = oracle.forward(D, K, alpha=1)
        v = ref.valid == 1
        a = angle(ref.n_hat[v], n.numpy()[v])
        assert np.median(a) < 1e-2, seed
        kinds = {type(p).__name__ for p in scene.prims}
        assert {"Box", "Cylinder"} <= kinds
