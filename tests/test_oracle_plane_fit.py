"""Pins of the plane-fitting oracle (the paper's ground-truth method): points of
a plane give its normal exactly with a zero smallest eigenvalue; the fitted
normal of a sphere converges to the radial direction as the window shrinks;
validity is brute force over the window; orientation and depth-scale
invariance; agreement with the method's own normals on smooth surfaces."""
import math

import numpy as np
import pytest

import oracle
from oracle.plane_fit import plane_fit
from synth import scenes


def rays(H, W, K):
    fx, fy, cx, cy = K
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    uu, vv = np.meshgrid(u, v)
    return np.stack([uu, vv, np.ones_like(uu)], -1)


def angle(a, b):
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1))


@pytest.mark.parametrize("radius", [1, 2, 3])
@pytest.mark.parametrize("tilt", [0.0, 0.4, 1.1])
def test_plane_is_exact(radius, tilt):
    H, W, K = 20, 24, (300.0, 310.0, 11.5, 9.5)
    n0 = np.array([math.sin(tilt) * 0.6, math.sin(tilt) * 0.8, math.cos(tilt)])
    D = 1.7 / (rays(H, W, K) @ n0)
    n, v, ev = plane_fit(D, K, radius)
    inner = np.zeros((H, W), bool)
    inner[radius:H - radius, radius:W - radius] = True
    assert (v.astype(bool) == inner).all()
    assert angle(n[inner], np.broadcast_to(n0, n[inner].shape)).max() < 1e-10
    assert (np.abs(ev[inner][:, 0]) <= 1e-12 * ev[inner][:, 2]).all()   # points are coplanar
    assert ((n[inner] * (rays(H, W, K)[inner])).sum(-1) > 0).all()      # away from the camera


def test_sphere_fit_converges_to_radial_normal():
    H, W = 241, 321
    C = np.array([0.15, -0.05, 2.0])
    R = 0.5
    prim = scenes.Sphere(C, R)
    errs = []
    for f in (500.0, 1000.0, 2000.0):
        K = (f, f, 160.0, 120.0)
        D = scenes.cast(scenes.Scene([prim]), W, H, K, "cpu").numpy()
        D = np.where(np.isfinite(D), D, 0.0)
        n, v, _ = plane_fit(D, K, 2)
        y, x = 110, 175
        assert v[y, x]
        P = D[y, x] * rays(H, W, K)[y, x]
        true = -(P - C) / R
        errs.append(float(angle(n[y, x], true)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


def test_validity_is_brute_force_over_the_window():
    rng = np.random.default_rng(0)
    H, W = 15, 17
    D = rng.uniform(1.0, 1.3, size=(H, W))
    for (y, x) in [(3, 4), (10, 12), (7, 0)]:
        D[y, x] = 0.0
    D[12, 2] = np.nan
    K = (100.0, 100.0, 8.0, 7.0)
    n, v, _ = plane_fit(D, K, 2)
    ok = np.isfinite(D) & (D > 0)
    for y in range(H):
        for x in range(W):
            exp = 2 <= y < H - 2 and 2 <= x < W - 2 and ok[y - 2:y + 3, x - 2:x + 3].all()
            assert bool(v[y, x]) == exp
    assert (n[v == 0] == 0).all()


def test_depth_scale_invariance_and_uint16():
    d, K = scenes.random_frame(31, 64, 48, kind="f64", holes=False, clip_range=False)
    D = d.numpy()
    n1, v1, _ = plane_fit(D, K, 2)
    n2, v2, _ = plane_fit(3.0 * D, K, 2)
    assert (v1 == v2).all()
    np.testing.assert_allclose(n1, n2, atol=1e-9)
    raw = np.clip(np.round(D * 1000), 1, 65535).astype(np.uint16)
    n3, v3, _ = plane_fit(raw, K, 2, depth_scale=0.001)
    n4, v4, _ = plane_fit(raw.astype(np.float64) * 0.001, K, 2)
    np.testing.assert_array_equal(v3, v4)
    np.testing.assert_allclose(n3, n4, atol=1e-12)


def test_agrees_with_the_method_on_a_smooth_scene():
    d, K = scenes.cfg1_depth("cpu", noise=False)
    D = d.numpy().astype(np.float64)
    pn, pv, _ = plane_fit(D, K, 2)
    ref = oracle.forward(D, K, alpha=2, tau=1e300)
    both = (pv == 1) & (ref.valid == 1)
    ang = angle(pn[both], ref.n_hat[both])
    # Away from the depth steps the two estimates agree closely.
    assert np.median(ang) < 1e-3


def test_banded_oracle_equals_one_call():
    from parity import plane_fit_banded
    d, K = scenes.random_frame(7, 40, 90, kind="f32", noise=True, holes=True)
    D = d.numpy()
    for R in (1, 3):
        n1, v1, e1 = plane_fit(D, K, R)
        n2, v2, e2 = plane_fit_banded(D, K, R, band=16)
        np.testing.assert_array_equal(v1, v2)
        np.testing.assert_allclose(n2, n1, atol=1e-12)
        np.testing.assert_allclose(e2, e1, atol=1e-15, rtol=1e-9)
