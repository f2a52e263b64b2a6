"""Pins of the multi-scale oracle (Section 2's previous method and its scale
averages; Section 3.1's four-direction form averaged the same way).

The pair form is checked against the paper's printed closed form (Eq. 1-3),
an identity it implies (n . ray = alpha^2 d2 d3 / (fx fy)), exact planes, its
first-order convergence on a sphere, brute-force validity and the noise
reduction that motivates averaging over scales; the quad form against the
single-scale oracle and the same plane and noise properties."""
import math

import numpy as np
import pytest

import oracle
from oracle import STAT_RAW, STAT_SECANT
from oracle.multiscale import multiscale
from synth import scenes


def rays(H, W, K):
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    return np.stack([uu, vv, np.ones_like(uu)], -1)


def angle(a, b):
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1))


def plane_depth(H, W, K, n0, D0):
    return D0 / (rays(H, W, K) @ n0)


@pytest.mark.parametrize("alpha", [1, 3])
def test_pair_form_equals_printed_closed_form(alpha):
    """Eq. 1-3 as printed (u pairs with the column, v with the row)."""
    rng = np.random.default_rng(alpha)
    H, W, K = 9, 11, (410.0, 380.0, 4.7, 3.9)
    D = rng.uniform(0.8, 2.5, size=(H, W))
    res = multiscale(D, K, [alpha], "pair", STAT_RAW, np.inf)
    fx, fy, cx, cy = K
    for row in range(H - alpha):
        for col in range(W - alpha):
            d1, d2, d3 = D[row, col], D[row, col + alpha], D[row + alpha, col]
            u1, v1 = (col - cx) / fx, (row - cy) / fy
            nx = -(alpha / fy) * d3 * (d2 - d1)
            ny = -(alpha / fx) * d2 * (d3 - d1)
            nz = (alpha / fx) * v1 * d2 * (d3 - d1) + (alpha / fy) * u1 * d3 * (d2 - d1) \
                + alpha ** 2 / (fx * fy) * d2 * d3
            np.testing.assert_allclose(res.n_raw[row, col], [nx, ny, nz], rtol=1e-12, atol=1e-15)
            # Implied by Eq. 1-3: the normal's component along the viewing ray.
            ray = np.array([u1, v1, 1.0])
            assert res.n_raw[row, col] @ ray == pytest.approx(alpha ** 2 * d2 * d3 / (fx * fy), rel=1e-11)


def test_quad_form_single_scale_equals_single_scale_oracle():
    d, K = scenes.random_frame(21, 96, 64, kind="f32")
    D = d.numpy()
    for a in (1, 2, 4):
        ms = multiscale(D, K, [a], "quad", STAT_SECANT, 12.0)
        ref = oracle.forward(D, K, alpha=a, stat_mode=STAT_SECANT, tau=12.0)
        np.testing.assert_array_equal(ms.valid, ref.valid)
        np.testing.assert_allclose(ms.n_raw, np.where(np.isfinite(ref.r)[..., None], ref.n_raw, 0),
                                   rtol=0, atol=0)
        np.testing.assert_allclose(ms.n_hat, ref.n_hat, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("form", ["pair", "quad"])
@pytest.mark.parametrize("tilt", [0.0, 0.5, 1.2])
def test_planes_are_exact_for_any_scale_set(form, tilt):
    H, W, K = 40, 52, (260.0, 255.0, 25.5, 19.5)
    n0 = np.array([math.sin(tilt) * 0.8, -math.sin(tilt) * 0.6, math.cos(tilt)])
    D = plane_depth(H, W, K, n0, 1.9)
    res = multiscale(D, K, [1, 2, 5], form, STAT_RAW, np.inf)
    v = res.valid == 1
    assert v.sum() > 0.5 * H * W
    assert angle(res.n_hat[v], np.broadcast_to(n0, res.n_hat[v].shape)).max() < 1e-10
    assert ((res.n_hat[v] * rays(H, W, K)[v]).sum(-1) > 0).all()   # away from the camera


def test_pair_form_is_first_order_on_a_sphere():
    """One-sided differences: doubling alpha doubles the leading error (the
    four-direction form's central differences are second order instead)."""
    H, W = 401, 401
    K = (900.0, 900.0, 200.0, 200.0)
    C, R = np.array([0.0, 0.0, 2.0]), 0.6
    D = scenes.cast(scenes.Scene([scenes.Sphere(C, R)]), W, H, K, "cpu").numpy()
    D = np.where(np.isfinite(D), D, 0.0)
    y, x = 150, 260
    P = D[y, x] * rays(H, W, K)[y, x]
    true = (C - P) / R   # away from the camera, like the estimates
    errs = {}
    for form in ("pair", "quad"):
        for a in (2, 4):
            res = multiscale(D, K, [a], form, STAT_RAW, np.inf)
            assert res.valid[y, x]
            errs[form, a] = float(angle(res.n_hat[y, x], true))
    assert 1.7 < errs["pair", 4] / errs["pair", 2] < 2.3
    assert 3.5 < errs["quad", 4] / errs["quad", 2] < 4.5
    assert errs["quad", 2] < errs["pair", 2]


@pytest.mark.parametrize("form", ["pair", "quad"])
def test_validity_is_brute_force_over_all_scales(form):
    rng = np.random.default_rng(5)
    H, W = 17, 23
    D = rng.uniform(1.0, 1.2, size=(H, W))
    for (y, x) in [(4, 6), (12, 2), (0, 20), (9, 9)]:
        D[y, x] = 0.0
    D[15, 15] = np.nan
    K = (120.0, 120.0, 11.0, 8.0)
    alphas = [1, 3]
    res = multiscale(D, K, alphas, form, STAT_RAW, np.inf)
    ok = np.isfinite(D) & (D > 0)
    offs = [(0, 1), (1, 0)] if form == "pair" else [(0, 1), (1, 0), (0, -1), (-1, 0)]
    for y in range(H):
        for x in range(W):
            exp = bool(ok[y, x])
            for a in alphas:
                for dy, dx in offs:
                    yy, xx = y + a * dy, x + a * dx
                    exp = exp and 0 <= yy < H and 0 <= xx < W and bool(ok[yy, xx])
            assert bool(res.valid[y, x]) == exp, (y, x)
    assert (res.n_hat[res.valid == 0] == 0).all()


@pytest.mark.parametrize("form", ["pair", "quad"])
def test_averaging_over_scales_reduces_noise(form):
    """The motivation of the multi-scale average (Section 2): on a noisy
    plane, averaging four scales lowers the angular error."""
    H, W, K = 120, 160, (200.0, 200.0, 79.5, 59.5)
    n0 = np.array([0.2, -0.3, 0.93])
    n0 /= np.linalg.norm(n0)
    D = plane_depth(H, W, K, n0, 2.0)
    D = D + np.random.default_rng(9).normal(0, 0.002, size=D.shape)
    one = multiscale(D, K, [1], form, STAT_RAW, np.inf)
    four = multiscale(D, K, [1, 2, 3, 4], form, STAT_RAW, np.inf)
    v = (one.valid == 1) & (four.valid == 1)
    e1 = np.mean(angle(one.n_hat[v], np.broadcast_to(n0, one.n_hat[v].shape)))
    e4 = np.mean(angle(four.n_hat[v], np.broadcast_to(n0, four.n_hat[v].shape)))
    assert e4 < 0.5 * e1


def test_orientation_order_and_duplicates():
    d, K = scenes.random_frame(33, 80, 60, kind="u16")
    D = d.numpy()
    a = multiscale(D, K, [1, 3], "pair")
    b = multiscale(D, K, [3, 1], "pair")
    np.testing.assert_array_equal(a.valid, b.valid)
    np.testing.assert_allclose(a.n_hat, b.n_hat, rtol=0, atol=1e-15)
    c = multiscale(D, K, [2, 2], "quad")
    e = multiscale(D, K, [2], "quad")
    np.testing.assert_array_equal(c.valid, e.valid)
    np.testing.assert_array_equal(c.n_hat, e.n_hat)
    np.testing.assert_array_equal(c.n_raw, e.n_raw)      # the average divides by K
    np.testing.assert_array_equal(c.stat, e.stat)
    f = multiscale(D, K, [1, 3], "pair", orient=1)
    np.testing.assert_array_equal(f.valid, a.valid)
    np.testing.assert_array_equal(f.n_hat, -a.n_hat)
    np.testing.assert_array_equal(f.stat, a.stat)


def test_secant_statistic_is_the_inverse_cosine_on_planes():
    """On a plane the averaged n stays along the plane normal, so the SECANT
    statistic is 1 / cos(normal, ray) for any scale set (Section 3.2's
    statistic, in the depth-invariant form used here)."""
    H, W, K = 30, 40, (150.0, 150.0, 19.5, 14.5)
    n0 = np.array([0.5, 0.1, 0.86])
    n0 /= np.linalg.norm(n0)
    D = plane_depth(H, W, K, n0, 1.4)
    res = multiscale(D, K, [1, 2, 4], "pair", STAT_SECANT, 1e9)
    v = res.valid == 1
    ray = rays(H, W, K)[v]
    cosang = (ray @ n0) / np.linalg.norm(ray, axis=-1)
    np.testing.assert_allclose(res.stat[v], 1.0 / cosang, rtol=1e-9)
