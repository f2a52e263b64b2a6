"""Pins of the evaluation oracle (Section 4: I_phi / I_theta images and their
MSE) against closed forms: the six axis directions and the diagonals give
known angles, a rotation about the optical axis shifts phi by a known amount
and leaves theta alone, and identical maps have zero error."""
import math

import numpy as np
import pytest

from oracle import evaluation


@pytest.mark.parametrize("n,phi,theta", [
    ((0, 0, 1), 0.0, 0.0),
    ((1, 0, 0), 0.0, math.pi / 2),
    ((0, 1, 0), math.pi / 2, math.pi / 2),
    ((-1, 0, 0), math.pi, math.pi / 2),
    ((0, -1, 0), 1.5 * math.pi, math.pi / 2),
    ((0, 0, -1), 0.0, math.pi),
    ((1, 1, math.sqrt(2)), math.pi / 4, math.pi / 4),
    ((-1, -1, -math.sqrt(2)), 1.25 * math.pi, 0.75 * math.pi),
])
def test_axis_and_diagonal_directions(n, phi, theta):
    v = np.array(n, np.float64)
    v /= np.linalg.norm(v)
    p, t = evaluation.spherical(v.reshape(1, 1, 3), np.ones((1, 1), bool))
    assert p[0, 0] == pytest.approx(phi, abs=1e-15)
    assert t[0, 0] == pytest.approx(theta, abs=1e-15)
    assert 0.0 <= p[0, 0] < 2 * math.pi


def test_masked_pixels_are_zero():
    n = np.tile(np.array([0.3, -0.4, 0.866]), (2, 3, 1))
    v = np.array([[1, 0, 1], [0, 1, 0]], np.uint8)
    p, t = evaluation.spherical(n, v)
    assert (p[v == 0] == 0).all() and (t[v == 0] == 0).all()
    assert (t[v == 1] > 0).all()


def test_rotation_about_the_optical_axis_shifts_phi_only():
    rng = np.random.default_rng(0)
    H, W = 16, 20
    phi0 = rng.uniform(0.2, 2 * math.pi - 0.6, size=(H, W))
    th0 = rng.uniform(0.1, 1.4, size=(H, W))
    n = np.stack([np.sin(th0) * np.cos(phi0), np.sin(th0) * np.sin(phi0), np.cos(th0)], -1)
    d = 0.3
    c, s = math.cos(d), math.sin(d)
    m = n.copy()
    m[..., 0] = c * n[..., 0] - s * n[..., 1]
    m[..., 1] = s * n[..., 0] + c * n[..., 1]
    ones = np.ones((H, W), bool)
    mt, mp, cnt = evaluation.angle_mse(m, ones, n, ones)
    assert cnt == H * W
    assert mt == pytest.approx(0.0, abs=1e-24)
    assert mp == pytest.approx(d * d, rel=1e-12)


def test_identical_maps_and_disjoint_masks():
    rng = np.random.default_rng(1)
    n = rng.normal(size=(8, 8, 3))
    v = rng.integers(0, 2, size=(8, 8))
    assert evaluation.angle_mse(n, v, n, v)[:2] == (0.0, 0.0)
    assert evaluation.angle_mse(n, v, n, 1 - v) == (0.0, 0.0, 0)
