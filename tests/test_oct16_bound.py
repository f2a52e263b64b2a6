"""The octahedral tolerance (tests/parity.py, ANG_TOL_OCT16) holds for the
16-bit octahedral code by brute force: unit directions (random, on the fold
diagonals, at the poles and on the equator) encoded exactly in FP64 from the
published definition (project onto |x| + |y| + |z| = 1, fold the lower half,
round 32767 p to the nearest integer) and decoded with the tests' decoder
come back within ANG_TOL_OCT16, and the worst case found stays within the
analytic bound sqrt(6)/32767. The half-output tolerance is pinned the same
way against float16 rounding. CPU only."""
import math

import numpy as np

from parity import ANG_TOL_OCT16, decode_oct16


def _encode(v):
    v = np.asarray(v, np.float64)
    p = v[..., :2] / np.abs(v).sum(-1, keepdims=True)
    lower = v[..., 2] < 0
    fx = np.where(lower, (1.0 - np.abs(p[..., 1])) * np.where(p[..., 0] >= 0, 1.0, -1.0), p[..., 0])
    fy = np.where(lower, (1.0 - np.abs(p[..., 0])) * np.where(p[..., 1] >= 0, 1.0, -1.0), p[..., 1])
    return np.rint(np.stack([fx, fy], -1) * 32767.0).astype(np.int16)


def _angles(a, b):
    c = np.clip((a * b).sum(-1), -1.0, 1.0)
    s = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(s, c)


def test_round_trip_within_the_tolerance():
    rng = np.random.default_rng(11)
    v = rng.normal(size=(400000, 3))
    t = np.linspace(0.0, 2 * math.pi, 2001)
    diag = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], -1)            # equator
    fold = np.stack([np.cos(t), np.sin(t), -np.abs(np.cos(2 * t))], -1)      # lower half near the folds
    axes = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                     [1, 1, -1e-9], [-1, 1, -1e-9], [1, -1, 1e-9]], np.float64)
    v = np.concatenate([v, diag, fold, axes])
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    ang = _angles(decode_oct16(_encode(v)), v)
    assert ang.max() <= ANG_TOL_OCT16
    assert ang.max() <= math.sqrt(6) / 32767
    assert ang.max() > 1e-6  # the quantisation is really exercised


def test_half_output_rounding_within_its_tolerance():
    """The half4 tolerance (5e-3 rad): a unit normal rounded to float16 per
    component turns by at most ~sqrt(3) 2^-11 (about 8.5e-4 rad)."""
    from parity import ANG_TOL_F16
    rng = np.random.default_rng(12)
    v = rng.normal(size=(400000, 3))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    h = v.astype(np.float16).astype(np.float64)
    ang = _angles(h / np.linalg.norm(h, axis=-1, keepdims=True), v)
    assert ang.max() <= math.sqrt(3) * 2.0 ** -11 <= ANG_TOL_F16
