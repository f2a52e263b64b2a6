"""FP64 oracle of the paper's evaluation quantities (arXiv 2209.08241, Section 4).

TEST INFRASTRUCTURE (same rules as the rest of ``oracle/``): only the tests,
the smoke check and the benchmark's CPU legs use it; it shares nothing with
the CUDA path.

* Spherical images (Section 4, the I_phi and I_theta equations): the paper
  writes I_phi = atan(n_y / n_x) and I_theta = atan(sqrt(n_x^2 + n_y^2) / n_z)
  and states that all images are normalised to the range [0, 2 pi]. Reading:
  the quadrant-aware forms, phi = atan2(n_y, n_x) taken into [0, 2 pi) and
  theta = atan2(sqrt(n_x^2 + n_y^2), n_z) in [0, pi]. Masked pixels get 0.
* Mean squared error (Section 4, Tables 2-5): the mean over pixels valid in
  both maps of the squared difference of the angle images, taken as plain
  differences of the [0, 2 pi) values (the paper does not mention wrap-around).
"""
from __future__ import annotations

import numpy as np


def spherical(n: np.ndarray, valid: np.ndarray):
    """(phi, theta) images of normals n (H, W, >=3) where valid, else 0."""
    n = np.asarray(n, np.float64)[..., :3]
    v = np.asarray(valid).astype(bool)
    phi = np.arctan2(n[..., 1], n[..., 0])
    phi = np.where(phi < 0.0, phi + 2.0 * np.pi, phi)
    theta = np.arctan2(np.sqrt(n[..., 0] ** 2 + n[..., 1] ** 2), n[..., 2])
    return np.where(v, phi, 0.0), np.where(v, theta, 0.0)


def angle_mse(n_a, valid_a, n_b, valid_b):
    """(mse_theta, mse_phi, count) over pixels valid in both maps."""
    both = np.asarray(valid_a).astype(bool) & np.asarray(valid_b).astype(bool)
    pa, ta = spherical(n_a, both)
    pb, tb = spherical(n_b, both)
    count = int(both.sum())
    if count == 0:
        return 0.0, 0.0, 0
    return (float(((ta - tb)[both] ** 2).sum() / count), float(((pa - pb)[both] ** 2).sum() / count), count)
