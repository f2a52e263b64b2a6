"""FP64 oracle of the organised point cloud: the back-projection of every pixel
(Section 2, definitions below Eq. 3; Section 3.1 writes the points as
P = (u d, v d, d)).

TEST INFRASTRUCTURE (same rules as the rest of ``oracle/``).

For pixel (col, row) with valid depth d (float: positive and finite; uint16:
nonzero, times depth_scale): P = d (u, v, 1), u = (col - cx)/fx,
v = (row - cy)/fy. Reading: a pixel with invalid depth gets the point
(0, 0, 0), independent of the normal mask (a point exists wherever the depth
does).
"""
from __future__ import annotations

import numpy as np


def points(depth, K, depth_scale: float = 0.001) -> np.ndarray:
    """(H, W, 3) float64 points in metres; zero where the depth is invalid."""
    d = np.asarray(depth)
    if d.dtype == np.uint16:
        z = d.astype(np.float64) * depth_scale
        ok = d != 0
    else:
        z = d.astype(np.float64)
        ok = np.isfinite(z) & (z > 0)
    H, W = z.shape
    fx, fy, cx, cy = (float(k) for k in K)
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    P = np.stack([z * u[None, :], z * v[:, None], z], -1)
    return np.where(ok[..., None], P, 0.0)
