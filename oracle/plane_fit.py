"""FP64 oracle of local plane fitting ("plane-PCA"), the ground truth the paper
uses for its real-data comparison (arXiv 2209.08241: Section 1 describes the
method; Section 4 uses it with 25 neighbouring points).

TEST INFRASTRUCTURE (same rules as the rest of ``oracle/``).

Definition, for each pixel (col, row) and window radius R (R = 2: 25 points):
  1. back-project every pixel of the (2R+1) x (2R+1) window centred on it,
     P = d (u, v, 1), u = (col - cx)/fx, v = (row - cy)/fy (Section 2);
  2. scatter matrix S = sum over the window of (P - c)(P - c)^T, c the centroid;
  3. normal = unit eigenvector of S for its smallest eigenvalue (Section 1:
     "the eigen vector correspond to the smallest eigen value"), computed here
     with numpy.linalg.eigh;
  4. orientation, a reading: like the method's normal, away from the camera
     (n . P_centre > 0);
  5. validity, a reading: every depth of the window lies inside the image and
     is positive and finite; otherwise the pixel is invalid with normal 0.
Also returned: the three eigenvalues (ascending), which bound how well the
normal is determined (the gap between the two smallest).
"""
from __future__ import annotations

import numpy as np


def plane_fit(depth: np.ndarray, K, radius: int = 2, depth_scale: float = 0.001):
    """(normals (H, W, 3), valid (H, W) uint8, eigenvalues (H, W, 3)) in FP64."""
    d = np.asarray(depth)
    if d.dtype == np.uint16:
        z = d.astype(np.float64) * depth_scale
        ok = d != 0
    else:
        z = d.astype(np.float64)
        ok = np.isfinite(z) & (z > 0)
    H, W = z.shape
    fx, fy, cx, cy = (float(v) for v in K)
    R = int(radius)
    normals = np.zeros((H, W, 3))
    evals = np.zeros((H, W, 3))
    valid = np.zeros((H, W), np.uint8)
    if H < 2 * R + 1 or W < 2 * R + 1:
        return normals, valid, evals
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    X = z * u[None, :]
    Y = z * v[:, None]
    Hi, Wi = H - 2 * R, W - 2 * R  # pixels whose window is inside the image
    pts = []
    oks = np.ones((Hi, Wi), bool)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            ys, xs = slice(R + dy, R + dy + Hi), slice(R + dx, R + dx + Wi)
            pts.append(np.stack([X[ys, xs], Y[ys, xs], z[ys, xs]], -1))
            oks &= ok[ys, xs]
    P = np.stack(pts, axis=2)                         # (Hi, Wi, n, 3)
    Pn = np.where(oks[..., None, None], P, 0.0)
    c = Pn.mean(axis=2, keepdims=True)
    Q = Pn - c
    S = np.einsum("hwni,hwnj->hwij", Q, Q)
    w, V = np.linalg.eigh(S)                          # ascending eigenvalues
    n = V[..., :, 0]
    centre = np.stack([X[R:R + Hi, R:R + Wi], Y[R:R + Hi, R:R + Wi], z[R:R + Hi, R:R + Wi]], -1)
    flip = (n * centre).sum(-1) < 0
    n = np.where(flip[..., None], -n, n)
    normals[R:R + Hi, R:R + Wi] = np.where(oks[..., None], n, 0.0)
    evals[R:R + Hi, R:R + Wi] = np.where(oks[..., None], w, 0.0)
    valid[R:R + Hi, R:R + Wi] = oks.astype(np.uint8)
    return normals, valid, evals
