"""FP64 oracle of the multi-scale variant: the average of per-scale normals over
pixel distances alpha_1..alpha_K (Section 2, the authors' previous method,
and its equations after Eq. 3), with the Section 3.2 statistic and mask
applied to the average.

TEST INFRASTRUCTURE (same rules as the rest of ``oracle/``).

Steps, for each pixel (col, row):
  1. back-projection P = d (u, v, 1), u = (col - cx)/fx, v = (row - cy)/fy
     (Section 2, definitions below Eq. 3);
  2. for each scale alpha_i (reading: every neighbour depth is sampled at the
     scale's own distance alpha_i; the printed sums index alpha_i only):
       form "pair" (the previous method, Eq. 1-3 as a cross product):
         n_i = s12 x s13, s1k = P_k - P_1, with neighbours
         2 = (col + alpha_i, row) and 3 = (col, row + alpha_i);
       form "quad" (the proposed four-direction average, Section 3.1):
         n_i = the unnormalised normal of ``oracle.forward`` at alpha_i;
  3. n = (1/K) sum_i n_i (the printed averages);
  4. r = ||n||; statistic RAW = r, SECANT = r ||ray|| / (n . ray) (+inf when
     n . ray <= 0); valid iff every depth used at every scale lies in the image
     and is valid, r > 0 and statistic <= tau (Section 3.2);
  5. unit normal n / r (negated with ``orient``), zero where invalid.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import STAT_RAW, STAT_SECANT, OracleResult

FORMS = ("pair", "quad")


def _decode(depth, depth_scale):
    d = np.asarray(depth)
    if d.dtype == np.uint16:
        return d.astype(np.float64) * depth_scale, d != 0
    z = d.astype(np.float64)
    return z, np.isfinite(z) & (z > 0)


def _shift(a, dx, dy, fill):
    """b[row, col] = a[row + dy, col + dx] where inside, else ``fill``."""
    H, W = a.shape[:2]
    b = np.full_like(a, fill)
    ys0, ys1 = max(0, -dy), min(H, H - dy)
    xs0, xs1 = max(0, -dx), min(W, W - dx)
    if ys1 > ys0 and xs1 > xs0:
        b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return b


def _pair_normal(z, ok, K, alpha):
    """Eq. 1-3 as the cross product s12 x s13 at distance alpha, and the
    validity of its three depths."""
    H, W = z.shape
    fx, fy, cx, cy = K
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    P = np.stack([z * u[None, :], z * v[:, None], z], -1)
    P = np.where(ok[..., None], P, 0.0)
    P2 = _shift(P, alpha, 0, 0.0)
    P3 = _shift(P, 0, alpha, 0.0)
    good = ok & _shift(ok, alpha, 0, False) & _shift(ok, 0, alpha, False)
    return np.cross(P2 - P, P3 - P), good


def multiscale(depth, K, alphas, form: str = "pair", stat_mode: int = STAT_SECANT, tau: float = 12.0,
               depth_scale: float = 0.001, orient: int = 0) -> OracleResult:
    """Multi-scale normals, statistic and mask of one depth map (H x W)."""
    if form not in FORMS:
        raise ValueError(f"form must be one of {FORMS}")
    alphas = [int(a) for a in alphas]
    if not alphas or min(alphas) < 1:
        raise ValueError("need at least one positive scale")
    K = tuple(float(k) for k in K)
    z, ok = _decode(depth, depth_scale)
    H, W = z.shape
    acc = np.zeros((H, W, 3))
    good = np.ones((H, W), bool)
    for a in alphas:
        if form == "pair":
            n_i, g_i = _pair_normal(z, ok, K, a)
        else:
            res = oracle.forward(np.asarray(depth), K, alpha=a, stat_mode=STAT_RAW, tau=np.inf,
                                 depth_scale=depth_scale)
            n_i, g_i = res.n_raw, np.isfinite(res.r)
        acc += np.where(g_i[..., None], n_i, 0.0)
        good &= g_i
    n = np.where(good[..., None], acc / len(alphas), 0.0)
    r = np.sqrt((n * n).sum(-1))
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    ray = np.stack([uu, vv, np.ones_like(uu)], -1)
    if stat_mode == STAT_RAW:
        stat = r.copy()
    elif stat_mode == STAT_SECANT:
        along = (n * ray).sum(-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            stat = np.where(along > 0, r * np.sqrt((ray * ray).sum(-1)) / along, np.inf)
    else:
        raise ValueError("stat_mode")
    r = np.where(good, r, np.nan)
    stat = np.where(good, stat, np.nan)
    with np.errstate(invalid="ignore"):
        valid = good & (r > 0) & (stat <= tau)
    s = -1.0 if orient else 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        n_hat = np.where(valid[..., None], s * n / r[..., None], 0.0)
    return OracleResult(n, n_hat, r, stat, valid.astype(np.uint8))
