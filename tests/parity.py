"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances (fixed for this method; the FP32 closed form of Eq. 4-6 stays far inside them):
  * normals: angular error <= 1e-4 rad for float32 output, 5e-3 rad for half;
  * mask: bit-exact, except pixels whose oracle statistic lies within 1e-6
    relative of tau; those are excluded, counted and returned.
"""
import numpy as np
import torch

ANG_TOL_F32 = 1e-4
ANG_TOL_F16 = 5e-3
NEAR_TAU_REL = 1e-6


def angles(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    c = np.linalg.norm(np.cross(a, b), axis=-1)
    d = np.sum(a * b, axis=-1)
    return np.arctan2(c, d)


def decode_oct16(codes):
    """float64 unit vectors from octahedral int16 codes (..., 2): the inverse
    of the encoding documented in include/nrm.h, written independently here."""
    q = np.asarray(codes, np.float64) / 32767.0
    x, y = q[..., 0], q[..., 1]
    z = 1.0 - np.abs(x) - np.abs(y)
    sx = np.where(x >= 0, 1.0, -1.0)
    sy = np.where(y >= 0, 1.0, -1.0)
    vx = np.where(z < 0, (1.0 - np.abs(y)) * sx, x)
    vy = np.where(z < 0, (1.0 - np.abs(x)) * sy, y)
    v = np.stack([vx, vy, z], -1)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


# 16-bit octahedral quantisation: each code coordinate is off by at most
# 0.5/32767; each column of the decode's Jacobian has length sqrt(2), so the
# unnormalised v moves by at most sqrt(2)/32767, and |v| >= 1/sqrt(3), so the
# direction moves by at most sqrt(6)/32767 ~ 7.5e-5 rad (plus FP32 rounding).
ANG_TOL_OCT16 = 1e-4


def compare_oct16(codes, valid, ref, tau, what=""):
    """Octahedral codes (H, W, 2) int16 from the GPU against the oracle."""
    if isinstance(codes, torch.Tensor):
        codes = codes.cpu().numpy()
    if isinstance(valid, torch.Tensor):
        valid = valid.cpu().numpy()
    m = valid.astype(np.uint8)
    with np.errstate(invalid="ignore"):
        near = np.isfinite(ref.stat) & (np.abs(ref.stat - tau) <= NEAR_TAU_REL * tau)
    mism = (m != ref.valid) & ~near
    assert mism.sum() == 0, f"{what}: {int(mism.sum())} mask mismatches"
    assert (codes[m == 0] == 0).all(), f"{what}: masked pixels must carry code 0"
    both = (m == 1) & (ref.valid == 1)
    max_ang = 0.0
    if both.any():
        ang = angles(decode_oct16(codes[both]), ref.n_hat[both])
        max_ang = float(ang.max())
        assert max_ang <= ANG_TOL_OCT16, f"{what}: max angular error {max_ang:.3g} rad > {ANG_TOL_OCT16}"
    return int(near.sum()), max_ang, int(both.sum())


def compare(normals, valid, ref, tau, half=False, what=""):
    """normals (H, W, 4) and valid (H, W) from the GPU (torch or numpy) against an
    oracle result. Returns (near_tau_count, max_angle, n_valid)."""
    if isinstance(normals, torch.Tensor):
        normals = normals.detach().float().cpu().numpy()
    if isinstance(valid, torch.Tensor):
        valid = valid.cpu().numpy()
    n = normals[..., :3].astype(np.float64)
    m = valid.astype(np.uint8)
    assert set(np.unique(m)).issubset({0, 1}), f"{what}: mask bytes must be 0/1"
    with np.errstate(invalid="ignore"):
        near = np.isfinite(ref.stat) & (np.abs(ref.stat - tau) <= NEAR_TAU_REL * tau)
    mism = (m != ref.valid) & ~near
    assert mism.sum() == 0, (f"{what}: {int(mism.sum())} mask mismatches, e.g. at "
                             f"{np.argwhere(mism)[:5].tolist()}")
    assert (normals[m == 0] == 0).all(), f"{what}: masked pixels must carry (0,0,0,0)"
    assert (normals[..., 3] == 0).all(), f"{what}: 4th component must be 0"
    both = (m == 1) & (ref.valid == 1)
    max_ang = 0.0
    if both.any():
        ang = angles(n[both], ref.n_hat[both])
        max_ang = float(ang.max())
        tol = ANG_TOL_F16 if half else ANG_TOL_F32
        assert max_ang <= tol, f"{what}: max angular error {max_ang:.3g} rad > {tol}"
    return int(near.sum()), max_ang, int(both.sum())


def plane_fit_banded(depth, K, radius, depth_scale=0.001, band=64):
    """The plane-fitting oracle run on bands of rows (each with its radius-row
    halo and cy shifted to the band's first row): identical to one call on the
    whole image, in bounded memory."""
    from oracle.plane_fit import plane_fit
    D = np.asarray(depth)
    H, W = D.shape
    fx, fy, cx, cy = (float(v) for v in K)
    n = np.zeros((H, W, 3))
    v = np.zeros((H, W), np.uint8)
    ev = np.zeros((H, W, 3))
    for r0 in range(0, H, band):
        r1 = min(H, r0 + band)
        a, b = max(0, r0 - radius), min(H, r1 + radius)
        nn, vv, ee = plane_fit(D[a:b], (fx, fy, cx, cy - a), radius, depth_scale)
        n[r0:r1], v[r0:r1], ev[r0:r1] = nn[r0 - a:r1 - a], vv[r0 - a:r1 - a], ee[r0 - a:r1 - a]
    return n, v, ev


def window_moment(depth, K, radius, depth_scale=0.001):
    """M = sum over each pixel's window of |P - P_centre|^2 (the scale of the
    FP32 sums a kernel forms relative to the centre point); 0 where undefined."""
    D = np.asarray(depth)
    z = D.astype(np.float64) * (depth_scale if D.dtype == np.uint16 else 1.0)
    H, W = z.shape
    fx, fy, cx, cy = (float(v) for v in K)
    X = z * ((np.arange(W) - cx) / fx)[None, :]
    Y = z * ((np.arange(H) - cy) / fy)[:, None]
    P = np.stack([X, Y, z], -1)
    P = np.where(np.isfinite(P), P, 0.0)
    R = radius
    M = np.zeros((H, W))
    Hi, Wi = H - 2 * R, W - 2 * R
    if Hi <= 0 or Wi <= 0:
        return M
    c = P[R:R + Hi, R:R + Wi]
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            q = P[R + dy:R + dy + Hi, R + dx:R + dx + Wi] - c
            M[R:R + Hi, R:R + Wi] += (q * q).sum(-1)
    return M


# Per-pixel bound for an FP32 plane fit against the FP64 oracle. The kernel's
# window coordinates relative to the centre point carry relative errors of a
# few ulp, so its scatter matrix is off by at most ~45 eps M (eps = 2^-24, M
# the window moment above; products, 25-term sums and the mean subtraction),
# and Jacobi adds a few eps ||S|| <= eps M. By the Davis-Kahan bound the
# smallest eigenvector then moves by at most ~50 eps M / (lambda_2 - lambda_1)
# = 3e-6 M / gap, which is the tolerance (on the synthetic scenes the largest
# observed constant was 2.4e-7), plus 1e-6 rad for the final normalisation.
PLANE_TOL_ABS = 1e-6
PLANE_TOL_REL = 3e-6


def compare_plane_fit(normals, valid, ref_n, ref_v, ref_ev, M, K, orient_sign=1.0, what=""):
    """GPU (H, W, 4) float32 plane-fit normals and mask against the oracle.
    Returns (pixels compared, pixels where the bound is below 1e-3 rad, max of
    angle / bound)."""
    if isinstance(normals, torch.Tensor):
        normals = normals.cpu().numpy()
    if isinstance(valid, torch.Tensor):
        valid = valid.cpu().numpy()
    assert (valid.astype(np.uint8) == ref_v).all(), \
        f"{what}: {int((valid != ref_v).sum())} mask mismatches"
    assert (normals[valid == 0] == 0).all(), f"{what}: invalid pixels must carry normal 0"
    ok = valid == 1
    if not ok.any():
        return 0, 0, 0.0
    g = normals[ok][:, :3].astype(np.float64)
    assert (normals[ok][:, 3] == 0).all()
    assert np.abs(np.linalg.norm(g, axis=-1) - 1).max() < 1e-5, f"{what}: normals not unit"
    r = orient_sign * ref_n[ok]
    ev = ref_ev[ok]
    gap = ev[:, 1] - ev[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        tol = PLANE_TOL_ABS + PLANE_TOL_REL * M[ok] / gap
    tol = np.where(gap > 0, tol, np.inf)
    ang_signed = angles(g, r)
    ang = np.minimum(ang_signed, np.pi - ang_signed)      # the eigenvector's line
    bad = ang > tol
    assert not bad.any(), f"{what}: {int(bad.sum())} normals outside the bound (worst angle " \
                          f"{float(ang[bad].max()):.3g})"
    # Orientation: where the line is determined and the view is not grazing
    # (|n . ray| well above the bound), the side must match too.
    H, W = valid.shape
    fx, fy, cx, cy = (float(v) for v in K)
    yy, xx = np.nonzero(ok)
    ray = np.stack([(xx - cx) / fx, (yy - cy) / fy, np.ones_like(xx, dtype=np.float64)], -1)
    ray /= np.linalg.norm(ray, axis=-1, keepdims=True)
    decided = (tol < 1e-2) & (np.abs((r * ray).sum(-1)) > 2 * tol)
    flipped = ang_signed > np.pi / 2
    assert not (flipped & decided).any(), f"{what}: {int((flipped & decided).sum())} normals flipped"
    return int(ok.sum()), int((tol < 1e-3).sum()), float(np.max(ang / tol))


def ms_kappa(depth, K, alphas, form, depth_scale=0.001):
    """Cancellation factor of a multi-scale average, from the oracle: sum of the
    per-scale |n_i| over |sum of n_i| (1 where the scales agree, large where
    they cancel; inf where the sum vanishes)."""
    from oracle import STAT_RAW
    from oracle.multiscale import multiscale
    D = np.asarray(depth)
    tot = None
    mag = None
    for a in alphas:
        r = multiscale(D, K, [a], form, STAT_RAW, np.inf, depth_scale)
        tot = r.n_raw if tot is None else tot + r.n_raw
        m = np.linalg.norm(r.n_raw, axis=-1)
        mag = m if mag is None else mag + m
    den = np.linalg.norm(tot, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den > 0, mag / den, np.inf)


# The widened band may exclude at most this fraction of a frame's pixels
# beyond those the plain 1e-6 band excludes (kappa is large only where the
# per-scale normals nearly cancel, which is rare on real surfaces).
MS_KAPPA_EXCLUDED_FRAC = 1e-4


def compare_ms(normals, valid, ref, tau, kappa, half=False, what=""):
    """Multi-scale output against the multi-scale oracle. As ``compare``, but a
    pixel is excluded from the mask comparison when its statistic is within
    1e-6 kappa relative of tau: the FP32 sums over scales carry relative errors
    of a few ulp of the per-scale magnitudes, i.e. kappa times more relative to
    the average. The pixels excluded only because of the widening are counted
    and bounded by MS_KAPPA_EXCLUDED_FRAC of the frame. Returns
    (near_tau_count, max_angle, n_valid, max kappa over the compared pixels)."""
    if isinstance(normals, torch.Tensor):
        normals = normals.detach().float().cpu().numpy()
    if isinstance(valid, torch.Tensor):
        valid = valid.cpu().numpy()
    n = normals[..., :3].astype(np.float64)
    m = valid.astype(np.uint8)
    assert set(np.unique(m)).issubset({0, 1}), f"{what}: mask bytes must be 0/1"
    band = NEAR_TAU_REL * np.maximum(1.0, np.nan_to_num(kappa, nan=1.0, posinf=1e30))
    with np.errstate(invalid="ignore"):
        near = np.isfinite(ref.stat) & (np.abs(ref.stat - tau) <= band * tau)
        near_plain = np.isfinite(ref.stat) & (np.abs(ref.stat - tau) <= NEAR_TAU_REL * tau)
    widened_only = int((near & ~near_plain).sum())
    assert widened_only <= MS_KAPPA_EXCLUDED_FRAC * m.size, (
        f"{what}: the kappa-widened band excluded {widened_only} pixels (> {MS_KAPPA_EXCLUDED_FRAC} of {m.size})")
    mism = (m != ref.valid) & ~near
    assert mism.sum() == 0, (f"{what}: {int(mism.sum())} mask mismatches, e.g. at "
                             f"{np.argwhere(mism)[:5].tolist()}")
    assert (normals[m == 0] == 0).all(), f"{what}: masked pixels must carry (0,0,0,0)"
    assert (normals[..., 3] == 0).all(), f"{what}: 4th component must be 0"
    both = (m == 1) & (ref.valid == 1)
    max_ang, max_k = 0.0, 1.0
    if both.any():
        ang = angles(n[both], ref.n_hat[both])
        max_ang = float(ang.max())
        max_k = float(np.max(kappa[both]))
        tol = ANG_TOL_F16 if half else ANG_TOL_F32
        assert max_ang <= tol, f"{what}: max angular error {max_ang:.3g} rad > {tol} (max kappa {max_k:.3g})"
    return int(near.sum()), max_ang, int(both.sum()), max_k
