"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances (stated by the task for this method):
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
