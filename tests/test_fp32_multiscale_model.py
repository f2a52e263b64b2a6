"""FP32 error model of the multi-scale average (Section 2's scale average with
the Eq. 1-3 pair or the Eq. 4-6 four-direction stencil per scale), on the CPU.

The multi-scale kernel accumulates, per pixel and scale, n_x += (A_i S) D,
n_y += (B_i S') D', P += (C_i S'') S''' in FP32 fused multiply-adds starting
from -0, with per-scale constants formed in FP64 and rounded once (1/K, the
depth scale^2 and the sign folded in), then the single-scale epilogue. This
test restates that order in float32 (a fused multiply-add formed in float64
and rounded once) and compares it with the FP64 multi-scale oracle. It checks
the claims behind the multi-scale parity tolerances: the direction is within
1e-6 kappa rad of the oracle's (kappa = sum |n_i| / |sum n_i|, the per-pixel
cancellation factor), within the 1e-4 rad parity tolerance everywhere, and
the SECANT mask decides like the oracle outside the 1e-6 kappa band around
tau, a band that excludes at most MS_KAPPA_EXCLUDED_FRAC of a frame beyond the
plain 1e-6 band."""
import numpy as np
import pytest

import oracle
from oracle.multiscale import multiscale
from parity import MS_KAPPA_EXCLUDED_FRAC, ms_kappa
from synth import scenes
from test_fp32_error_model import angles, fma, shift

f32 = np.float32


def fp32_multiscale(depth, K, alphas, form, tau, depth_scale=0.001):
    fx, fy, cx, cy = K
    if depth.dtype == np.uint16:
        d = depth.astype(f32)
        ok = depth != 0
        s = depth_scale
    else:
        d = depth.astype(f32)
        ok = np.isfinite(d) & (d > 0)
        s = 1.0
    d = np.where(ok, d, f32(np.nan))
    H, W = depth.shape
    nsc = len(alphas)
    q4 = 4.0 if form == "quad" else 1.0
    ax = np.full((H, W), f32(-0.0))
    ay = np.full((H, W), f32(-0.0))
    ap = np.full((H, W), f32(-0.0))
    for a in alphas:
        A = f32(-(a / (q4 * fy) * s * s) / nsc)
        B = f32(-(a / (q4 * fx) * s * s) / nsc)
        C = f32((a * a / (q4 * fx * fy) * s * s) / nsc)
        d2, d3 = shift(d, a, 0, np.nan), shift(d, 0, a, np.nan)
        if form == "pair":
            D21, D31 = (d2 - d).astype(f32), (d3 - d).astype(f32)
            ax = fma((A * d3).astype(f32), D21, ax)
            ay = fma((B * d2).astype(f32), D31, ay)
            ap = fma((C * d2).astype(f32), d3, ap)
        else:
            d4, d5 = shift(d, -a, 0, np.nan), shift(d, 0, -a, np.nan)
            S24, D24 = (d2 + d4).astype(f32), (d2 - d4).astype(f32)
            S35, D35 = (d3 + d5).astype(f32), (d3 - d5).astype(f32)
            ax = fma((A * S35).astype(f32), D24, ax)
            ay = fma((B * S24).astype(f32), D35, ay)
            ap = fma((C * S24).astype(f32), S35, ap)
    u = ((np.arange(W, dtype=f32) - f32(cx)) * f32(1.0 / fx)).astype(f32)[None, :] * np.ones((H, 1), f32)
    v = ((np.arange(H, dtype=f32) - f32(cy)) * f32(1.0 / fy)).astype(f32)[:, None] * np.ones((1, W), f32)
    nz = fma(-u, ax, fma(-v, ay, ap))
    q = fma(ax, ax, fma(ay, ay, (nz * nz).astype(f32)))
    lhs = (q * (fma(u, u, np.ones_like(u)) + (v * v).astype(f32)).astype(f32)).astype(f32)
    rhs = (f32(tau * tau) * (ap * ap).astype(f32)).astype(f32)
    good = np.isfinite(q) & ok
    with np.errstate(invalid="ignore"):
        mask = good & (q >= f32(1.17549435e-38)) & (lhs <= rhs)
    return np.stack([ax, ay, nz], -1), mask, good


@pytest.mark.parametrize("form", ["pair", "quad"])
@pytest.mark.parametrize("alphas", [(1, 2, 3, 4), (1, 3, 8), (2,)])
@pytest.mark.parametrize("kind", ["u16", "f32"])
def test_multiscale_fp32_model(form, alphas, kind):
    tau = 12.0
    d, K = scenes.random_frame(303 + sum(alphas), 320, 240, "cpu", kind=kind)
    D = d.numpy()
    n, mask, good = fp32_multiscale(D, K, list(alphas), form, tau)
    ref = multiscale(D, K, list(alphas), form, oracle.STAT_SECANT, tau, 0.001, 0)
    kappa = ms_kappa(D, K, list(alphas), form)
    both = good & (ref.valid == 1) & mask
    assert both.sum() > 1000
    ang = angles(n[both].astype(np.float64), ref.n_hat[both])
    assert ang.max() <= 1e-4
    assert (ang <= 1e-6 * np.maximum(kappa[both], 1.0)).all(), float((ang / np.maximum(kappa[both], 1.0)).max())
    with np.errstate(invalid="ignore"):
        stat_ok = np.isfinite(ref.stat)
        near_plain = stat_ok & (np.abs(ref.stat - tau) <= 1e-6 * tau)
        near = stat_ok & (np.abs(ref.stat - tau) <= 1e-6 * np.where(np.isfinite(kappa), np.maximum(kappa, 1.0),
                                                                    np.inf) * tau)
    amax = max(alphas)
    inner = np.zeros(D.shape, bool)
    inner[amax:-amax, amax:-amax] = True
    mism = (mask != (ref.valid == 1)) & inner & ~near
    assert mism.sum() == 0, int(mism.sum())
    assert int((near & ~near_plain).sum()) <= MS_KAPPA_EXCLUDED_FRAC * D.size
