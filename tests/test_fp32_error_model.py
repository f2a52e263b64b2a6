"""FP32 error model of the closed form (Eq. 4-6), on the CPU.

The kernel evaluates Eq. 4-6 in FP32 in a fixed order: the sums and
differences of opposite neighbours (exact for uint16 depths, which are scaled
only through the per-frame constants a, b, c), the products n_x = (a' S35) D24,
n_y = (b' S24) D35, P = (c' S24) S35, then n_z = fma(-u1, n_x, fma(-v1, n_y, P))
and q = |n|^2 by fused multiply-adds. This test restates that order in float32
arithmetic (every operation rounded to float32; a fused multiply-add formed in
float64 and rounded once) and compares it with the FP64 oracle on inputs that
stress it: random-primitive scenes, uint16 and float32, and planes tilted up
to the SECANT limit tau = 12 (about 85 degrees), for alpha = 1 to 16. It checks
the two claims behind the parity tolerances (reading C7):

* the direction of n is within 1e-6 rad of the oracle's (measured worst
  2.1e-7 rad; the parity tolerance is 1e-4 rad);
* the SECANT test q (1 + u1^2 + v1^2) <= tau^2 P^2 decides like the oracle's
  statistic except where that statistic is within 1e-6 relative of tau.
"""
import numpy as np
import pytest

import oracle
from synth import scenes

f32 = np.float32


def fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def shift(a, dx, dy, fill):
    H, W = a.shape
    b = np.full_like(a, fill)
    ys0, ys1 = max(0, -dy), min(H, H - dy)
    xs0, xs1 = max(0, -dx), min(W, W - dx)
    b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return b


def fp32_closed_form(depth, K, alpha, tau, depth_scale=0.001):
    """(n (H, W, 3) float32, secant mask, stencil-valid) in the kernel's order."""
    fx, fy, cx, cy = K
    if depth.dtype == np.uint16:
        d = depth.astype(f32)               # exact integers; the scale goes into a, b, c
        ok = depth != 0
        s = depth_scale
    else:
        d = depth.astype(f32)
        ok = np.isfinite(d) & (d > 0)
        s = 1.0
    d = np.where(ok, d, f32(np.nan))
    d2, d4 = shift(d, alpha, 0, np.nan), shift(d, -alpha, 0, np.nan)
    d3, d5 = shift(d, 0, alpha, np.nan), shift(d, 0, -alpha, np.nan)
    a = f32(-alpha / (4.0 * fy) * s * s)
    b = f32(-alpha / (4.0 * fx) * s * s)
    c = f32(alpha * alpha / (4.0 * fx * fy) * s * s)
    S24, D24 = (d2 + d4).astype(f32), (d2 - d4).astype(f32)
    S35, D35 = (d3 + d5).astype(f32), (d3 - d5).astype(f32)
    nx = (a * S35).astype(f32) * D24
    ny = (b * S24).astype(f32) * D35
    P = (c * S24).astype(f32) * S35
    H, W = depth.shape
    u = ((np.arange(W, dtype=f32) - f32(cx)) * f32(1.0 / fx)).astype(f32)[None, :] * np.ones((H, 1), f32)
    v = ((np.arange(H, dtype=f32) - f32(cy)) * f32(1.0 / fy)).astype(f32)[:, None] * np.ones((1, W), f32)
    nz = fma(-u, nx, fma(-v, ny, P))
    q = fma(nx, nx, fma(ny, ny, (nz * nz).astype(f32)))
    lhs = (q * (fma(u, u, np.ones_like(u)) + (v * v).astype(f32)).astype(f32)).astype(f32)
    rhs = (f32(tau * tau) * (P * P).astype(f32)).astype(f32)
    good = np.isfinite(q) & ok  # every stencil depth valid, the centre's too
    with np.errstate(invalid="ignore"):
        mask = good & (q >= f32(1.17549435e-38)) & (lhs <= rhs)
    return np.stack([nx, ny, nz], -1), mask, good


def angles(a, b):
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1))


def check(depth, K, alpha, tau=12.0):
    n, mask, good = fp32_closed_form(depth, K, alpha, tau)
    ref = oracle.forward(depth, K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=tau, nthreads=4)
    both = good & (ref.valid == 1) & mask
    assert both.sum() > 0
    ang = angles(n[both].astype(np.float64), ref.n_hat[both])
    assert ang.max() <= 1e-6, ang.max()
    with np.errstate(invalid="ignore"):
        near = np.isfinite(ref.stat) & (np.abs(ref.stat - tau) <= 1e-6 * tau)
    inner = np.zeros(depth.shape, bool)
    inner[alpha:-alpha, alpha:-alpha] = True
    mism = (mask != (ref.valid == 1)) & inner & ~near
    assert mism.sum() == 0, int(mism.sum())
    return ang.max()


@pytest.mark.parametrize("kind", ["u16", "f32"])
@pytest.mark.parametrize("alpha", [1, 2, 8, 16])
def test_scenes(kind, alpha):
    d, K = scenes.random_frame(77 + alpha, 640, 480, "cpu", kind=kind)
    check(d.numpy(), K, alpha)


@pytest.mark.parametrize("tilt_deg", [60, 75, 80, 84])
@pytest.mark.parametrize("alpha", [1, 4])
def test_grazing_planes(tilt_deg, alpha):
    """Planes up to just inside the SECANT limit, quantised to millimetres."""
    H, W = 120, 160
    K = (140.0, 140.0, 79.5, 59.5)
    t = np.radians(tilt_deg)
    n0 = np.array([np.sin(t) * 0.6, np.sin(t) * 0.8, np.cos(t)])
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    along = n0[0] * uu + n0[1] * vv + n0[2]
    with np.errstate(divide="ignore"):
        z = np.where(along > 1e-3, 1.5 / along, 0.0)
    raw = np.clip(np.round(z * 1000.0), 0, 65535).astype(np.uint16)
    raw[(z < 0.4) | (z > 6.0)] = 0
    check(raw, K, alpha)


@pytest.mark.parametrize("k", [2.0 ** -18, 2.0 ** 33])
@pytest.mark.parametrize("alpha", [1, 2])
def test_numerical_domain_ends(k, alpha):
    """The documented FP32 domain, 2^-28 <= alpha d / f <= 2^28: a float32 scene
    (0.4 .. 6 m, f = 525 px) scaled by k to depths of about 1.5e-6 .. 2.3e-5 m
    and 3.4e9 .. 5.2e10 m still meets both claims."""
    d, K = scenes.random_frame(91, 640, 480, "cpu", kind="f32")
    dd = (d.numpy().astype(np.float64) * k).astype(f32)
    valid = dd[dd > 0]
    f = min(K[0], K[1])
    assert alpha * valid.min() / f >= 2.0 ** -28 and alpha * valid.max() / f <= 2.0 ** 28
    check(dd, K, alpha)
