"""FP32 error model of the adjoint (derivatives of Eq. 4-6 and of the
normalisation, mask held fixed), on the CPU.

The adjoint kernel forms, per valid pixel, the four weights w2..w5 in FP32 in a
fixed order (the Eq. 4-6 factors a S35, b D35, c S35, a D24, b S24, c S24,
n, q, rsqrt, the projection h of the upstream gradient, then the weights by
fused multiply-adds) and gathers dL/dd_q = w2(q - a x) + w4(q + a x) + w3(q - a y)
+ w5(q + a y) in that order. This test restates the order in float32 (fused
multiply-adds formed in float64 and rounded once; the reciprocal square root
exact, where the kernel's hardware rsqrt adds up to about 2 ulp) and compares
it with the oracle's complex-step VJP of the direct four-cross form. It checks
the claim behind the adjoint parity tolerance (1e-3 relative on entries above
1e-3 of the crop maximum): the FP32 restatement stays within 1e-4 of it
(measured 2.5e-5 to 4.4e-5: the gather's four-term sums cancel on the
smaller entries), ten times inside."""
import numpy as np
import pytest

import oracle
from synth import scenes
from test_fp32_error_model import fma, shift

f32 = np.float32


def fp32_adjoint(depth, K, g, valid, alpha, sign=1.0):
    fx, fy, cx, cy = K
    d = depth.astype(f32)
    H, W = d.shape
    ka, kb, kc = f32(alpha / (4.0 * fy)), f32(alpha / (4.0 * fx)), f32(alpha * alpha / (4.0 * fx * fy))
    d2, d4 = shift(d, alpha, 0, 0.0), shift(d, -alpha, 0, 0.0)
    d3, d5 = shift(d, 0, alpha, 0.0), shift(d, 0, -alpha, 0.0)
    S24, D24 = (d2 + d4).astype(f32), (d2 - d4).astype(f32)
    S35, D35 = (d3 + d5).astype(f32), (d3 - d5).astype(f32)
    u1 = ((np.arange(W, dtype=f32) - f32(cx)) * f32(1.0 / fx)).astype(f32)[None, :] * np.ones((H, 1), f32)
    v1 = ((np.arange(H, dtype=f32) - f32(cy)) * f32(1.0 / fy)).astype(f32)[:, None] * np.ones((1, W), f32)
    A35, B35, C35 = (ka * S35).astype(f32), (kb * D35).astype(f32), (kc * S35).astype(f32)
    A24, B24, C24 = (ka * D24).astype(f32), (kb * S24).astype(f32), (kc * S24).astype(f32)
    nx, ny, P = (-A35 * D24).astype(f32), (-B24 * D35).astype(f32), (C24 * S35).astype(f32)
    nz = fma(-u1, nx, fma(-v1, ny, P))
    q = fma(nx, nx, fma(ny, ny, (nz * nz).astype(f32)))
    inv = (1.0 / np.sqrt(np.maximum(q, f32(1.17549435e-38)).astype(np.float64))).astype(f32)
    hx0, hy0, hz0 = (nx * inv).astype(f32), (ny * inv).astype(f32), (nz * inv).astype(f32)
    gx, gy, gz = (g[..., k].astype(f32) for k in range(3))
    gd = fma(gx, hx0, fma(gy, hy0, (gz * hz0).astype(f32)))
    si = (f32(sign) * inv).astype(f32)
    hx = (fma(-gd, hx0, gx) * si).astype(f32)
    hy = (fma(-gd, hy0, gy) * si).astype(f32)
    hz = (fma(-gd, hz0, gz) * si).astype(f32)
    e_x, e_y = fma(-u1, hz, hx), fma(-v1, hz, hy)
    c35 = fma(hz, C35, (-e_y * B35).astype(f32))
    c24 = fma(hz, C24, (-e_x * A24).astype(f32))
    on = valid == 1
    w2 = np.where(on, fma(-e_x, A35, c35), f32(0))
    w3 = np.where(on, fma(-e_y, B24, c24), f32(0))
    w4 = np.where(on, fma(e_x, A35, c35), f32(0))
    w5 = np.where(on, fma(e_y, B24, c24), f32(0))
    # dL/dd_q = w2(q - a x) + w4(q + a x) + w3(q - a y) + w5(q + a y)
    out = (shift(w2, -alpha, 0, 0.0) + shift(w4, alpha, 0, 0.0)).astype(f32)
    out = (out + shift(w3, 0, -alpha, 0.0)).astype(f32)
    out = (out + shift(w5, 0, alpha, 0.0)).astype(f32)
    return out


@pytest.mark.parametrize("alpha", [1, 2, 4])
def test_adjoint_fp32_model(alpha):
    d, K = scenes.random_frame(4004, 160, 120, "cpu", kind="f32", holes=False, clip_range=False)
    D = d.numpy()
    ref = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=12.0, nthreads=4)
    valid = ref.valid.astype(np.uint8)
    rng = np.random.default_rng(alpha)
    g = rng.normal(size=D.shape + (3,))
    got = fp32_adjoint(D, K, g, valid, alpha).astype(np.float64)
    exact = oracle.vjp(D, K, g, valid, alpha=alpha, nthreads=4)
    scale = np.abs(exact).max()
    big = np.abs(exact) > 1e-3 * scale
    rel = np.abs(got - exact)[big] / np.abs(exact)[big]
    assert rel.max() <= 1e-4, rel.max()
    assert np.abs(got - exact)[~big].max(initial=0) <= 1e-4 * scale
