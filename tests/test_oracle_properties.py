"""Property-based pins of the oracles over random planes, intrinsics, pixel
distances and depth maps (Section 3.1, Eq. 4-6; Section 3.2; the multi-scale
average of Section 2; the plane fit of Sections 1 and 4):

* a plane n0 . P = c0 seen from the origin gives n_hat = n0 / |n0| exactly on
  every pixel whose stencil is inside the image;
* n . (u1, v1, 1) = alpha^2 (d2 + d4)(d3 + d5) / (4 fx fy) for any depths (the
  n_z row of Eq. 6);
* scaling the depth map by k leaves n_hat and the SECANT statistic unchanged
  and multiplies the RAW statistic by k^2;
* on a plane, the multi-scale average (either form, any scale set) and the
  plane fit (any radius) return the plane's normal.
"""
import numpy as np
import pytest

import oracle

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import assume, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

BIG = 1e300


def rays(H, W, K):
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    return np.stack([uu, vv, np.ones_like(uu)], -1)


def shift(a, dx, dy):
    H, W = a.shape
    b = np.full_like(a, np.nan)
    ys0, ys1 = max(0, -dy), min(H, H - dy)
    xs0, xs1 = max(0, -dx), min(W, W - dx)
    b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return b


intrinsics = st.tuples(st.floats(50.0, 600.0), st.floats(50.0, 600.0), st.floats(-5.0, 25.0),
                       st.floats(-5.0, 25.0))


@settings(max_examples=60, deadline=None, derandomize=True)
@given(nx=st.floats(-0.6, 0.6), ny=st.floats(-0.6, 0.6), c0=st.floats(0.3, 8.0), K=intrinsics,
       alpha=st.integers(1, 3), H=st.integers(7, 20), W=st.integers(7, 20))
def test_random_plane_is_exact(nx, ny, c0, K, alpha, H, W):
    n0 = np.array([nx, ny, 1.0])
    n0 /= np.linalg.norm(n0)
    along = rays(H, W, K) @ n0
    assume(along.min() > 0.05)  # the plane is in front of every pixel
    D = c0 / along
    res = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=BIG)
    inner = np.zeros((H, W), bool)
    inner[alpha:H - alpha, alpha:W - alpha] = True
    assert (res.valid.astype(bool) == inner).all()
    if inner.any():
        assert np.abs(res.n_hat[inner] @ n0 - 1.0).max() < 1e-11


@settings(max_examples=60, deadline=None, derandomize=True)
@given(seed=st.integers(0, 2**31 - 1), K=intrinsics, alpha=st.integers(1, 3), lo=st.floats(0.2, 5.0),
       spread=st.floats(0.0, 3.0))
def test_ray_identity_for_any_depths(seed, K, alpha, lo, spread):
    rng = np.random.default_rng(seed)
    H, W = 12, 15
    D = lo + spread * rng.random((H, W))
    res = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=BIG)
    v = res.valid.astype(bool)
    got = (res.n_raw * rays(H, W, K)).sum(-1)
    want = alpha ** 2 * (shift(D, alpha, 0) + shift(D, -alpha, 0)) * (shift(D, 0, alpha) + shift(D, 0, -alpha)) \
        / (4 * K[0] * K[1])
    np.testing.assert_allclose(got[v], want[v], rtol=1e-10)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(seed=st.integers(0, 2**31 - 1), k=st.floats(0.01, 100.0), alpha=st.integers(1, 2))
def test_depth_scaling(seed, k, alpha):
    rng = np.random.default_rng(seed)
    H, W = 10, 13
    K = (120.0, 110.0, 6.0, 4.5)
    D = 1.0 + 0.05 * rng.random((H, W))
    a = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=BIG)
    b = oracle.forward(k * D, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=BIG)
    v = a.valid.astype(bool)
    assert (b.valid == a.valid).all()
    np.testing.assert_allclose(b.n_hat[v], a.n_hat[v], atol=1e-12)
    np.testing.assert_allclose(b.r[v], k * k * a.r[v], rtol=1e-12)
    s1 = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=BIG)
    s2 = oracle.forward(k * D, K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=BIG)
    np.testing.assert_allclose(s2.stat[v], s1.stat[v], rtol=1e-12)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(nx=st.floats(-0.5, 0.5), ny=st.floats(-0.5, 0.5), c0=st.floats(0.5, 6.0), K=intrinsics,
       alphas=st.lists(st.integers(1, 4), min_size=1, max_size=4, unique=True),
       form=st.sampled_from(["pair", "quad"]))
def test_multiscale_random_plane_is_exact(nx, ny, c0, K, alphas, form):
    """Every scale's stencil on a plane spans the plane, so the averaged
    normal is the plane's for any set of pixel distances and either form."""
    from oracle.multiscale import multiscale
    H, W = 16, 18
    n0 = np.array([nx, ny, 1.0])
    n0 /= np.linalg.norm(n0)
    along = rays(H, W, K) @ n0
    assume(along.min() > 0.05)
    res = multiscale(c0 / along, K, alphas, form, oracle.STAT_RAW, BIG)
    v = res.valid.astype(bool)
    amax = max(alphas)
    lo = 0 if form == "pair" else amax
    assert v.sum() == (H - amax - lo) * (W - amax - lo)
    assert np.abs(res.n_hat[v] @ n0 - 1.0).max() < 1e-11


@settings(max_examples=30, deadline=None, derandomize=True)
@given(nx=st.floats(-0.5, 0.5), ny=st.floats(-0.5, 0.5), c0=st.floats(0.5, 6.0), K=intrinsics,
       radius=st.integers(1, 3))
def test_plane_fit_random_plane_is_exact(nx, ny, c0, K, radius):
    """The window of a plane has a zero smallest eigenvalue whose eigenvector
    is the plane's normal, oriented away from the camera."""
    from oracle.plane_fit import plane_fit
    H, W = 14, 15
    n0 = np.array([nx, ny, 1.0])
    n0 /= np.linalg.norm(n0)
    along = rays(H, W, K) @ n0
    assume(along.min() > 0.05)
    n, valid, ev = plane_fit(c0 / along, K, radius)
    v = valid.astype(bool)
    assert v.sum() == (H - 2 * radius) * (W - 2 * radius)
    assert np.abs(n[v] @ n0 - 1.0).max() < 1e-9
    assert (ev[v][:, 0] <= 1e-12 * ev[v][:, 2]).all()
