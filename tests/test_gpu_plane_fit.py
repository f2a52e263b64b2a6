"""GPU plane-fitting ground truth (Sections 1 and 4: the smallest-eigenvalue
eigenvector of the window's scatter matrix; radius 2 = the paper's 25 points)
against the FP64 plane-fit oracle. Masks are compared bit-exactly; normals
within the per-pixel Davis-Kahan bound derived in parity.py (the FP32 kernel's
scatter matrix is accurate to a few ulp of the window moment, so the error of
the eigenvector scales with moment / eigen-gap); the tests also require that
most valid pixels have a bound below 1e-3 rad (on these scenes the median
bound is 1e-5 to 1e-4 rad), so the comparison is not vacuous."""
import numpy as np
import pytest
import torch

import paper_2209_08241_gb300 as nrm
from oracle.plane_fit import plane_fit
from parity import angles, compare_plane_fit, plane_fit_banded, window_moment
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


def run_and_compare(depth, K, radius, orient=False, what=""):
    H, W = depth.shape
    in_dtype = "u16" if depth.dtype == torch.uint16 else "f32"
    est = nrm.NormalEstimator(K, H, W, nrm.NormalParams(orient_to_camera=orient), in_dtype=in_dtype)
    n, v = est.plane_fit(depth, radius)
    est.sync_status()
    D = depth.cpu().numpy()
    rn, rv, rev = plane_fit_banded(D, K, radius)
    M = window_moment(D, K, radius)
    return compare_plane_fit(n, v, rn, rv, rev, M, K, -1.0 if orient else 1.0, what)


@pytest.mark.parametrize("radius", [1, 2, 3, 4])
def test_cfg1_scene_f32(radius):
    d, K = scenes.cfg1_depth(DEV)
    cmp, tight, worst = run_and_compare(d, K, radius, what=f"cfg1 r{radius}")
    assert cmp > 0.8 * 480 * 640
    assert tight > 0.9 * cmp
    assert worst <= 1.0


@pytest.mark.parametrize("shape", [(173, 301), (8, 33), (250, 97)])
@pytest.mark.parametrize("orient", [False, True])
def test_u16_ragged_with_holes(shape, orient):
    H, W = shape
    d, K = scenes.random_frame(500 + H + W, W, H, DEV, kind="u16")
    cmp, tight, _ = run_and_compare(d, K, 2, orient, what=f"u16 {shape}")
    if H >= 40:
        assert tight > 0.85 * cmp


def test_tilted_plane_gives_its_normal():
    H, W, K = 120, 200, (180.0, 185.0, 99.5, 60.5)
    n0 = np.array([0.3, -0.45, 0.84])
    n0 /= np.linalg.norm(n0)
    u = (np.arange(W) - K[2]) / K[0]
    v = (np.arange(H) - K[3]) / K[1]
    uu, vv = np.meshgrid(u, v)
    D = (2.2 / (uu * n0[0] + vv * n0[1] + n0[2])).astype(np.float32)
    est = nrm.NormalEstimator(K, H, W)
    n, m = est.plane_fit(torch.from_numpy(D).to(DEV), 2)
    m = m.cpu().numpy()
    inner = np.zeros((H, W), bool)
    inner[2:-2, 2:-2] = True
    assert (m.astype(bool) == inner).all()
    g = n.cpu().numpy()[inner][:, :3].astype(np.float64)
    # atan2-based angles: arccos of a float32 dot product cannot resolve
    # angles below ~3e-4 rad.
    assert angles(g, np.broadcast_to(n0, g.shape)).max() < 1e-4


@pytest.mark.parametrize("shape", [(1, 1), (3, 3), (4, 7), (5, 5)])
def test_tiny_frames(shape):
    H, W = shape
    D = np.full((H, W), 1.5, np.float32)
    K = (100.0, 100.0, (W - 1) / 2, (H - 1) / 2)
    est = nrm.NormalEstimator(K, H, W)
    n, m = est.plane_fit(torch.from_numpy(D).to(DEV), 2)
    rn, rv, _ = plane_fit(D, K, 2)
    assert (m.cpu().numpy() == rv).all()
    if rv.any():  # the 5 x 5 frame: a fronto-parallel plane, normal (0, 0, 1)
        np.testing.assert_allclose(n.cpu().numpy()[rv == 1][:, :3], [[0.0, 0.0, 1.0]], atol=1e-6)


def test_radius_outside_range_is_rejected():
    est = nrm.NormalEstimator((100.0, 100.0, 10.0, 10.0), 20, 20)
    d = torch.ones((20, 20), device=DEV)
    for r in (0, -1, nrm._lib.NRM_MAX_PLANE_RADIUS + 1):
        with pytest.raises(nrm._lib.NrmError):
            est.plane_fit(d, r)


def test_fullsize_1080p_u16_sampled_bands():
    """The bench's frame size and input type (1920 x 1080 uint16 millimetres):
    three row bands (top edge, middle, bottom edge), each with its halo, against
    the oracle on the band."""
    W, H, R = 1920, 1080, 2
    d, K = scenes.random_frame(4242, W, H, DEV, kind="u16")
    est = nrm.NormalEstimator(K, H, W, in_dtype="u16")
    n, v = est.plane_fit(d, R)
    est.sync_status()
    D = d.cpu().numpy()
    n, v = n.cpu().numpy(), v.cpu().numpy()
    fx, fy, cx, cy = K
    for r0, r1 in ((0, 24), (530, 560), (1056, 1080)):
        a, b = max(0, r0 - R), min(H, r1 + R)
        Kc = (fx, fy, cx, cy - a)
        rn, rv, rev = plane_fit(D[a:b], Kc, R)
        M = window_moment(D[a:b], Kc, R)
        s = slice(r0 - a, r1 - a)
        cmp, tight, _ = compare_plane_fit(n[r0:r1], v[r0:r1], rn[s], rv[s], rev[s], M[s], (fx, fy, cx, cy - r0),
                                          what=f"1080p rows {r0}-{r1}")
        assert cmp > 0
