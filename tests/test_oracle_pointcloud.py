"""Pins of the point-cloud oracle (Section 2's back-projection): points of a
ray-cast plane lie on that plane, every point lies on its pixel's viewing ray
with z equal to the depth, invalid depths give the origin, uint16 scaling."""
import math

import numpy as np

from oracle.pointcloud import points
from synth import scenes


def test_ray_cast_plane_points_lie_on_the_plane():
    H, W, K = 48, 64, (300.0, 280.0, 31.5, 23.5)
    n0 = np.array([0.3, -0.2, 0.93])
    n0 /= np.linalg.norm(n0)
    plane = scenes.Plane(n0, 2.1)
    D = scenes.cast(scenes.Scene([plane]), W, H, K, "cpu").numpy()
    P = points(D, K)
    np.testing.assert_allclose(P @ n0, 2.1, rtol=1e-13)


def test_points_lie_on_their_rays_with_z_the_depth():
    rng = np.random.default_rng(3)
    H, W, K = 13, 17, (120.0, 130.0, 7.0, 5.5)
    D = rng.uniform(0.5, 4.0, size=(H, W))
    P = points(D, K)
    np.testing.assert_array_equal(P[..., 2], D)
    for row in range(H):
        for col in range(W):
            assert math.isclose(P[row, col, 0], D[row, col] * (col - K[2]) / K[0], rel_tol=1e-15)
            assert math.isclose(P[row, col, 1], D[row, col] * (row - K[3]) / K[1], rel_tol=1e-15)
    # The principal point's ray is the optical axis.
    K2 = (100.0, 100.0, 3.0, 4.0)
    P2 = points(D, K2)
    assert P2[4, 3, 0] == 0.0 and P2[4, 3, 1] == 0.0


def test_invalid_depth_gives_the_origin_and_uint16_scales():
    D = np.array([[0.0, -1.0, np.nan], [np.inf, 1.0, 2.0]])
    P = points(D, (10.0, 10.0, 1.0, 0.5))
    assert (P[0] == 0).all() and (P[1, 0] == 0).all()
    assert (P[1, 1:, 2] == [1.0, 2.0]).all()
    raw = np.array([[0, 1500], [65535, 7]], np.uint16)
    Pu = points(raw, (50.0, 60.0, 0.5, 0.5), depth_scale=0.001)
    Pf = points(raw.astype(np.float64) * 0.001, (50.0, 60.0, 0.5, 0.5))
    Pf[0, 0] = 0.0
    np.testing.assert_allclose(Pu, Pf, rtol=1e-15)
    assert (Pu[0, 0] == 0).all()
