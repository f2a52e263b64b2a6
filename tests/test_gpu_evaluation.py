"""GPU evaluation kernels (Section 4: I_phi / I_theta images, MSE of Tables
2-5) against the FP64 evaluation oracle on identical float32 normal maps.

Tolerances: the kernels' arctangent (a polynomial fit after octant
reduction, about 3e-7 rad) and sqrtf give angles within 4e-6 rad
(absolute, phi compared modulo 2 pi). The MSE inputs keep every phi at least
0.1 rad from the 0 / 2 pi cut, where a rounding difference could move a
pixel's phi by 2 pi; there the MSE agrees to 1e-4 relative."""
import math

import numpy as np
import pytest
import torch

import paper_2209_08241_gb300 as nrm
from oracle import evaluation
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


def random_map(H, W, seed, phi_lo=0.1, phi_hi=2 * math.pi - 0.1):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(phi_lo, phi_hi, size=(H, W))
    th = rng.uniform(0.0, math.pi, size=(H, W))
    n = np.zeros((H, W, 4), np.float32)
    n[..., 0] = np.sin(th) * np.cos(phi)
    n[..., 1] = np.sin(th) * np.sin(phi)
    n[..., 2] = np.cos(th)
    v = (rng.random((H, W)) > 0.1).astype(np.uint8)
    return torch.from_numpy(n).to(DEV), torch.from_numpy(v).to(DEV)


def test_spherical_images_match_oracle_on_estimated_normals():
    d, K = scenes.cfg1_depth(DEV)
    est = nrm.NormalEstimator(K, 480, 640)
    n, m = est(d)
    phi, theta = nrm.spherical_images(n, m)
    rp, rt = evaluation.spherical(n.double().cpu().numpy(), m.cpu().numpy())
    dp = np.abs(phi.double().cpu().numpy() - rp)
    dp = np.minimum(dp, 2 * math.pi - dp)
    assert dp.max() <= 4e-6
    assert np.abs(theta.double().cpu().numpy() - rt).max() <= 4e-6
    mm = m.cpu().numpy() == 0
    assert (phi.cpu().numpy()[mm] == 0).all() and (theta.cpu().numpy()[mm] == 0).all()
    assert float(phi.max()) < 2 * math.pi and float(phi.min()) >= 0.0


def test_spherical_axis_directions():
    dirs = [(0, 0, 1), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (0, 0, -1)]
    expect_phi = [0.0, 0.0, math.pi / 2, math.pi, 1.5 * math.pi, 0.0]
    expect_th = [0.0, math.pi / 2, math.pi / 2, math.pi / 2, math.pi / 2, math.pi]
    n = torch.zeros((1, len(dirs), 4), device=DEV)
    n[0, :, :3] = torch.tensor(dirs, dtype=torch.float32)
    v = torch.ones((1, len(dirs)), dtype=torch.uint8, device=DEV)
    phi, theta = nrm.spherical_images(n, v)
    np.testing.assert_allclose(phi.cpu().numpy()[0], expect_phi, atol=4e-6)
    np.testing.assert_allclose(theta.cpu().numpy()[0], expect_th, atol=4e-6)


def test_spherical_signed_zeros_and_octant_boundaries():
    """atan2's conventions for signed zeros (-0 counts as negative x; the sign
    of y is kept, so phi = -0 stays -0 and -pi wraps to pi), both zero, and
    directions on the octant boundaries |x| = |y|, against the FP64 oracle on
    the same float32 inputs, exactly where the result is 0 or pi."""
    z, nz = 0.0, -0.0
    r = math.sqrt(0.5)
    dirs = [(z, z, 1), (nz, z, 1), (z, nz, 1), (nz, nz, 1), (-1, z, 0), (-1, nz, 0), (1, nz, 0), (1, z, 0),
            (z, z, -1), (nz, z, -1), (r, r, 0), (-r, r, 0), (-r, -r, 0), (r, -r, 0), (r, r, -1e-30),
            (1e-30, 1.0, 0), (-1e-30, 1.0, 0), (1.0, 1e-30, 0), (1.0, -1e-30, 0)]
    n = torch.zeros((1, len(dirs), 4), dtype=torch.float32)
    n[0, :, :3] = torch.tensor(dirs, dtype=torch.float32)
    v = torch.ones((1, len(dirs)), dtype=torch.uint8)
    phi, theta = nrm.spherical_images(n.to(DEV), v.to(DEV))
    rp, rt = evaluation.spherical(n.double().numpy(), v.numpy())
    gp, gt = phi.double().cpu().numpy(), theta.double().cpu().numpy()
    np.testing.assert_allclose(gp, rp, atol=4e-6, rtol=0)
    np.testing.assert_allclose(gt, rt, atol=4e-6, rtol=0)
    exact = (rp == 0) | (np.abs(rp - math.pi) < 1e-12)
    assert (np.abs(gp[exact] - rp[exact]) <= 2.5e-7).all()
    # phi = -1e-30 + 2 pi rounds to 2 pi itself (float32 here, float64 in the
    # oracle): the top of the range is reached only by such rounding.
    assert float(phi.max()) <= float(np.float32(2 * math.pi)) and float(phi.min()) >= -0.0


def test_spherical_dense_direction_sweep():
    """Unit normals on a dense grid of directions (every octant, both poles):
    both angle images within 4e-6 rad of the FP64 oracle (phi modulo 2 pi)."""
    ph = np.linspace(0.0, 2 * math.pi, 1441)
    th = np.linspace(0.0, math.pi, 721)
    P, T = np.meshgrid(ph, th)
    n = np.zeros(P.shape + (4,), np.float32)
    n[..., 0] = np.sin(T) * np.cos(P)
    n[..., 1] = np.sin(T) * np.sin(P)
    n[..., 2] = np.cos(T)
    v = np.ones(P.shape, np.uint8)
    phi, theta = nrm.spherical_images(torch.from_numpy(n).to(DEV), torch.from_numpy(v).to(DEV))
    rp, rt = evaluation.spherical(n.astype(np.float64), v)
    dp = np.abs(phi.double().cpu().numpy() - rp)
    dp = np.minimum(dp, 2 * math.pi - dp)
    assert dp.max() <= 4e-6
    assert np.abs(theta.double().cpu().numpy() - rt).max() <= 4e-6


@pytest.mark.parametrize("shape", [(1, 1), (7, 300), (480, 640), (1080, 1920)])
def test_angle_mse_matches_oracle_and_is_deterministic(shape):
    H, W = shape
    na, va = random_map(H, W, 1)
    nb, vb = random_map(H, W, 2)
    est = nrm.NormalEstimator((100.0, 100.0, 1.0, 1.0), 8, 8)
    out = nrm.angle_mse(est, na, va, nb, vb)
    out2 = nrm.angle_mse(est, na, va, nb, vb)
    assert torch.equal(out, out2)
    mt, mp, cnt = evaluation.angle_mse(na.double().cpu().numpy(), va.cpu().numpy(), nb.double().cpu().numpy(),
                                       vb.cpu().numpy())
    got = out.cpu().numpy()
    assert int(got[2]) == cnt
    if cnt:
        assert got[0] == pytest.approx(mt, rel=1e-4)
        assert got[1] == pytest.approx(mp, rel=1e-4)


def test_angle_mse_of_a_map_with_itself_is_zero_and_empty_masks_give_zero_count():
    na, va = random_map(64, 96, 3)
    est = nrm.NormalEstimator((100.0, 100.0, 1.0, 1.0), 8, 8)
    out = nrm.angle_mse(est, na, va, na, va).cpu().numpy()
    assert out[0] == 0.0 and out[1] == 0.0 and int(out[2]) == int(va.sum())
    zero = torch.zeros_like(va)
    out = nrm.angle_mse(est, na, zero, na, va).cpu().numpy()
    assert tuple(out) == (0.0, 0.0, 0.0)
