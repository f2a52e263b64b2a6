"""Planted mistakes in copies of the Python oracles (multi-scale, plane fit,
point cloud, evaluation) are each caught by at least one check below, which
the real oracles pass. A mutant is the module's source with one edit,
executed as a separate module; the real modules are never touched."""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import evaluation, multiscale, plane_fit, pointcloud

K = (80.0, 90.0, 15.3, 11.7)  # fx != fy and cx != cy
H, W = 24, 32


def load_variant(module, old=None, new=None):
    """The module itself (old is None) or a copy of it with one edit."""
    if old is None:
        return module
    path = module.__file__
    src = open(path).read()
    assert src.count(old) == 1, f"mutation site not unique in {os.path.basename(path)}: {old!r}"
    m = types.ModuleType(module.__name__ + "_mutant")
    m.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), m.__dict__)
    return m


def plane_depth(n0, c):
    fx, fy, cx, cy = K
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    return c / (n0[0] * u[None, :] + n0[1] * v[:, None] + n0[2])


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def shift(a, dx, dy, fill=np.nan):
    b = np.full_like(a, fill)
    ys0, ys1 = max(0, -dy), min(H, H - dy)
    xs0, xs1 = max(0, -dx), min(W, W - dx)
    b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return b


def caught(checks, mod):
    failed = []
    for c in checks:
        try:
            c(mod)
        except (AssertionError, ValueError, IndexError):
            failed.append(c.__name__)
    return failed


# ---------------------------------------------------------------- multi-scale
def ms_plane(ms):
    """Pair form on a plane: unit normals along the plane's, and
    n . ray = (1/K) sum_i alpha_i^2 d2_i d3_i / (fx fy) (Eq. 1-3)."""
    n0 = unit([0.3, -0.2, 0.93])
    d = plane_depth(n0, 2.0)
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    ray = np.stack([uu, vv, np.ones_like(uu)], -1)
    r = ms.multiscale(d, K, (1, 2), "pair", oracle.STAT_RAW, np.inf)
    v = r.valid == 1
    assert v.sum() == (H - 2) * (W - 2)
    assert np.abs(r.n_hat[v] @ n0 - 1.0).max() < 1e-12
    want = sum(a * a * shift(d, a, 0) * shift(d, 0, a) for a in (1, 2)) / (2 * fx * fy)
    np.testing.assert_allclose((r.n_raw * ray).sum(-1)[v], want[v], rtol=1e-11)


def ms_quad_single_scale(ms):
    rng = np.random.default_rng(21)
    d = rng.uniform(1.0, 1.1, size=(H, W))
    a = ms.multiscale(d, K, (2,), "quad", oracle.STAT_SECANT, 12.0)
    b = oracle.forward(d, K, alpha=2, stat_mode=oracle.STAT_SECANT, tau=12.0)
    np.testing.assert_allclose(a.n_raw, b.n_raw, rtol=1e-13, atol=1e-18)
    assert (a.valid == b.valid).all()


def ms_invalid(ms):
    """Valid only where every depth used at every scale is inside the image and valid."""
    rng = np.random.default_rng(22)
    d = rng.uniform(1.0, 1.05, size=(H, W))
    d[rng.random((H, W)) < 0.05] = 0.0
    ok = d > 0
    want = ok.copy()
    for a in (1, 3):
        want &= shift(ok.astype(float), a, 0, 0.0) > 0
        want &= shift(ok.astype(float), 0, a, 0.0) > 0
    got = ms.multiscale(d, K, (1, 3), "pair", oracle.STAT_RAW, np.inf).valid
    assert (got == want).all()


def ms_secant(ms):
    rng = np.random.default_rng(23)
    d = rng.uniform(1.0, 1.01, size=(H, W))
    r = ms.multiscale(d, K, (1, 2), "quad", oracle.STAT_SECANT, np.inf)
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    ray = np.stack([uu, vv, np.ones_like(uu)], -1)
    v = r.valid == 1
    want = np.linalg.norm(ray[v], axis=-1) / (r.n_hat[v] * ray[v]).sum(-1)
    np.testing.assert_allclose(r.stat[v], want, rtol=1e-12)


# ----------------------------------------------------------------- plane fit
def pf_plane(pf):
    n0 = unit([-0.25, 0.3, 0.92])
    d = plane_depth(n0, 1.7)
    n, valid, ev = pf.plane_fit(d, K, 2)
    v = valid == 1
    assert v.sum() == (H - 4) * (W - 4)
    assert np.abs(n[v] @ n0 - 1.0).max() < 1e-10
    assert (ev[v][:, 0] <= 1e-12 * ev[v][:, 2]).all()


def pf_window_validity(pf):
    """A hole invalidates exactly the pixels whose (2R+1)^2 window holds it."""
    d = plane_depth(unit([0.1, 0.1, 1.0]), 1.5)
    d[10, 14] = 0.0
    _, valid, _ = pf.plane_fit(d, K, 2)
    want = np.zeros((H, W), bool)
    want[2:H - 2, 2:W - 2] = True
    want[8:13, 12:17] = False
    assert (valid.astype(bool) == want).all()


def pf_uint16_scale(pf):
    rng = np.random.default_rng(24)
    raw = rng.integers(900, 1100, size=(H, W)).astype(np.uint16)
    _, _, ea = pf.plane_fit(raw, K, 1, depth_scale=0.002)
    _, _, eb = pf.plane_fit(raw.astype(np.float64) * 0.002, K, 1)
    np.testing.assert_allclose(ea, eb, rtol=1e-10, atol=1e-18)


# --------------------------------------------------------------- point cloud
def pc_rays(pc):
    rng = np.random.default_rng(25)
    d = rng.uniform(0.5, 4.0, size=(H, W))
    d[3, 4], d[5, 6] = -1.0, np.nan
    P = pc.points(d, K)
    fx, fy, cx, cy = K
    assert (P[3, 4] == 0).all() and (P[5, 6] == 0).all()
    ok = np.isfinite(d) & (d > 0)
    np.testing.assert_array_equal(P[..., 2][ok], d[ok])
    np.testing.assert_allclose(P[..., 0], np.where(ok, d * (np.arange(W)[None, :] - cx) / fx, 0.0), rtol=1e-15)
    np.testing.assert_allclose(P[..., 1], np.where(ok, d * (np.arange(H)[:, None] - cy) / fy, 0.0), rtol=1e-15)


# ---------------------------------------------------------------- evaluation
def ev_directions(ev):
    n = np.array([[[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]], np.float64)
    phi, theta = ev.spherical(n, np.ones((1, 6)))
    np.testing.assert_allclose(phi[0, :4], [0, np.pi / 2, np.pi, 3 * np.pi / 2], atol=1e-15)
    np.testing.assert_allclose(theta[0], [np.pi / 2] * 4 + [0, np.pi], atol=1e-15)
    phi, theta = ev.spherical(n, np.zeros((1, 6)))
    assert (phi == 0).all() and (theta == 0).all()


def ev_mse(ev):
    a = np.tile(np.array([0.0, 0.0, 1.0]), (2, 3, 1))
    b = a.copy()
    b[0, 0] = [1.0, 0.0, 0.0]          # theta differs by pi/2, phi by 0
    va = np.ones((2, 3), np.uint8)
    vb = va.copy()
    vb[1, 2] = 0
    mt, mp, cnt = ev.angle_mse(a, va, b, vb)
    assert cnt == 5
    np.testing.assert_allclose([mt, mp], [(np.pi / 2) ** 2 / 5, 0.0], atol=1e-15)


CASES = {
    "multiscale": (multiscale, [ms_plane, ms_quad_single_scale, ms_invalid, ms_secant], [
        ("P3 = _shift(P, 0, alpha, 0.0)", "P3 = _shift(P, 0, -alpha, 0.0)"),
        ("np.cross(P2 - P, P3 - P)", "np.cross(P3 - P, P2 - P)"),
        ("acc / len(alphas)", "acc / max(1, len(alphas) - 1)"),
        ("good &= g_i", "good |= g_i"),
        ("r * np.sqrt((ray * ray).sum(-1)) / along", "r / along"),
        ("b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]",
         "b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dy:xs1 + dy]"),
    ]),
    "plane_fit": (plane_fit, [pf_plane, pf_window_validity, pf_uint16_scale], [
        ("n = V[..., :, 0]", "n = V[..., :, 2]"),
        ("Q = Pn - c", "Q = Pn"),
        ("flip = (n * centre).sum(-1) < 0", "flip = (n * centre).sum(-1) > 0"),
        ("for dx in range(-R, R + 1):", "for dx in range(-R, R):"),
        ("z = d.astype(np.float64) * depth_scale", "z = d.astype(np.float64) * 0.001"),
        ("u = (np.arange(W) - cx) / fx", "u = (np.arange(W) - cx) / fy"),
    ]),
    "pointcloud": (pointcloud, [pc_rays], [
        ("P = np.stack([z * u[None, :], z * v[:, None], z], -1)",
         "P = np.stack([z * v[:, None], z * u[None, :], z], -1)"),
        ("return np.where(ok[..., None], P, 0.0)", "return P"),
        ("v = (np.arange(H) - cy) / fy", "v = (np.arange(H) - cx) / fy"),
    ]),
    "evaluation": (evaluation, [ev_directions, ev_mse], [
        ("phi = np.arctan2(n[..., 1], n[..., 0])", "phi = np.arctan2(n[..., 0], n[..., 1])"),
        ("phi = np.where(phi < 0.0, phi + 2.0 * np.pi, phi)", "phi = phi"),
        ("theta = np.arctan2(np.sqrt(n[..., 0] ** 2 + n[..., 1] ** 2), n[..., 2])",
         "theta = np.arctan2(n[..., 2], np.sqrt(n[..., 0] ** 2 + n[..., 1] ** 2))"),
        ("count = int(both.sum())", "count = int(both.size)"),
        ("both = np.asarray(valid_a).astype(bool) & np.asarray(valid_b).astype(bool)",
         "both = np.asarray(valid_a).astype(bool)"),
    ]),
}

PARAMS = [(name, i) for name, (_, _, muts) in CASES.items() for i in range(len(muts))]


@pytest.mark.parametrize("name", list(CASES))
def test_real_oracle_passes(name):
    module, checks, _ = CASES[name]
    assert caught(checks, load_variant(module)) == []


@pytest.mark.parametrize("name,i", PARAMS, ids=[f"{n}-{i}" for n, i in PARAMS])
def test_planted_mistake_is_caught(name, i):
    module, checks, muts = CASES[name]
    old, new = muts[i]
    assert caught(checks, load_variant(module, old, new)), f"{name}: nothing caught {old!r} -> {new!r}"
