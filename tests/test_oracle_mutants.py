"""The oracle's pins are strong enough: plausible mistakes planted in copies of
the oracle source (a neighbour on the wrong side, a flipped tangent, a dropped
or transposed cross product, a mixed-up intrinsic, a missing factor, a strict
threshold, a skipped validity test, an ignored flag, a wrong statistic, a wrong
adjoint stencil) each fail at least one of the checks below, which the real
oracle passes. The mutants are compiled on the CPU into a temporary directory
and swapped in for the real library only inside this test."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle

K = (80.0, 90.0, 15.3, 11.7)  # fx != fy and cx != cy, so mixed-up intrinsics show
H, W = 24, 32
FLAGS = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread"]

# (name, text in oracle/nrm_oracle.cpp, replacement); each text occurs once.
MUTANTS = [
    ("neighbour 2 on the wrong side", "back_project(d[1], col + alpha, row, K)",
     "back_project(d[1], col - alpha, row, K)"),
    ("tangent s13 reversed", "Vec3<T> s13 = P3 - P1;", "Vec3<T> s13 = P1 - P3;"),
    ("a cross product dropped",
     "cross(s12, s13) + cross(s13, s14) + cross(s14, s15) + cross(s15, s12)",
     "cross(s12, s13) + cross(s13, s14) + cross(s14, s15)"),
    ("operands of a cross product transposed",
     "cross(s12, s13) + cross(s13, s14)", "cross(s13, s12) + cross(s13, s14)"),
    ("u uses the row principal point", "double u = ((double)col - K.cx) / K.fx;",
     "double u = ((double)col - K.cy) / K.fx;"),
    ("v uses the column focal length", "double v = ((double)row - K.cy) / K.fy;\n  return",
     "double v = ((double)row - K.cy) / K.fx;\n  return"),
    ("the 1/4 dropped", "scaled(sum, T(0.25))", "scaled(sum, T(1.0))"),
    ("strict threshold", "stat <= p.tau", "stat < p.tau"),
    ("centre depth not validated", "return ok[0] && ok[1] && ok[2] && ok[3] && ok[4];",
     "return ok[1] && ok[2] && ok[3] && ok[4];"),
    ("orientation flag ignored", "double s = (p.orient ? -1.0 : 1.0) / r;", "double s = 1.0 / r;"),
    ("uint16 scale ignored", "* f.depth_scale;", "* 0.001;"),
    ("secant statistic without the ray length", "r * std::sqrt(dot(ray, ray)) / along", "r / along"),
    ("adjoint stencil with a neighbour counted twice",
     "const int pr[5] = {qrow, qrow, qrow - alpha, qrow, qrow + alpha};",
     "const int pr[5] = {qrow, qrow, qrow + alpha, qrow, qrow + alpha};"),
]


def plane_depth(n0, c):
    fx, fy, cx, cy = K
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    return c / (n0[0] * u[None, :] + n0[1] * v[:, None] + n0[2])


def ray_grid():
    fx, fy, cx, cy = K
    uu, vv = np.meshgrid((np.arange(W) - cx) / fx, (np.arange(H) - cy) / fy)
    return np.stack([uu, vv, np.ones_like(uu)], -1)


def shift(a, dx, dy):
    """b[row, col] = a[row + dy, col + dx] where inside, else NaN."""
    b = np.full_like(a, np.nan)
    ys0, ys1 = max(0, -dy), min(H, H - dy)
    xs0, xs1 = max(0, -dx), min(W, W - dx)
    b[ys0:ys1, xs0:xs1] = a[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return b


def check_plane():
    """A tilted plane: unit normals parallel to the plane's (paper sign), and
    n . ray equal to alpha^2 (d2 + d4)(d3 + d5) / (4 fx fy) (Eq. 6)."""
    n0 = np.array([0.3, -0.2, 0.93])
    n0 /= np.linalg.norm(n0)
    d = plane_depth(n0, 2.0)
    ray = ray_grid()
    for alpha in (1, 2):
        r = oracle.forward(d, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=np.inf)
        v = r.valid == 1
        assert v.sum() == (H - 2 * alpha) * (W - 2 * alpha)
        assert np.abs(r.n_hat[v] @ n0 - 1.0).max() < 1e-12
        along = (r.n_raw * ray).sum(-1)
        want = alpha ** 2 * (shift(d, alpha, 0) + shift(d, -alpha, 0)) * \
            (shift(d, 0, alpha) + shift(d, 0, -alpha)) / (4 * K[0] * K[1])
        np.testing.assert_allclose(along[v], want[v], rtol=1e-11)


def check_threshold_tie():
    """stat == tau counts as valid; the next smaller tau rejects the pixel."""
    n0 = np.array([-0.4, 0.35, 0.85])
    d = plane_depth(n0 / np.linalg.norm(n0), 1.5)
    r = oracle.forward(d, K, alpha=1, stat_mode=oracle.STAT_SECANT, tau=np.inf)
    t = float(r.stat[H // 2, W // 2])
    assert oracle.forward(d, K, alpha=1, tau=t).valid[H // 2, W // 2] == 1
    assert oracle.forward(d, K, alpha=1, tau=np.nextafter(t, 0.0)).valid[H // 2, W // 2] == 0


def check_invalid_depths():
    """Brute force: valid exactly where all five stencil depths are inside the
    image and positive finite (RAW, tau = inf)."""
    rng = np.random.default_rng(11)
    d = rng.uniform(1.0, 1.3, size=(H, W))
    bad = rng.random((H, W)) < 0.08
    d[bad] = rng.choice([0.0, -1.0, np.nan, np.inf], size=bad.sum())
    ok = np.isfinite(d) & (d > 0)
    for alpha in (1, 2):
        want = ok.copy()
        for dx, dy in ((alpha, 0), (-alpha, 0), (0, alpha), (0, -alpha)):
            s = shift(ok.astype(float), dx, dy)
            want &= np.nan_to_num(s, nan=0.0) > 0
        got = oracle.forward(d, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=np.inf).valid
        assert (got == want).all()


def check_orientation():
    rng = np.random.default_rng(12)
    d = rng.uniform(1.0, 1.1, size=(H, W))
    a = oracle.forward(d, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=np.inf)
    b = oracle.forward(d, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=np.inf, orient=1)
    assert (a.valid == b.valid).all() and a.valid.any()
    np.testing.assert_array_equal(b.n_hat, -a.n_hat)


def check_uint16_scale():
    rng = np.random.default_rng(13)
    raw = rng.integers(800, 1200, size=(H, W)).astype(np.uint16)
    a = oracle.forward(raw, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=np.inf, depth_scale=0.002)
    b = oracle.forward(raw.astype(np.float64) * 0.002, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=np.inf)
    np.testing.assert_allclose(a.r, b.r, rtol=1e-12)
    np.testing.assert_allclose(a.n_hat, b.n_hat, rtol=1e-12, atol=1e-15)


def check_secant():
    """SECANT statistic = ||ray|| / (n_hat . ray), the inverse cosine of the
    angle between the normal and the viewing ray."""
    rng = np.random.default_rng(14)
    d = rng.uniform(1.0, 1.02, size=(H, W))
    r = oracle.forward(d, K, alpha=1, stat_mode=oracle.STAT_SECANT, tau=np.inf)
    ray = ray_grid()
    v = r.valid == 1
    want = np.linalg.norm(ray[v], axis=-1) / (r.n_hat[v] * ray[v]).sum(-1)
    np.testing.assert_allclose(r.stat[v], want, rtol=1e-12)


def check_vjp():
    """The complex-step adjoint against central differences of the forward
    (mask held fixed) on a small crop."""
    rng = np.random.default_rng(15)
    n0 = np.array([0.2, 0.1, 0.97])
    d = plane_depth(n0 / np.linalg.norm(n0), 1.8) + 0.01 * rng.standard_normal((H, W))
    g = rng.standard_normal((H, W, 3))
    m = oracle.forward(d, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=np.inf).valid

    def loss(x):
        n = oracle.forward(x, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=np.inf).n_hat
        return float((g * n * m[..., None]).sum())

    got = oracle.vjp(d, K, g, m, alpha=1, crop=(8, 10, 3, 4))
    for i in range(3):
        for j in range(4):
            h = 1e-6
            dp, dm = d.copy(), d.copy()
            dp[8 + i, 10 + j] += h
            dm[8 + i, 10 + j] -= h
            fd = (loss(dp) - loss(dm)) / (2 * h)
            assert abs(got[i, j] - fd) <= 1e-6 * max(1.0, abs(fd))


CHECKS = [check_plane, check_threshold_tie, check_invalid_depths, check_orientation, check_uint16_scale,
          check_secant, check_vjp]


def failing_checks():
    failed = []
    for c in CHECKS:
        try:
            c()
        except (AssertionError, ValueError):
            failed.append(c.__name__)
    return failed


def test_real_oracle_passes_every_check():
    assert failing_checks() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path, monkeypatch):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not unique"
    path = tmp_path / "mutant.cpp"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(FLAGS + [str(path), "-o", str(lib)], check=True)
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(str(lib))))
    assert failing_checks(), f"no check caught the planted mistake: {name}"
