"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test states what it pins and which plausible mistake it catches:
closed-form surfaces (tilted planes, spheres, cylinders), the paper's own
reformulation (Eq. "proof of efficiency" last line, Eq. 4-6) and single-pair
form (Eq. 1-3), invariants that follow from Eq. 4-6, brute-force labels on
hand-made step edges, a hand-worked fixture, and the gradient against finite
differences and a closed form.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from synth import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BIG = 1e300  # a threshold that masks nothing


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def angle(a, b):
    """Angle (rad) between vectors along the last axis, robust near 0."""
    a, b = unit(a), unit(b)
    c = np.linalg.norm(np.cross(a, b), axis=-1)
    d = np.sum(a * b, axis=-1)
    return np.arctan2(c, d)


def rays(H, W, K):
    fx, fy, cx, cy = K
    u = (np.arange(W) - cx) / fx
    v = (np.arange(H) - cy) / fy
    uu, vv = np.meshgrid(u, v)
    return np.stack([uu, vv, np.ones_like(uu)], -1)


def border_mask(H, W, alpha):
    m = np.zeros((H, W), bool)
    m[alpha:H - alpha, alpha:W - alpha] = True
    return m


# ----------------------------------------------------------- golden fixture

def _load_golden(name):
    rec = {"pixel": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "pixel":
                rec["pixel"].append([float(v) for v in vals])
            else:
                rec[key] = [float(v) for v in vals]
    return rec


def test_hand_worked_fixture():
    """Hand-worked 5x5 example (tests/golden/hand_worked_5x5.txt): pins the
    neighbour layout, the 1/4 factor, the sign and the secant statistic."""
    g = _load_golden("hand_worked_5x5.txt")
    D = np.array(g["depth"], np.float64).reshape(5, 5)
    K = g["K"]
    a = int(g["alpha"][0])
    res = oracle.forward(D, K, alpha=a, stat_mode=oracle.STAT_SECANT, tau=BIG)
    for col, row, nx, ny, nz, r, stat in g["pixel"]:
        col, row = int(col), int(row)
        np.testing.assert_allclose(res.n_raw[row, col], [nx, ny, nz], rtol=0, atol=1e-14)
        assert res.r[row, col] == pytest.approx(r, rel=1e-15)
        assert res.stat[row, col] == pytest.approx(stat, rel=1e-15)
        np.testing.assert_allclose(res.n_hat[row, col], np.array([nx, ny, nz]) / r, atol=1e-15)
    assert int((res.valid == 0).sum()) == int(g["invalid_border"][0])
    assert res.valid[1:4, 1:4].all()


def test_threshold_tie_counts_as_valid():
    """Reading C6: a pixel is invalid iff stat > tau, so stat == tau is valid.
    On the hand-worked fixture r(2, 2) = sqrt(5.5) exactly in FP64."""
    g = _load_golden("hand_worked_5x5.txt")
    D = np.array(g["depth"], np.float64).reshape(5, 5)
    r = math.sqrt(5.5)
    at = oracle.forward(D, g["K"], alpha=1, stat_mode=oracle.STAT_RAW, tau=r)
    below = oracle.forward(D, g["K"], alpha=1, stat_mode=oracle.STAT_RAW,
                           tau=float(np.nextafter(r, 0.0)))
    assert at.r[2, 2] == r
    assert at.valid[2, 2] == 1 and below.valid[2, 2] == 0
    assert (below.n_hat[2, 2] == 0).all()


# ------------------------------------------------------------- tilted plane

def plane_depth(n0, c0, H, W, K):
    return c0 / (rays(H, W, K) @ np.asarray(n0, np.float64))


@pytest.mark.parametrize("axis", ["x", "y", "xy"])
@pytest.mark.parametrize("tilt_deg", [0, 15, 30, 45, 60, 70, 80])
def test_tilted_plane_exact(axis, tilt_deg):
    """A plane n0 . P = c0 gives n_hat = sign(c0) n0/|n0| exactly (s24 and s35
    are chords of the plane). Catches any dropped term, wrong index or sign."""
    t = math.radians(tilt_deg)
    if axis == "x":
        n0 = [0.0, math.sin(t), math.cos(t)]
    elif axis == "y":
        n0 = [math.sin(t), 0.0, math.cos(t)]
    else:
        n0 = [math.sin(t) * 0.6, math.sin(t) * 0.8, math.cos(t)]
    H, W = 24, 32
    K = (400.0, 380.0, 15.5, 11.5)  # narrow field of view keeps n0 . ray > 0
    D = plane_depth(n0, 2.0, H, W, K)
    assert (D > 0).all()
    for alpha in (1, 2, 3):
        res = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=BIG)
        inner = border_mask(H, W, alpha)
        assert (res.valid.astype(bool) == inner).all()
        err = angle(res.n_hat[inner], np.broadcast_to(n0, res.n_hat[inner].shape))
        assert err.max() <= 1e-11, (tilt_deg, alpha, err.max())
        # The secant statistic of a plane is 1/cos of the normal-ray angle.
        R = rays(H, W, K)[inner]
        cos_g = (R @ unit(n0)) / np.linalg.norm(R, axis=-1)
        np.testing.assert_allclose(res.stat[inner], 1.0 / cos_g, rtol=1e-11)


def test_plane_sign_follows_offset():
    """n0 . P = c0 with c0 > 0 viewed from the origin: n_hat = +n0/|n0| and it
    points away from the camera (n_hat . P > 0). orient=1 negates it."""
    H, W, K = 16, 16, (300.0, 300.0, 7.5, 7.5)
    n0 = unit([0.2, -0.1, 1.0])
    D = plane_depth(n0, 1.5, H, W, K)
    res = oracle.forward(D, K, alpha=1, tau=BIG)
    inner = border_mask(H, W, 1)
    np.testing.assert_allclose(res.n_hat[inner], np.broadcast_to(n0, (inner.sum(), 3)), atol=1e-12)
    flipped = oracle.forward(D, K, alpha=1, tau=BIG, orient=1)
    np.testing.assert_allclose(flipped.n_hat[inner], -res.n_hat[inner], atol=0)


# ------------------------------------------------------- sphere and cylinder

def _exact_depth(prim, H, W, K):
    d = scenes.cast(scenes.Scene([prim]), W, H, K, "cpu").numpy()
    return np.where(np.isfinite(d), d, 0.0)


def _curved_errors(prim, true_normal_fn, col, row, alphas, K, H, W):
    D = _exact_depth(prim, H, W, K)
    errs = []
    for a in alphas:
        res = oracle.forward(D, K, alpha=a, tau=BIG)
        assert res.valid[row, col]
        P = D[row, col] * rays(H, W, K)[row, col]
        n_true = true_normal_fn(P)
        # Paper sign: the normal points away from the camera.
        if np.dot(n_true, P) < 0:
            n_true = -n_true
        assert np.dot(res.n_hat[row, col], n_true) > 0
        errs.append(float(angle(res.n_hat[row, col], n_true)))
    return errs


def test_sphere_second_order_convergence():
    """The estimator is a central difference: the angular error on a sphere is
    O(alpha^2) (ratio 4 per halving of alpha/f) and small at alpha = 1."""
    H, W = 241, 321
    K = (525.0, 525.0, 160.0, 120.0)
    C = np.array([0.15, -0.05, 2.0])
    R = 0.5
    sph = scenes.Sphere(C, R)
    errs = _curved_errors(sph, lambda P: (P - C) / R, 190, 100, (1, 2, 4, 8), K, H, W)
    ratios = [errs[i + 1] / errs[i] for i in range(3)]
    for q in ratios:
        assert 3.6 <= q <= 4.4, (errs, ratios)
    # Bound: (alpha d / f)^2 / R^2 with d ~ 2 m.
    assert errs[0] < (1 * 2.0 / 525.0) ** 2 / R ** 2


def test_cylinder_second_order_convergence():
    H, W = 241, 321
    K = (525.0, 525.0, 160.0, 120.0)
    C = np.array([-0.1, 0.05, 1.8])
    A = unit([0.3, 1.0, 0.2])
    R = 0.35
    cyl = scenes.Cylinder(C, A, R, 2.0)

    def radial(P):
        w = P - C
        return w - np.dot(w, A) * A

    errs = _curved_errors(cyl, radial, 140, 130, (1, 2, 4, 8), K, H, W)
    ratios = [errs[i + 1] / errs[i] for i in range(3)]
    for q in ratios:
        assert 3.6 <= q <= 4.4, (errs, ratios)


# -------------------------------------------------------- form equivalence

def _closed_form(D, K, alpha):
    """Eq. 4-6 written out (independent of the oracle's direct form)."""
    fx, fy, cx, cy = K
    H, W = D.shape
    out = np.full((H, W, 3), np.nan)
    a = alpha
    for y in range(a, H - a):
        for x in range(a, W - a):
            d2, d4 = D[y, x + a], D[y, x - a]
            d3, d5 = D[y + a, x], D[y - a, x]
            u1, v1 = (x - cx) / fx, (y - cy) / fy
            nx = -a / (4 * fy) * (d3 + d5) * (d2 - d4)
            ny = -a / (4 * fx) * (d2 + d4) * (d3 - d5)
            nz = -u1 * nx - v1 * ny + a * a / (4 * fx * fy) * (d2 + d4) * (d3 + d5)
            out[y, x] = (nx, ny, nz)
    return out


def _one_cross(D, K, alpha):
    """1/4 s24 x s35 from back-projected points (last line of the "proof of
    efficiency" equation)."""
    fx, fy, cx, cy = K
    H, W = D.shape
    out = np.full((H, W, 3), np.nan)
    a = alpha

    def P(x, y):
        return D[y, x] * np.array([(x - cx) / fx, (y - cy) / fy, 1.0])

    for y in range(a, H - a):
        for x in range(a, W - a):
            s24 = P(x - a, y) - P(x + a, y)
            s35 = P(x, y - a) - P(x, y + a)
            out[y, x] = 0.25 * np.cross(s24, s35)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("alpha", [1, 2])
def test_direct_form_equals_reformulations(seed, alpha):
    """Direct four-cross average (oracle) == 1/4 s24 x s35 == Eq. 4-6 on random
    8x8 maps. Pins the neighbour layout (C2) and the 1/4 factor."""
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.5, 5.0, size=(8, 8))
    K = (rng.uniform(300, 700), rng.uniform(300, 700), rng.uniform(2, 6), rng.uniform(2, 6))
    res = oracle.forward(D, K, alpha=alpha, tau=BIG)
    inner = border_mask(8, 8, alpha)
    cf = _closed_form(D, K, alpha)[inner]
    oc = _one_cross(D, K, alpha)[inner]
    got = res.n_raw[inner]
    scale = np.linalg.norm(cf, axis=-1, keepdims=True)
    assert np.abs(got - cf).max() / scale.min() <= 1e-11
    assert (np.abs(got - cf) / scale).max() <= 1e-12
    assert (np.abs(oc - cf) / scale).max() <= 1e-12


def test_single_pair_layout_eq_1_3():
    """Eq. 1-3 (single tangent pair of the earlier method) equal s12 x s13 only
    with point 2 at +alpha along the column and point 3 at +alpha along the row:
    the layout reading that the oracle uses."""
    rng = np.random.default_rng(7)
    fx, fy, cx, cy = 500.0, 470.0, 3.2, 2.9
    for _ in range(20):
        x, y, a = 4, 3, int(rng.integers(1, 3))
        d1, d2, d3 = rng.uniform(0.5, 4, size=3)
        u1, v1 = (x - cx) / fx, (y - cy) / fy
        P1 = d1 * np.array([u1, v1, 1])
        P2 = d2 * np.array([(x + a - cx) / fx, v1, 1])
        P3 = d3 * np.array([u1, (y + a - cy) / fy, 1])
        n = np.cross(P2 - P1, P3 - P1)
        nx = -a / fy * d3 * (d2 - d1)
        ny = -a / fx * d2 * (d3 - d1)
        nz = a / fx * v1 * d2 * (d3 - d1) + a / fy * u1 * d3 * (d2 - d1) + a * a / (fx * fy) * d2 * d3
        np.testing.assert_allclose(n, [nx, ny, nz], rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def scene_f64():
    d, K = scenes.random_frame(11, 160, 120, kind="f64", holes=True, dropout=0.01)
    return d.numpy(), K


def test_unit_length_and_sign(scene_f64):
    D, K = scene_f64
    res = oracle.forward(D, K, alpha=2, tau=BIG)
    v = res.valid.astype(bool)
    assert v.sum() > 0.8 * v.size
    np.testing.assert_allclose(np.linalg.norm(res.n_hat[v], axis=-1), 1.0, atol=1e-15)
    R = rays(*D.shape, K)
    assert ((res.n_hat[v] * R[v]).sum(-1) > 0).all()
    assert (res.n_hat[~v] == 0).all()


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_ray_identity_from_eq6(scene_f64, alpha):
    """Eq. 6 rearranged: n . (u1, v1, 1) = alpha^2/(4 fx fy) (d2+d4)(d3+d5)."""
    D, K = scene_f64
    fx, fy, cx, cy = K
    res = oracle.forward(D, K, alpha=alpha, tau=BIG)
    v = res.valid.astype(bool)
    H, W = D.shape
    a = alpha
    Dp = np.pad(D, a)
    d2 = Dp[a:a + H, 2 * a:2 * a + W]
    d4 = Dp[a:a + H, 0:W]
    d3 = Dp[2 * a:2 * a + H, a:a + W]
    d5 = Dp[0:H, a:a + W]
    rhs = a * a / (4 * fx * fy) * (d2 + d4) * (d3 + d5)
    lhs = (res.n_raw * rays(H, W, K)).sum(-1)
    # The direct form subtracts back-projected points a few pixels apart, which
    # costs about f/alpha (~130 here) in relative rounding: 1e-12 covers it.
    np.testing.assert_allclose(lhs[v], rhs[v], rtol=1e-12)


def test_centre_depth_does_not_enter(scene_f64):
    """Eq. 4-6 have no d1: changing the centre depth leaves n unchanged."""
    D, K = scene_f64
    base = oracle.forward(D, K, alpha=2, tau=BIG)
    D2 = D.copy()
    D2[40, 50] *= 1.37
    moved = oracle.forward(D2, K, alpha=2, tau=BIG)
    n0, n1 = base.n_raw[40, 50], moved.n_raw[40, 50]
    assert base.valid[40, 50] and moved.valid[40, 50]
    assert np.abs(n0 - n1).max() <= 1e-13 * np.linalg.norm(n0)


def test_depth_scale_invariance(scene_f64):
    """D -> kD: n_hat unchanged, RAW r scales by k^2, SECANT unchanged."""
    D, K = scene_f64
    k = 2.5
    a = oracle.forward(D, K, alpha=2, stat_mode=oracle.STAT_RAW, tau=BIG)
    b = oracle.forward(k * D, K, alpha=2, stat_mode=oracle.STAT_RAW, tau=BIG)
    v = a.valid.astype(bool)
    np.testing.assert_allclose(b.n_hat[v], a.n_hat[v], atol=1e-13)
    np.testing.assert_allclose(b.r[v], k * k * a.r[v], rtol=1e-13)
    s1 = oracle.forward(D, K, alpha=2, stat_mode=oracle.STAT_SECANT, tau=BIG)
    s2 = oracle.forward(k * D, K, alpha=2, stat_mode=oracle.STAT_SECANT, tau=BIG)
    np.testing.assert_allclose(s2.stat[v], s1.stat[v], rtol=1e-13)


def test_mirror_and_transpose_symmetry(scene_f64):
    """With a centred camera, flipping columns negates n_x; flipping rows negates
    n_y; transposing (with fx<->fy, cx<->cy) swaps n_x and n_y. Pins which image
    axis is u and which is v, and the signs of Eq. 4-5."""
    D, _ = scene_f64
    H, W = D.shape
    K = (300.0, 280.0, (W - 1) / 2, (H - 1) / 2)
    base = oracle.forward(D, K, alpha=2, tau=BIG)
    fl = oracle.forward(D[:, ::-1].copy(), K, alpha=2, tau=BIG)
    m = fl.n_hat[:, ::-1]
    np.testing.assert_allclose(m[..., 0], -base.n_hat[..., 0], atol=1e-13)
    np.testing.assert_allclose(m[..., 1:], base.n_hat[..., 1:], atol=1e-13)
    fv = oracle.forward(D[::-1, :].copy(), K, alpha=2, tau=BIG)
    m = fv.n_hat[::-1, :]
    np.testing.assert_allclose(m[..., 1], -base.n_hat[..., 1], atol=1e-13)
    np.testing.assert_allclose(m[..., [0, 2]], base.n_hat[..., [0, 2]], atol=1e-13)
    KT = (K[1], K[0], K[3], K[2])
    tr = oracle.forward(D.T.copy(), KT, alpha=2, tau=BIG)
    t = tr.n_hat.transpose(1, 0, 2)
    np.testing.assert_allclose(t[..., 0], base.n_hat[..., 1], atol=1e-13)
    np.testing.assert_allclose(t[..., 1], base.n_hat[..., 0], atol=1e-13)
    np.testing.assert_allclose(t[..., 2], base.n_hat[..., 2], atol=1e-13)


def test_uint16_decoding_matches_metres():
    """uint16 depth is raw * depth_scale metres, 0 = invalid."""
    rng = np.random.default_rng(5)
    raw = rng.integers(400, 6000, size=(20, 24)).astype(np.uint16)
    raw[5, 7] = 0
    K = (200.0, 210.0, 11.5, 9.5)
    a = oracle.forward(raw, K, alpha=1, depth_scale=0.001, stat_mode=oracle.STAT_RAW, tau=BIG)
    b = oracle.forward(raw.astype(np.float64) * 0.001, K, alpha=1, stat_mode=oracle.STAT_RAW, tau=BIG)
    np.testing.assert_array_equal(a.valid, b.valid)
    np.testing.assert_allclose(a.n_raw, b.n_raw, rtol=0, atol=0)
    assert not a.valid[5, 7] and not a.valid[5, 8] and not a.valid[4, 7]
    c = oracle.forward(raw, K, alpha=1, depth_scale=0.002, stat_mode=oracle.STAT_RAW, tau=BIG)
    v = a.valid.astype(bool)
    np.testing.assert_allclose(c.r[v], 4 * a.r[v], rtol=1e-14)


# --------------------------------------------- border, holes, degenerate maps

@pytest.mark.parametrize("alpha", [1, 2, 4])
def test_invalid_depth_and_border_brute_force(alpha):
    """A pixel is valid iff its 5-point stencil is inside the image and every
    stencil depth is a positive finite number (readings C3, C4)."""
    rng = np.random.default_rng(alpha)
    H, W = 23, 29
    D = rng.uniform(1.0, 1.2, size=(H, W)).astype(np.float32)
    bad_vals = [0.0, -1.0, np.nan, np.inf, -np.inf]
    for i in range(12):
        D[rng.integers(0, H), rng.integers(0, W)] = bad_vals[i % len(bad_vals)]
    K = (300.0, 300.0, 14.0, 11.0)
    res = oracle.forward(D, K, alpha=alpha, tau=BIG)
    ok = np.isfinite(D) & (D > 0)
    expect = np.zeros((H, W), bool)
    for y in range(H):
        for x in range(W):
            pts = [(y, x), (y, x + alpha), (y + alpha, x), (y, x - alpha), (y - alpha, x)]
            expect[y, x] = all(0 <= r < H and 0 <= c < W and ok[r, c] for r, c in pts)
    np.testing.assert_array_equal(res.valid.astype(bool), expect)
    assert (res.n_hat[~expect] == 0).all()


@pytest.mark.parametrize("shape", [(0, 0), (1, 1), (1, 7), (4, 4), (5, 3)])
def test_degenerate_sizes(shape):
    """Maps with H or W < 2 alpha + 1 have no valid pixel; empty maps are fine."""
    H, W = shape
    D = np.ones((H, W), np.float32)
    res = oracle.forward(D, (100.0, 100.0, 0.0, 0.0), alpha=2, tau=BIG)
    assert res.valid.sum() == 0


# ------------------------------------------------------------- step edges

def _step_map(H, W, K, edge, where, za, zb, tilt=0.0):
    """Two planes joined at a column (edge='col') or row (edge='row') step."""
    R = rays(H, W, K)
    na = unit([math.sin(tilt), 0.0, math.cos(tilt)])
    nb = unit([0.0, math.sin(tilt), math.cos(tilt)])
    Da = za / (R @ na) * na[2]
    Db = zb / (R @ nb) * nb[2]
    D = Da.copy()
    if edge == "col":
        D[:, where:] = Db[:, where:]
    else:
        D[where:, :] = Db[where:, :]
    return D


@pytest.mark.parametrize("edge", ["col", "row"])
@pytest.mark.parametrize("alpha", [1, 2, 3])
@pytest.mark.parametrize("tilt", [0.0, 0.5])
def test_step_edge_mask_equals_brute_force(edge, alpha, tilt):
    """Section 3.2: r (and the secant statistic) is large exactly where the
    stencil straddles a depth step. With tau between the flat and step values the
    mask equals the brute-force label 'stencil straddles the edge'."""
    H, W = 40, 48
    K = (525.0, 525.0, 23.5, 19.5)
    where = 21
    D = _step_map(H, W, K, edge, where, 1.0, 1.5, tilt)
    inner = border_mask(H, W, alpha)
    label = np.zeros((H, W), bool)  # True = stencil straddles the step
    for y in range(H):
        for x in range(W):
            if edge == "col":
                label[y, x] = (x - alpha < where) != (x + alpha < where)
            else:
                label[y, x] = (y - alpha < where) != (y + alpha < where)
    sec = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_SECANT, tau=12.0)
    np.testing.assert_array_equal(sec.valid.astype(bool), inner & ~label)
    # RAW: tau between the flat value alpha^2 z^2/(fx fy) (z up to 1.5 m, plus the
    # tilt) and the step value.
    flat = alpha ** 2 * 1.5 ** 2 / (K[0] * K[1])
    raw = oracle.forward(D, K, alpha=alpha, stat_mode=oracle.STAT_RAW, tau=3.0 * flat)
    np.testing.assert_array_equal(raw.valid.astype(bool), inner & ~label)
    assert (raw.n_hat[label] == 0).all()


# -------------------------------------------------------------- gradient

def test_vjp_closed_form_fronto_parallel():
    """On a fronto-parallel plane at depth z, d(n_hat_x)/d(d2) = -fx/(2 alpha z)
    and d(n_hat_y)/d(d3) = -fy/(2 alpha z) (derived from Eq. 4-6 and the
    derivative of a normalisation); d(n_hat)/d(d1) = 0."""
    H, W, z, a = 15, 17, 1.7, 2
    K = (410.0, 370.0, 7.3, 6.9)
    D = np.full((H, W), z)
    res = oracle.forward(D, K, alpha=a, tau=BIG)
    p = (7, 8)  # (row, col)
    for comp, q, expect in ((0, (7, 8 + a), -K[0] / (2 * a * z)),
                            (1, (7 + a, 8), -K[1] / (2 * a * z)),
                            (0, (7, 8), 0.0), (1, (7, 8), 0.0), (2, (7, 8), 0.0)):
        g = np.zeros((H, W, 3))
        g[p[0], p[1], comp] = 1.0
        grad = oracle.vjp(D, K, g, res.valid, alpha=a)
        assert grad[q] == pytest.approx(expect, rel=1e-12, abs=1e-12)


def test_vjp_against_central_differences():
    """Complex-step VJP vs central finite differences (h = 1e-4 m, FP64) of the
    forward oracle on random pixels of a noisy scene, mask held fixed."""
    d, K = scenes.random_frame(21, 96, 72, kind="f64", holes=False, clip_range=False)
    D = d.numpy()
    H, W = D.shape
    alpha = 2
    base = oracle.forward(D, K, alpha=alpha, tau=BIG)
    rng = np.random.default_rng(3)
    g = rng.normal(size=(H, W, 3)) * base.valid[..., None]
    grad = oracle.vjp(D, K, g, base.valid, alpha=alpha)
    h = 1e-4
    v = base.valid.astype(bool)
    qs = list(zip(rng.integers(alpha, H - alpha, 40), rng.integers(alpha, W - alpha, 40)))
    for (y, x) in qs:
        def L(step):
            Dq = D.copy()
            Dq[y, x] += step
            f = oracle.forward(Dq, K, alpha=alpha, tau=BIG)
            assert (f.valid[v] == 1).all()
            # Only the pixels whose stencil holds (y, x) change.
            rows = slice(max(0, y - alpha), y + alpha + 1)
            cols = slice(max(0, x - alpha), x + alpha + 1)
            return float((f.n_hat[rows, cols] * g[rows, cols]).sum())
        # Fourth-order central difference: the second-order one has a truncation
        # error near 1e-5 relative here (third derivative ~ (f/(alpha z))^3).
        fd = (8 * (L(h) - L(-h)) - (L(2 * h) - L(-2 * h))) / (12 * h)
        assert grad[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(grad).max())


def test_vjp_crop_matches_full():
    d, K = scenes.random_frame(22, 64, 48, kind="f32", holes=False, clip_range=False)
    D = d.numpy()
    res = oracle.forward(D, K, alpha=2, tau=BIG)
    g = np.random.default_rng(0).normal(size=(48, 64, 3))
    full = oracle.vjp(D, K, g, res.valid, alpha=2)
    crop = oracle.vjp(D, K, g, res.valid, alpha=2, crop=(10, 20, 16, 24), nthreads=3)
    np.testing.assert_array_equal(crop, full[10:26, 20:44])


def test_threads_do_not_change_results(scene_f64):
    D, K = scene_f64
    a = oracle.forward(D, K, alpha=2, nthreads=1)
    b = oracle.forward(D, K, alpha=2, nthreads=5)
    np.testing.assert_array_equal(a.n_hat, b.n_hat)
    np.testing.assert_array_equal(a.valid, b.valid)
