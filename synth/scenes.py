"""Seeded synthetic depth maps for tests and benchmarks.

This module generates INPUTS only. It ray-casts simple 3-D primitives (planes,
rectangular patches, spheres, cylinders, oriented boxes) through a pinhole
camera and returns z-depth maps with Kinect-style noise, millimetre
quantisation and dropout holes. It contains none of the normal-estimation
arithmetic, so both the oracle tests and the GPU tests may use it.

Camera frame: x right, y down, z forward. Pixel (col, row) looks along the ray
(u, v, 1) with u = (col - cx)/fx and v = (row - cy)/fy, so the ray parameter t
of a hit IS its z-depth.

Everything is float64 torch arithmetic on the device given (CPU in tests, the
GPU in the benchmark, where generating 64 full-HD frames on the host would take
minutes). Scene parameters come from a numpy ``Generator`` seeded with the frame
seed; per-pixel noise and dropout come from a ``torch.Generator`` on the target
device seeded the same way, so a frame is deterministic given (seed, device).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

# The five frame sizes of the uneven-batch workload and their draw weights.
SIZE_MIX = ((320, 240), (640, 480), (1280, 720), (1920, 1080), (4096, 3072))
SIZE_WEIGHTS = (0.30, 0.30, 0.20, 0.15, 0.05)

KINECT_NOISE = 0.0012   # sigma = KINECT_NOISE * z^2 (metres)
RANGE = (0.4, 6.0)      # valid sensor range (metres); outside -> 0


def intrinsics_for(W: int, H: int, f_ratio: float = 0.82):
    """Pinhole intrinsics (fx, fy, cx, cy) with fx = fy = f_ratio * W, centred."""
    f = f_ratio * W
    return (f, f, (W - 1) / 2.0, (H - 1) / 2.0)


CFG1_K = (525.0, 525.0, 319.5, 239.5)


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], np.float64)


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], np.float64)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], np.float64)


# ---------------------------------------------------------------- primitives
# Each primitive returns the ray parameter t (= z-depth) of its nearest hit for
# rays (u, v, 1), or +inf where the ray misses. ``bound`` gives a conservative
# bounding sphere (centre, radius) used to restrict work to a screen rectangle.

@dataclass
class Plane:
    normal: np.ndarray      # n0
    offset: float           # n0 . X = offset

    bound = None

    def hit(self, u, v):
        n = self.normal
        den = n[0] * u + n[1] * v + n[2]
        t = self.offset / den
        return torch.where((den.abs() > 1e-12) & (t > 0), t, torch.full_like(t, math.inf))

    def normal_at(self, X):
        return torch.as_tensor(self.normal, dtype=X.dtype, device=X.device).expand_as(X)


@dataclass
class Patch:
    centre: np.ndarray
    e1: np.ndarray          # unit in-plane axes
    e2: np.ndarray
    h1: float               # half extents
    h2: float

    @property
    def bound(self):
        return self.centre, math.hypot(self.h1, self.h2)

    def hit(self, u, v):
        n = np.cross(self.e1, self.e2)
        den = n[0] * u + n[1] * v + n[2]
        safe = torch.where(den.abs() > 1e-12, den, torch.ones_like(den))
        t = float(n @ self.centre) / safe
        X = (t * u - self.centre[0], t * v - self.centre[1], t - self.centre[2])
        a = X[0] * self.e1[0] + X[1] * self.e1[1] + X[2] * self.e1[2]
        b = X[0] * self.e2[0] + X[1] * self.e2[1] + X[2] * self.e2[2]
        ok = (den.abs() > 1e-12) & (t > 0) & (a.abs() <= self.h1) & (b.abs() <= self.h2)
        return torch.where(ok, t, torch.full_like(t, math.inf))

    def normal_at(self, X):
        n = np.cross(self.e1, self.e2)
        return torch.as_tensor(n, dtype=X.dtype, device=X.device).expand_as(X)


@dataclass
class Sphere:
    centre: np.ndarray
    radius: float

    @property
    def bound(self):
        return self.centre, self.radius

    def hit(self, u, v):
        C = self.centre
        a = u * u + v * v + 1.0
        b = C[0] * u + C[1] * v + C[2]          # ray . C
        c = float(C @ C) - self.radius ** 2
        disc = b * b - a * c
        sq = torch.sqrt(torch.clamp(disc, min=0.0))
        t0 = (b - sq) / a
        t1 = (b + sq) / a
        t = torch.where(t0 > 0, t0, t1)
        return torch.where((disc >= 0) & (t > 0), t, torch.full_like(t, math.inf))

    def normal_at(self, X):
        return (X - torch.as_tensor(self.centre, dtype=X.dtype, device=X.device)) / self.radius


@dataclass
class Cylinder:
    centre: np.ndarray
    axis: np.ndarray        # unit
    radius: float
    half_len: float

    @property
    def bound(self):
        return self.centre, math.hypot(self.radius, self.half_len)

    def hit(self, u, v):
        C, A, R, L = self.centre, self.axis, self.radius, self.half_len
        inf = math.inf
        # Ray X(t) = t d with d = (u, v, 1); w = X - C.
        dA = u * A[0] + v * A[1] + A[2]
        cA = float(C @ A)
        # Side: |(t d - C) - ((t d - C).A) A|^2 = R^2
        dd = u * u + v * v + 1.0
        dC = u * C[0] + v * C[1] + C[2]
        qa = dd - dA * dA
        qb = dC - dA * cA                       # half of the linear coefficient (negated)
        qc = float(C @ C) - cA * cA - R * R
        disc = qb * qb - qa * qc
        sq = torch.sqrt(torch.clamp(disc, min=0.0))
        safe_a = torch.where(qa.abs() > 1e-15, qa, torch.ones_like(qa))
        best = torch.full_like(u, inf)
        for sgn in (-1.0, 1.0):
            t = (qb + sgn * sq) / safe_a
            h = t * dA - cA
            ok = (disc >= 0) & (qa.abs() > 1e-15) & (t > 0) & (h.abs() <= L)
            best = torch.where(ok & (t < best), t, best)
        # Caps: planes A . X = cA +- L, inside radius.
        safe_d = torch.where(dA.abs() > 1e-15, dA, torch.ones_like(dA))
        for sgn in (-1.0, 1.0):
            t = (cA + sgn * L) / safe_d
            X0 = t * u - C[0]
            X1 = t * v - C[1]
            X2 = t - C[2]
            along = X0 * A[0] + X1 * A[1] + X2 * A[2]
            rad2 = X0 * X0 + X1 * X1 + X2 * X2 - along * along
            ok = (dA.abs() > 1e-15) & (t > 0) & (rad2 <= R * R)
            best = torch.where(ok & (t < best), t, best)
        return best

    def normal_at(self, X):
        # Side: the radial direction; caps: +-axis. A point is on a cap when its
        # height along the axis is closer to +-half_len than its radius is to R.
        A = torch.as_tensor(self.axis, dtype=X.dtype, device=X.device)
        w = X - torch.as_tensor(self.centre, dtype=X.dtype, device=X.device)
        h = (w * A).sum(-1, keepdim=True)
        radial = w - h * A
        r = radial.norm(dim=-1, keepdim=True)
        cap = (h.abs() - self.half_len).abs() < (r - self.radius).abs()
        side = radial / r.clamp(min=1e-300)
        return torch.where(cap, torch.sign(h) * A, side)


@dataclass
class Box:
    centre: np.ndarray
    rot: np.ndarray         # columns = box axes in camera frame
    half: np.ndarray        # half extents along the box axes

    @property
    def bound(self):
        return self.centre, float(np.linalg.norm(self.half))

    def hit(self, u, v):
        # Slab test in the box frame: origin o = R^T (0 - C), direction R^T d.
        R, C, e = self.rot, self.centre, self.half
        o = -(R.T @ C)
        tnear = torch.full_like(u, -math.inf)
        tfar = torch.full_like(u, math.inf)
        for k in range(3):
            dk = R[0, k] * u + R[1, k] * v + R[2, k]
            small = dk.abs() < 1e-15
            safe = torch.where(small, torch.ones_like(dk), dk)
            ta = (-e[k] - o[k]) / safe
            tb = (e[k] - o[k]) / safe
            lo = torch.minimum(ta, tb)
            hi = torch.maximum(ta, tb)
            inside = abs(o[k]) <= e[k]
            lo = torch.where(small, torch.full_like(lo, -math.inf if inside else math.inf), lo)
            hi = torch.where(small, torch.full_like(hi, math.inf if inside else -math.inf), hi)
            tnear = torch.maximum(tnear, lo)
            tfar = torch.minimum(tfar, hi)
        ok = (tnear <= tfar) & (tfar > 0)
        t = torch.where(tnear > 0, tnear, tfar)
        return torch.where(ok, t, torch.full_like(t, math.inf))

    def normal_at(self, X):
        # The face whose slab the point is closest to leaving: largest |p_k| / e_k
        # in the box frame.
        R = torch.as_tensor(self.rot, dtype=X.dtype, device=X.device)
        p = (X - torch.as_tensor(self.centre, dtype=X.dtype, device=X.device)) @ R
        e = torch.as_tensor(self.half, dtype=X.dtype, device=X.device)
        k = (p.abs() / e).argmax(dim=-1, keepdim=True)
        sgn = torch.sign(torch.gather(p, -1, k))
        return sgn * R.T[k.squeeze(-1)]


@dataclass
class Scene:
    prims: list = field(default_factory=list)


def _screen_rect(bound, K, W, H):
    """Conservative pixel rectangle [c0, c1) x [r0, r1) covering a bounding sphere."""
    if bound is None:
        return 0, W, 0, H
    C, rb = bound
    zmin, zmax = C[2] - rb, C[2] + rb
    if zmax <= 0:
        return 0, 0, 0, 0
    if zmin < 0.05:
        return 0, W, 0, H
    fx, fy, cx, cy = K
    us = [(C[0] - rb) / zmin, (C[0] - rb) / zmax, (C[0] + rb) / zmin, (C[0] + rb) / zmax]
    vs = [(C[1] - rb) / zmin, (C[1] - rb) / zmax, (C[1] + rb) / zmin, (C[1] + rb) / zmax]
    c0 = max(0, int(math.floor(min(us) * fx + cx)) - 1)
    c1 = min(W, int(math.ceil(max(us) * fx + cx)) + 2)
    r0 = max(0, int(math.floor(min(vs) * fy + cy)) - 1)
    r1 = min(H, int(math.ceil(max(vs) * fy + cy)) + 2)
    return c0, max(c0, c1), r0, max(r0, r1)


def cast(scene: Scene, W: int, H: int, K, device="cpu") -> torch.Tensor:
    """Nearest-hit z-depth (float64, H x W); +inf where every primitive misses."""
    fx, fy, cx, cy = K
    dev = torch.device(device)
    u_all = (torch.arange(W, dtype=torch.float64, device=dev) - cx) / fx
    v_all = (torch.arange(H, dtype=torch.float64, device=dev) - cy) / fy
    depth = torch.full((H, W), math.inf, dtype=torch.float64, device=dev)
    for p in scene.prims:
        c0, c1, r0, r1 = _screen_rect(p.bound, K, W, H)
        if c1 <= c0 or r1 <= r0:
            continue
        u = u_all[c0:c1].unsqueeze(0).expand(r1 - r0, c1 - c0)
        v = v_all[r0:r1].unsqueeze(1).expand(r1 - r0, c1 - c0)
        t = p.hit(u, v)
        sub = depth[r0:r1, c0:c1]
        torch.minimum(sub, t, out=sub)
    return depth


def cast_normals(scene: Scene, W: int, H: int, K, device="cpu"):
    """Nearest-hit z-depth (float64, H x W; +inf on a miss) and the exact
    surface normal of the primitive hit there (float64, H x W x 3, unit),
    oriented away from the camera (n . ray > 0, the convention of the
    estimated normals); zero on a miss. Scene geometry only: the analytic
    ground truth against which estimates are scored."""
    fx, fy, cx, cy = K
    dev = torch.device(device)
    u_all = (torch.arange(W, dtype=torch.float64, device=dev) - cx) / fx
    v_all = (torch.arange(H, dtype=torch.float64, device=dev) - cy) / fy
    depth = torch.full((H, W), math.inf, dtype=torch.float64, device=dev)
    normals = torch.zeros((H, W, 3), dtype=torch.float64, device=dev)
    for p in scene.prims:
        c0, c1, r0, r1 = _screen_rect(p.bound, K, W, H)
        if c1 <= c0 or r1 <= r0:
            continue
        u = u_all[c0:c1].unsqueeze(0).expand(r1 - r0, c1 - c0)
        v = v_all[r0:r1].unsqueeze(1).expand(r1 - r0, c1 - c0)
        t = p.hit(u, v)
        sub = depth[r0:r1, c0:c1]
        closer = t < sub
        if not bool(closer.any()):
            continue
        tt = torch.where(closer, t, torch.zeros_like(t))
        X = torch.stack([tt * u, tt * v, tt], -1)
        n = p.normal_at(X)
        ray = torch.stack([u, v, torch.ones_like(u)], -1)
        n = torch.where(((n * ray).sum(-1, keepdim=True) < 0), -n, n)
        nsub = normals[r0:r1, c0:c1]
        nsub[closer] = n[closer]
        sub[closer] = t[closer]
    return depth, normals


# ------------------------------------------------------------------ scenes

def cfg1_scene() -> Scene:
    """The 640x480 single-frame scene: a background plane at z = 3.5 m tilted
    20 deg about x, a radius-0.4 m sphere at (-0.35, 0, 1.8) and a 0.5 x 0.4 m
    patch at (0.45, 0.10, 1.2) tilted 30 deg about y."""
    n_bg = _rot_x(math.radians(20.0)) @ np.array([0.0, 0.0, 1.0])
    bg = Plane(n_bg, float(n_bg @ np.array([0.0, 0.0, 3.5])))
    sph = Sphere(np.array([-0.35, 0.0, 1.8]), 0.4)
    Ry = _rot_y(math.radians(30.0))
    patch = Patch(np.array([0.45, 0.10, 1.2]), Ry @ np.array([1.0, 0, 0]),
                  Ry @ np.array([0, 1.0, 0]), 0.25, 0.20)
    return Scene([bg, sph, patch])


def random_scene(rng: np.random.Generator, W: int, H: int, K, n_min=20, n_max=60) -> Scene:
    """Floor plane at y = +1.2 m, a back wall 4.5-6.5 m away (yawed up to 20 deg)
    and U{n_min..n_max} random boxes (axis-aligned or rotated), spheres
    (r 0.1-0.6 m) and cylinders (r 0.05-0.4 m, length 0.2-1.5 m) with centres at
    z in U(0.6, 5.5) m, placed so that each centre projects inside the image."""
    fx, fy, cx, cy = K
    prims = [Plane(np.array([0.0, 1.0, 0.0]), 1.2)]
    yaw = rng.uniform(-math.radians(20), math.radians(20))
    n_wall = _rot_y(yaw) @ np.array([0.0, 0.0, 1.0])
    prims.append(Plane(n_wall, float(n_wall @ np.array([0.0, 0.0, rng.uniform(4.5, 6.5)]))))
    count = int(rng.integers(n_min, n_max + 1))
    while len(prims) < count + 2:
        z = rng.uniform(0.6, 5.5)
        px, py = rng.uniform(0, W), rng.uniform(0, H)
        C = np.array([(px - cx) / fx * z, (py - cy) / fy * z, z])
        kind = rng.integers(0, 3)
        if kind == 0:
            half = rng.uniform(0.05, 0.5, size=3)
            if rng.random() < 0.5:
                R = np.eye(3)
            else:
                R = _rot_y(rng.uniform(0, 2 * math.pi)) @ _rot_x(rng.uniform(-0.8, 0.8))
            prim = Box(C, R, half)
        elif kind == 1:
            prim = Sphere(C, rng.uniform(0.1, 0.6))
        else:
            a = rng.normal(size=3)
            a /= np.linalg.norm(a)
            prim = Cylinder(C, a, rng.uniform(0.05, 0.4), rng.uniform(0.1, 0.75))
        # Keep every object beyond the sensor's near range: its bounding sphere
        # must stay at z >= 0.5 m; otherwise redraw.
        centre, rb = prim.bound
        if centre[2] - rb >= 0.5:
            prims.append(prim)
    return Scene(prims)


def _noise_gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def add_kinect_noise(depth: torch.Tensor, seed: int) -> torch.Tensor:
    """depth + N(0, (0.0012 z^2)^2) on finite pixels."""
    g = _noise_gen(seed, depth.device)
    z = torch.where(torch.isfinite(depth), depth, torch.zeros_like(depth))
    eps = torch.randn(depth.shape, generator=g, dtype=torch.float64, device=depth.device)
    return torch.where(torch.isfinite(depth), depth + KINECT_NOISE * z * z * eps, depth)


def cfg1_normals(device="cpu") -> torch.Tensor:
    """Exact surface normals of the 640x480 scene (H x W x 3 float64, oriented
    away from the camera; zero where no surface is hit)."""
    return cast_normals(cfg1_scene(), 640, 480, CFG1_K, device)[1]


def cfg1_depth(device="cpu", noise=True, seed=1) -> tuple[torch.Tensor, tuple]:
    """640 x 480 float32 depth (metres) of the single-frame scene and its K."""
    d = cast(cfg1_scene(), 640, 480, CFG1_K, device)
    if noise:
        d = add_kinect_noise(d, seed)
    d = torch.where(torch.isfinite(d), d, torch.zeros_like(d))
    return d.to(torch.float32), CFG1_K


def random_frame(seed: int, W: int, H: int, device="cpu", kind="u16",
                 noise=True, holes=True, dropout=0.02, clip_range=True):
    """One random-primitive frame and its intrinsics (fx = fy = 0.82 W).

    kind = "u16": millimetres, rounded, clamped to [1, 65535], 0 = invalid;
           "f32": metres, float32, 0 = invalid;
           "f64": metres, float64 (no quantisation).
    holes: i.i.d. dropout of ``dropout`` of the pixels to 0.
    clip_range: depth outside [0.4, 6] m becomes 0.
    """
    K = intrinsics_for(W, H)
    rng = np.random.default_rng(seed)
    d = cast(random_scene(rng, W, H, K), W, H, K, device)
    if noise:
        d = add_kinect_noise(d, seed + 7919)
    bad = ~torch.isfinite(d) | (d <= 0)
    if clip_range:
        bad |= (d < RANGE[0]) | (d > RANGE[1])
    if holes and dropout > 0:
        g = _noise_gen(seed + 104729, d.device)
        bad |= torch.rand(d.shape, generator=g, dtype=torch.float64, device=d.device) < dropout
    if kind == "u16":
        mm = torch.clamp(torch.round(d * 1000.0), 1.0, 65535.0)
        mm = torch.where(bad, torch.zeros_like(mm), mm)
        return mm.to(torch.int32).to(torch.uint16) if hasattr(torch, "uint16") else mm, K
    d = torch.where(bad, torch.zeros_like(d), d)
    if kind == "f32":
        return d.to(torch.float32), K
    if kind == "f64":
        return d, K
    raise ValueError(kind)


def size_mix(n: int, seed: int = 3):
    """n frame sizes (W, H) drawn from SIZE_MIX with SIZE_WEIGHTS."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(SIZE_MIX), size=n, p=np.asarray(SIZE_WEIGHTS))
    return [SIZE_MIX[i] for i in idx]


def unit_targets(n: int, H: int, W: int, seed: int = 4, device="cpu") -> torch.Tensor:
    """Target unit normals uniform on the sphere, (n, H, W, 3) float32."""
    g = _noise_gen(seed, device)
    t = torch.randn((n, H, W, 3), generator=g, dtype=torch.float64, device=torch.device(device))
    t = t / t.norm(dim=-1, keepdim=True)
    return t.to(torch.float32)


def u16_batch(n: int = 64, W: int = 1920, H: int = 1080, seed0: int = 1000, device="cpu"):
    """The full-HD uint16 batch: frame i uses seed seed0 + i. Returns [(depth, K)]."""
    return [random_frame(seed0 + i, W, H, device, kind="u16") for i in range(n)]


def mixed_batch(n: int = 256, seed: int = 3, device="cpu", kind="f32"):
    """The uneven batch: n sizes drawn from SIZE_MIX; frame i uses seed 3000 + i.
    Returns [(depth, K)]."""
    return [random_frame(3000 + i, W, H, device, kind=kind)
            for i, (W, H) in enumerate(size_mix(n, seed))]
