"""The bench line's parity record (bench.py: parity_frame, new_parity,
finish_parity) counts what it claims to count: fed the FP64 oracle's own
result it passes; one planted mistake of each kind (a mask flip outside the
near-tau band, a normal turned by 3e-4 rad, a flipped normal, a masked pixel
with a nonzero normal, a mask byte other than 0/1) is counted and fails the
record. CPU only (the planted mistakes go into the checked arrays)."""
import importlib.util
import os

import numpy as np

import oracle
from synth import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _frame():
    d, K = scenes.random_frame(1000, 96, 64, "cpu", kind="u16")
    depth = d.numpy()
    ref = oracle.forward(depth, K, alpha=2, stat_mode=oracle.STAT_SECANT, tau=12.0, depth_scale=0.001, nthreads=2)
    n = np.zeros(depth.shape + (4,), np.float32)
    n[..., :3] = np.where(ref.valid[..., None] == 1, ref.n_hat, 0.0)
    return depth, K, n, ref.valid.astype(np.uint8).copy(), ref


def _record(b, n, v, depth, K, out="f32"):
    acc = b.new_parity(out, 1)
    b.parity_frame(n, v, depth, K, 0.001, 2, acc)
    return b.finish_parity(acc)


def _far_from_tau(ref, valid_value):
    with np.errstate(invalid="ignore"):
        far = np.isfinite(ref.stat) & (np.abs(ref.stat - 12.0) > 1e-3 * 12.0)
    ys, xs = np.nonzero(far & (ref.valid == valid_value))
    return int(ys[len(ys) // 2]), int(xs[len(xs) // 2])


def test_oracle_result_passes():
    b = _bench()
    depth, K, n, v, ref = _frame()
    r = _record(b, n, v, depth, K)
    assert r["pass"] and r["mask_mismatches_outside_band"] == 0 and r["max_angle_rad"] < 1e-6
    assert r["pixels"] == depth.size and r["valid_pixels_compared"] == int((ref.valid == 1).sum())


def test_each_planted_mistake_is_counted():
    b = _bench()
    depth, K, n0, v0, ref = _frame()
    # A mask flip away from tau.
    n, v = n0.copy(), v0.copy()
    y, x = _far_from_tau(ref, 1)
    v[y, x] = 0
    n[y, x] = 0.0
    r = _record(b, n, v, depth, K)
    assert r["mask_mismatches_outside_band"] == 1 and not r["pass"]
    # A normal turned by 3e-4 rad about an axis perpendicular to it.
    n, v = n0.copy(), v0.copy()
    y, x = _far_from_tau(ref, 1)
    a = ref.n_hat[y, x]
    p = np.cross(a, [0.0, 0.0, 1.0] if abs(a[2]) < 0.9 else [1.0, 0.0, 0.0])
    p /= np.linalg.norm(p)
    n[y, x, :3] = np.cos(3e-4) * a + np.sin(3e-4) * p
    r = _record(b, n, v, depth, K)
    assert abs(r["max_angle_rad"] - 3e-4) < 2e-6 and not r["pass"]
    # The same turn within the half-output tolerance passes there.
    assert _record(b, n, v, depth, K, out="f16")["pass"]
    # A flipped normal.
    n, v = n0.copy(), v0.copy()
    n[y, x, :3] = -n[y, x, :3]
    assert _record(b, n, v, depth, K)["max_angle_rad"] > 3.0
    # A masked pixel that kept a normal.
    n, v = n0.copy(), v0.copy()
    y, x = _far_from_tau(ref, 0)
    n[y, x, 2] = 1.0
    r = _record(b, n, v, depth, K)
    assert r["masked_pixels_not_zero"] == 1 and not r["pass"]
    # A mask byte that is neither 0 nor 1.
    n, v = n0.copy(), v0.copy()
    y, x = _far_from_tau(ref, 1)
    v[y, x] = 2
    r = _record(b, n, v, depth, K)
    assert r["mask_bytes_not_0_or_1"] == 1 and not r["pass"]
