"""Coefficients of the arctangent polynomial in nrm_eval.cu.

atan(t) on 0 <= t <= 1 is approximated by t * (c0 + c1 s + ... + c7 s^7),
s = t^2, with the coefficients chosen to minimise the largest absolute error
(Lawson's iteratively reweighted least squares on a dense Chebyshev grid,
which converges to the minimax fit). Run it to print the coefficients as
float32 literals and the error of the fit and of its float32 Horner
evaluation (about 4e-8 and 1.1e-7 rad)."""
import numpy as np


def fit(n=8, iters=30, points=20001):
    t = 0.5 - 0.5 * np.cos(np.linspace(0.0, np.pi, points))
    s = t * t
    A = t[:, None] * s[:, None] ** np.arange(n)[None, :]
    y = np.arctan(t)
    w = np.ones_like(t)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y)
        w = w * (e + 1e-30)
        w /= w.sum()
    return c, float(np.abs(A @ c - y).max())


def f32_horner_error(c, points=200001):
    t = np.linspace(0.0, 1.0, points).astype(np.float32)
    s = t * t
    p = np.float32(c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p * s + np.float32(c[k])).astype(np.float32)
    r = (t * p).astype(np.float32)
    return float(np.abs(r.astype(np.float64) - np.arctan(t.astype(np.float64))).max())


if __name__ == "__main__":
    c, e = fit()
    print("fit error %.3g, float32 evaluation error %.3g" % (e, f32_horner_error(c)))
    print(", ".join("%.9ef" % np.float32(x) for x in c))
