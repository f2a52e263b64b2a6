"""The arctangent polynomial of the evaluation kernels (nrm_eval.cu) is the
one its generator (csrc/atan_fit.py) fits: the coefficients in the source
equal a fresh fit to float32 precision, the fit's error over [0, 1] is below
4e-8 rad and its float32 Horner evaluation below 1.2e-7 rad, and the octant
reconstruction written the kernel's way in float32 reproduces numpy's atan2
(signed zeros included) to 3e-7 rad. CPU only."""
import importlib.util
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_08241_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("atan_fit", os.path.join(CSRC, "atan_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _source_coefficients():
    src = open(os.path.join(CSRC, "nrm_eval.cu")).read()
    body = src[src.index("float atan2_fit("):src.index("float r = t * p;")]
    lines = [ln for ln in body.splitlines() if re.match(r"\s*(float )?p = ", ln)]
    lits = [re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", ln)[-1] for ln in lines]
    # Horner order in the source: highest power first.
    return [float(x) for x in lits][::-1]


def test_source_coefficients_are_the_fit():
    fit = _fit_module()
    c, err = fit.fit()
    src = _source_coefficients()
    assert len(src) == len(c) == 8
    np.testing.assert_allclose(np.float32(src), np.float32(c), rtol=2e-7, atol=1e-9)
    assert err < 4e-8
    assert fit.f32_horner_error(c) < 1.2e-7


def _atan2_kernel_way(y, x, c):
    f = np.float32
    y, x = f(y), f(x)
    ax, ay = abs(x), abs(y)
    hi, lo = max(ax, ay), min(ax, ay)
    t = f(lo * f(f(1.0) / max(hi, f(1.17549435e-38))))
    s = f(t * t)
    p = f(c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = f(p * s + f(c[k]))
    r = f(t * p)
    if ay > ax:
        r = f(f(math.pi / 2) - r)
    if np.signbit(x):
        r = f(f(math.pi) - r)
    return float(np.copysign(r, y))


def test_octant_reconstruction_matches_atan2():
    c = _source_coefficients()
    rng = np.random.default_rng(7)
    pts = list(rng.normal(size=(4000, 2))) + [(0.0, 0.0), (-0.0, 0.0), (0.0, -0.0), (-0.0, -0.0), (1.0, -0.0),
                                               (-1.0, 0.0), (-1.0, -0.0), (1.0, 1.0), (-1.0, 1.0), (1e-30, -1.0)]
    for x, y in pts:
        xf, yf = float(np.float32(x)), float(np.float32(y))
        got = _atan2_kernel_way(yf, xf, c)
        ref = math.atan2(yf, xf)
        assert abs(got - ref) <= 3e-7, (x, y, got, ref)
        if ref == 0.0:
            assert math.copysign(1.0, got) == math.copysign(1.0, ref), (x, y)
