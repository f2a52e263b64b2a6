"""Failure reporting on the GPU without a fault: a kernel waits on a barrier
that nothing completes, with the same bounded waits every kernel here uses;
both wait flavours give up after their limit, report NRM_ERR_TIMEOUT through
the status word, and the context stays usable for ordinary work."""
import ctypes
import time

import pytest
import torch

import paper_2209_08241_gb300 as nrm
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("timeout_ns", [1_000_000, 20_000_000])
def test_bounded_waits_expire_and_report(timeout_ns):
    lib = nrm._lib.load()
    ms = ctypes.c_float(0.0)
    t = time.perf_counter()
    rc = lib.nrm_selftest_wait_expiry(timeout_ns, ctypes.byref(ms))
    wall = time.perf_counter() - t
    assert rc == nrm._lib.NRM_OK, lib.nrm_last_error()
    # The waits lasted at least their limit and ended well within a second.
    assert ms.value >= timeout_ns / 1e6 * 0.9
    assert wall < 1.0
    # The context is still usable.
    d, K = scenes.random_frame(2000, 320, 240, "cuda", kind="f32")
    est = nrm.NormalEstimator(K, 240, 320)
    n, m = est(d)
    est.sync_status()
    assert int(m.sum()) > 0


def test_selftest_rejects_out_of_range_limits():
    lib = nrm._lib.load()
    assert lib.nrm_selftest_wait_expiry(10, None) == nrm._lib.NRM_ERR_INVALID_ARG
    assert lib.nrm_selftest_wait_expiry(5_000_000_000, None) == nrm._lib.NRM_ERR_INVALID_ARG


def test_bounds_selftest():
    """In the checking build the range checks accept in-range and reject
    out-of-range addresses (formed, never dereferenced) and record
    NRM_ERR_BOUNDS; the ordinary build reports that it has no checks."""
    import ctypes
    import os
    from paper_2209_08241_gb300 import _lib
    lib = _lib.load()
    res = (ctypes.c_int * 8)()
    rc = lib.nrm_selftest_bounds(res)
    if os.environ.get("NRM_LIB_VARIANT", "") == "debug":
        assert rc == _lib.NRM_OK, lib.nrm_last_error()
        assert list(res)[:7] == [1, 1, 0, 0, 1, 0, 0]
        assert res[7] == _lib.NRM_ERR_BOUNDS
    else:
        assert rc == _lib.NRM_ERR_UNSUPPORTED
