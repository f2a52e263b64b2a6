"""The range-checking build (``build.py --debug``, ``-DNRM_DEBUG_CHECKS``) over the
edge-case inputs: in it every shared-memory access of the kernels and every
global access that depends on frame geometry is range-checked, and a failed
check skips the access, prints ``NRM_BOUNDS`` with the site and records
NRM_ERR_BOUNDS in the status word. This test builds that library, runs a set of
the GPU tests against it in a child process (the binding loads it when
NRM_LIB_VARIANT=debug), and requires them to pass, which includes every
status word reading NRM_OK and every guard band staying intact, with no
bounds report in the output. (It stands in for a memory checker, which this
GPU pool does not offer.)"""
import os
import subprocess
import sys

import pytest

from paper_2209_08241_gb300 import build as nbuild

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    "tests/test_gpu_canaries.py",
    "tests/test_gpu_forward.py::test_tiny_and_degenerate_maps",
    "tests/test_gpu_forward.py::test_special_depth_values",
    "tests/test_gpu_forward.py::test_alpha_limits",
    "tests/test_gpu_forward.py::test_u16_plain_parity_ragged",
    "tests/test_gpu_forward.py::test_unaligned_pitches_use_plain_loads_and_byte_stores",
    "tests/test_gpu_forward.py::test_mixed_size_batch_parity",
    "tests/test_gpu_forward.py::test_oct16_output_parity",
    "tests/test_gpu_backward.py::test_adjoint_matches_complex_step_oracle",
    "tests/test_gpu_backward.py::test_scaled_adjoint_equals_adjoint_of_scaled_gradient",
    "tests/test_gpu_multiscale.py::test_u16_ragged_with_holes",
    "tests/test_gpu_multiscale.py::test_batched_mixed_sizes_dtypes_and_intrinsics",
    "tests/test_gpu_plane_fit.py::test_u16_ragged_with_holes",
    "tests/test_gpu_plane_fit.py::test_tiny_frames",
    "tests/test_gpu_points.py::test_plain_points",
    "tests/test_gpu_evaluation.py::test_angle_mse_matches_oracle_and_is_deterministic",
    "tests/test_gpu_failure.py::test_bounds_selftest",
]


def test_checked_build_passes_the_edge_cases():
    lib = nbuild.build(debug=True)
    assert lib.endswith("libnrm_debug.so")
    env = dict(os.environ, NRM_LIB_VARIANT="debug")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", "-s", *SELECTION]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    text = out.stdout + out.stderr
    # The bounds self-test's planted rejections print "expected report"; any
    # other report is a real out-of-range index.
    bad = [ln for ln in text.splitlines() if "NRM_BOUNDS" in ln and "expected report" not in ln]
    assert not bad, "\n".join(bad)[:4000]
    assert sum("expected report" in ln for ln in text.splitlines()) == 4
    assert out.returncode == 0, text[-4000:]
    assert " passed" in text and " failed" not in text
