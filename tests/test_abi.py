"""The C ABI library builds, loads and exports every function include/nrm.h
declares; the ctypes structures match the C layouts; host-side validation
rejects bad arguments before any device work. No test here needs a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2209_08241_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nrm.h")


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"NRM_API\s+[\w\s\*]+?\b(nrm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("nrm_create", "nrm_estimate", "nrm_estimate_batched", "nrm_backward",
                     "nrm_destroy", "nrm_status_string", "nrm_last_error"):
        assert required in names


def test_library_exports_every_header_symbol():
    lib = _lib.load()
    for name in header_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib._build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (nrm_\w+)", out))
    assert exported == set(header_functions())


def test_binding_declares_every_header_symbol():
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == header_functions()


def test_struct_layouts_match_c(tmp_path):
    """Compile a probe against include/nrm.h and compare sizes and offsets."""
    src = tmp_path / "probe.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "nrm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(nrm_intrinsics), sizeof(nrm_params), sizeof(nrm_frame),
         sizeof(nrm_tile_config), sizeof(nrm_stats), sizeof(nrm_scales));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", offsetof(nrm_frame, depth), offsetof(nrm_frame, normals),
         offsetof(nrm_frame, valid), offsetof(nrm_frame, H), offsetof(nrm_frame, W),
         offsetof(nrm_frame, depth_pitch), offsetof(nrm_frame, out_pitch), offsetof(nrm_frame, K),
         offsetof(nrm_frame, in_dtype), offsetof(nrm_frame, points));
  printf("%zu %zu %zu\n", offsetof(nrm_stats, launches), offsetof(nrm_stats, kernel_ms),
         offsetof(nrm_stats, tiles));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", f"-I{os.path.dirname(HEADER)}", str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    assert sizes == [ctypes.sizeof(_lib.Intrinsics), ctypes.sizeof(_lib.Params), ctypes.sizeof(_lib.Frame),
                     ctypes.sizeof(_lib.TileConfig), ctypes.sizeof(_lib.Stats), ctypes.sizeof(_lib.Scales)]
    F = _lib.Frame
    offs = [int(v) for v in lines[1].split()]
    assert offs == [F.depth.offset, F.normals.offset, F.valid.offset, F.H.offset, F.W.offset,
                    F.depth_pitch.offset, F.out_pitch.offset, F.K.offset, F.in_dtype.offset, F.points.offset]
    S = _lib.Stats
    assert [int(v) for v in lines[2].split()] == [S.launches.offset, S.kernel_ms.offset, S.tiles.offset]


def test_default_params_and_status_strings():
    lib = _lib.load()
    p = _lib.Params()
    lib.nrm_default_params(ctypes.byref(p))
    assert (p.alpha, p.mask_mode, p.tau, p.in_dtype, p.out_dtype, p.orient_to_camera) == (2, 1, 12.0, 0, 0, 0)
    assert p.depth_scale == pytest.approx(0.001)
    for code, name in [(0, b"NRM_OK"), (1, b"NRM_ERR_INVALID_ARG"), (2, b"NRM_ERR_UNSUPPORTED"),
                       (5, b"NRM_ERR_TIMEOUT"), (6, b"NRM_ERR_NO_DEVICE")]:
        assert lib.nrm_status_string(code) == name
    assert lib.nrm_version().startswith(b"nrm")


def _create(lib, K=(525.0, 525.0, 319.5, 239.5), H=480, W=640, **kw):
    p = _lib.Params()
    lib.nrm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    rc = lib.nrm_create(ctypes.byref(_lib.Intrinsics(*K)) if K else None, H, W, ctypes.byref(p),
                        ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("kw,code", [
    ({"alpha": 0}, _lib.NRM_ERR_UNSUPPORTED),
    ({"alpha": 17}, _lib.NRM_ERR_UNSUPPORTED),
    ({"tau": -1.0}, _lib.NRM_ERR_INVALID_ARG),
    ({"tau": float("nan")}, _lib.NRM_ERR_INVALID_ARG),
    ({"mask_mode": 7}, _lib.NRM_ERR_INVALID_ARG),
    ({"depth_scale": 0.0}, _lib.NRM_ERR_INVALID_ARG),
    ({"in_dtype": 3}, _lib.NRM_ERR_INVALID_ARG),
    ({"out_dtype": 3}, _lib.NRM_ERR_INVALID_ARG),
])
def test_create_rejects_bad_params(kw, code):
    lib = _lib.load()
    rc, h = _create(lib, **kw)
    assert rc == code
    assert not h.value
    assert lib.nrm_last_error()


def test_create_rejects_bad_sizes_and_intrinsics():
    lib = _lib.load()
    assert _create(lib, H=-1)[0] == _lib.NRM_ERR_INVALID_ARG
    assert _create(lib, H=0, W=5)[0] == _lib.NRM_ERR_INVALID_ARG
    assert _create(lib, K=(0.0, 1.0, 0.0, 0.0))[0] == _lib.NRM_ERR_INVALID_ARG
    assert _create(lib, K=(-500.0, 500.0, 0.0, 0.0))[0] == _lib.NRM_ERR_INVALID_ARG
    assert _create(lib, K=(float("inf"), 1.0, 0.0, 0.0))[0] == _lib.NRM_ERR_INVALID_ARG
    assert _create(lib, K=None)[0] == _lib.NRM_ERR_INVALID_ARG


def test_null_handle_calls_fail_cleanly():
    lib = _lib.load()
    assert lib.nrm_estimate(None, None, None, None, None) == _lib.NRM_ERR_INVALID_ARG
    assert lib.nrm_estimate_batched(None, None, 0, None) == _lib.NRM_ERR_INVALID_ARG
    assert lib.nrm_backward(None, None, None, None, None, None) == _lib.NRM_ERR_INVALID_ARG
    assert lib.nrm_sync_status(None) == _lib.NRM_ERR_INVALID_ARG
    lib.nrm_destroy(None)


def test_no_device_is_reported_not_hidden():
    """Without a GPU, creating a handle fails loudly (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = _lib.load()
    rc, h = _create(lib)
    assert rc == _lib.NRM_ERR_NO_DEVICE
    assert not h.value


def test_binding_refuses_tensors_the_library_cannot_write():
    """The binding's tensor check (it runs before every call that passes a raw
    pointer): host tensors, another device, wrong shape, dtype or layout."""
    import torch

    import paper_2209_08241_gb300 as nrm

    dev = torch.device("cuda", 0)
    with pytest.raises(ValueError, match="CUDA tensor"):
        nrm._check_dense(torch.empty((2, 3)), (2, 3), torch.float32, dev, "x")
    with pytest.raises(ValueError, match="CUDA tensor"):
        nrm._check_cuda(torch.empty((2, 3), dtype=torch.uint8), "mask", dev)


def test_functional_handle_cache_is_bounded():
    """The handles the functional calls create are kept most-recently-used
    last and at most _CACHE_MAX of them."""
    from collections import OrderedDict

    import paper_2209_08241_gb300 as nrm

    cache = OrderedDict()
    made = []
    for i in range(nrm._CACHE_MAX + 5):
        nrm._cached(cache, i, lambda i=i: made.append(i) or f"h{i}")
    assert len(cache) == nrm._CACHE_MAX and list(cache)[0] == 5
    assert nrm._cached(cache, 5, lambda: "new") == "h5" and list(cache)[-1] == 5
    assert len(made) == nrm._CACHE_MAX + 5
