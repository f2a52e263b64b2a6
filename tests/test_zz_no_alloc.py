"""nrm_estimate_batched_noalloc: the batched launch for callers that cannot
allocate device memory (programs with a fixed, reserved device memory budget,
or code whose device memory belongs to another allocator and which must not
call cudaMalloc / cudaFree). Its descriptors live in a static device array
inside the library instead of handle-owned memory.

This file is collected last on purpose. The test calls the entry point through
the C ABI twice in a row (the second call overwrites the first call's
descriptors in the shared static array) and checks each result against
nrm_estimate_batched on the same frames. It must pass both alone in a fresh
process and after the other tests.
"""
import ctypes

import pytest
import torch

import paper_2209_08241_gb300 as nrm
from paper_2209_08241_gb300 import _lib
from synth import scenes

pytestmark = pytest.mark.gpu


def _params(**kw):
    p = _lib.Params()
    _lib.load().nrm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_noalloc_matches_batched_on_two_calls_in_a_row():
    lib = _lib.load()
    dev = "cuda"
    batches = [
        [scenes.random_frame(700 + i, W, H, dev, kind=k)
         for i, (W, H, k) in enumerate([(640, 480, "f32"), (333, 197, "u16"), (1920, 1080, "u16")])],
        [scenes.random_frame(800 + i, W, H, dev, kind=k)
         for i, (W, H, k) in enumerate([(1280, 720, "u16"), (320, 240, "f32")])],
    ]
    stream = torch.cuda.current_stream()
    for out in ("f32", "f16", "oct16"):
        params = nrm.NormalParams(out_dtype=out)
        c_params = params.to_c(0)
        ref_est = nrm.BatchedEstimator(params)
        for batch in batches:
            ref = ref_est(batch)
            arr, outs = ref_est.make_frames(batch)  # fresh output tensors
            for nm, vm in outs:
                nm.fill_(7)
                vm.fill_(9)
            status = torch.zeros(1, dtype=torch.int32, device=dev)
            rc = lib.nrm_estimate_batched_noalloc(arr, len(batch), ctypes.byref(c_params),
                                                  status.data_ptr(), stream.cuda_stream)
            assert rc == 0, lib.nrm_last_error()
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            for (rn, rm), (nm, vm) in zip(ref, outs):
                assert torch.equal(nm, rn)
                assert torch.equal(vm, rm)
        ref_est.sync_status()


def test_noalloc_without_status_word_or_stream_matches_batched():
    """device_status = NULL (errors go to the status word inside the static
    array) and cuda_stream = NULL (the legacy default stream): a successful
    call still gives nrm_estimate_batched's results bit for bit."""
    lib = _lib.load()
    batch = [scenes.random_frame(900 + i, W, H, "cuda", kind=k)
             for i, (W, H, k) in enumerate([(640, 480, "u16"), (257, 131, "f32")])]
    ref_est = nrm.BatchedEstimator()
    torch.cuda.synchronize()
    ref = ref_est(batch, stream=None)
    arr, outs = ref_est.make_frames(batch)
    for nm, vm in outs:
        nm.fill_(3)
        vm.fill_(5)
    rc = lib.nrm_estimate_batched_noalloc(arr, len(batch), None, None, None)
    assert rc == 0, lib.nrm_last_error()
    assert lib.nrm_last_error() == b""
    torch.cuda.synchronize()
    for (rn, rm), (nm, vm) in zip(ref, outs):
        assert torch.equal(nm, rn)
        assert torch.equal(vm, rm)


def test_noalloc_refuses_a_capturing_stream_and_runs_afterwards():
    """A call on a stream under capture returns NRM_ERR_UNSUPPORTED and records
    nothing; an ordinary call afterwards succeeds and matches the batched call."""
    lib = _lib.load()
    batch = [scenes.random_frame(950, 320, 240, "cuda", kind="u16")]
    ref_est = nrm.BatchedEstimator()
    ref = ref_est(batch)
    arr, outs = ref_est.make_frames(batch)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        rc = lib.nrm_estimate_batched_noalloc(arr, 1, None, None, side.cuda_stream)
    assert rc == _lib.NRM_ERR_UNSUPPORTED
    assert b"stream capture" in lib.nrm_last_error()
    stream = torch.cuda.current_stream()
    rc = lib.nrm_estimate_batched_noalloc(arr, 1, None, None, stream.cuda_stream)
    assert rc == 0, lib.nrm_last_error()
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], ref[0][0]) and torch.equal(outs[0][1], ref[0][1])


def test_noalloc_rejects_oversized_batches_and_bad_params():
    lib = _lib.load()
    d, K = scenes.random_frame(5, 64, 48, "cuda", kind="f32")
    b = nrm.BatchedEstimator()
    arr, _ = b.make_frames([(d, K)] * (_lib.NRM_NOALLOC_MAX_FRAMES + 1))
    rc = lib.nrm_estimate_batched_noalloc(arr, _lib.NRM_NOALLOC_MAX_FRAMES + 1, None, None, None)
    assert rc == _lib.NRM_ERR_UNSUPPORTED
    assert b"NRM_NOALLOC_MAX_FRAMES" in lib.nrm_last_error()
    bad = _params(alpha=0)
    assert lib.nrm_estimate_batched_noalloc(arr, 1, ctypes.byref(bad), None, None) == _lib.NRM_ERR_UNSUPPORTED
    assert lib.nrm_estimate_batched_noalloc(arr, 0, None, None, None) == 0
