"""Autotune cache file (JSON: key -> [tile_x, tile_y, threads, stages,
ctas_per_sm]) read and written through the C ABI: round trip, replacement,
several keys, absent and malformed entries, rejected keys. CPU tests (these
calls need no GPU); the GPU test checks that a tuned geometry recorded by one
handle is picked up by nrm_create for the next handle with the same key."""
import json
import os

import pytest
import torch

import paper_2209_08241_gb300 as nrm
from paper_2209_08241_gb300 import _lib


def test_round_trip_and_replace(tmp_path):
    path = str(tmp_path / "tune.json")
    assert nrm.autotune_cache_get(path, "k") is None          # no file yet
    nrm.autotune_cache_put(path, "NVIDIA GB300|sm152|in2|out1|a2|handle0x0", 128, 32, 256, 2, 3)
    nrm.autotune_cache_put(path, "other|key", 64, 64, 256, 3, 0)
    assert nrm.autotune_cache_get(path, "NVIDIA GB300|sm152|in2|out1|a2|handle0x0") == {
        "tile_x": 128, "tile_y": 32, "threads": 256, "stages": 2, "ctas_per_sm": 3}
    nrm.autotune_cache_put(path, "other|key", 128, 64, 512, 4, 1)  # replaces
    assert nrm.autotune_cache_get(path, "other|key")["threads"] == 512
    data = json.load(open(path))                               # the file is plain JSON
    assert data == {"NVIDIA GB300|sm152|in2|out1|a2|handle0x0": [128, 32, 256, 2, 3],
                    "other|key": [128, 64, 512, 4, 1]}
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]  # written to a temporary, then renamed
    assert nrm.autotune_cache_get(path, "missing") is None


def test_malformed_and_rejected(tmp_path):
    path = str(tmp_path / "bad.json")
    with open(path, "w") as f:
        f.write('{"k": [1, 2, 3]}\n')                          # too few fields
    assert nrm.autotune_cache_get(path, "k") is None
    lib = _lib.load()
    assert b"malformed" in lib.nrm_last_error()
    with pytest.raises(_lib.NrmError):
        nrm.autotune_cache_put(path, 'quote"key', 128, 16, 256, 3)
    with pytest.raises(_lib.NrmError):
        nrm.autotune_cache_put(str(tmp_path / "no_dir" / "x.json"), "k", 128, 16, 256, 3)
    c = _lib.TileConfig()
    assert lib.nrm_autotune_cache_get(None, b"k", ctypes_ref(c)) == _lib.NRM_ERR_INVALID_ARG


def ctypes_ref(c):
    import ctypes
    return ctypes.byref(c)


def _writer(path, tag, n):
    import paper_2209_08241_gb300 as nrm_
    for i in range(n):
        nrm_.autotune_cache_put(path, f"{tag}|{i}", 128, 16, 256, 2 + i % 3, i % 4)


def test_concurrent_writers_leave_a_valid_file(tmp_path):
    """One process per GPU may tune and record at the same time: every
    writer uses its own temporary file and an atomic rename, so the file is
    always a complete JSON object (entries may be lost to a later rename, but
    never mixed)."""
    import multiprocessing as mp
    path = str(tmp_path / "shared.json")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_writer, args=(path, f"w{k}", 40)) for k in range(4)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    data = json.load(open(path))
    assert data and all(len(v) == 5 for v in data.values())
    assert all(k.split("|")[0] in {"w0", "w1", "w2", "w3"} for k in data)
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]


def test_process_wide_path_can_be_set_and_cleared(tmp_path):
    nrm.set_autotune_cache(str(tmp_path / "t.json"))
    nrm.set_autotune_cache(None)


@pytest.mark.gpu
def test_tuned_geometry_is_picked_up_by_the_next_handle(tmp_path):
    from synth import scenes
    path = str(tmp_path / "tune.json")
    nrm.set_autotune_cache(path)
    try:
        params = nrm.NormalParams(out_dtype="f16")
        a = nrm.BatchedEstimator(params)
        key = a.autotune_key()
        assert key.endswith("|out1|a2|handle0x0") and "|sm" in key
        # Seed the handle's key with a non-default geometry, then tune a batch:
        # the sweep overwrites it with the winner, which the next handle loads.
        items = [scenes.random_frame(60 + i, 640, 480, "cuda", kind="u16") for i in range(4)]
        best = a.autotune(items)
        rec = nrm.autotune_cache_get(path, key)
        assert rec == best
        b = nrm.BatchedEstimator(params)                       # no autotune call
        assert b.config() == best
        # A second autotune of the same batch loads the batch key without timing.
        c = nrm.BatchedEstimator(params)
        assert c.autotune(items) == best
        # An entry that does not name a compiled geometry leaves the default.
        nrm.autotune_cache_put(path, key, 96, 16, 256, 3)
        d = nrm.BatchedEstimator(params)
        assert d.config()["tile_x"] == 128 and d.config()["tile_y"] == 16
        for e in (a, b, c, d):
            e.sync_status()
    finally:
        nrm.set_autotune_cache(None)
