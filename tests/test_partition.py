"""Pixel-balanced frame split of a batch over ranks (no collective on the data
path): every frame is assigned exactly once, the split is deterministic, and
per-rank pixel counts differ by at most the largest frame. The world-size-2
case runs as two gloo ranks on CPU, each computing its own share from the
batch description alone; the check gathers the shares afterwards."""
import multiprocessing as mp
import os
import random
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2209_08241_gb300 import partition  # noqa: E402

SIZES = [(320, 240), (640, 480), (1280, 720), (1920, 1080), (4096, 3072)]
WEIGHTS = [0.3, 0.3, 0.2, 0.15, 0.05]


def uneven_mix(n, seed):
    rng = random.Random(seed)
    return [w * h for w, h in rng.choices(SIZES, weights=WEIGHTS, k=n)]


def check_split(px, parts):
    assigned = sorted(i for p in parts for i in p)
    assert assigned == list(range(len(px)))           # each frame exactly once
    for p in parts:
        assert p == sorted(p)
    loads = [sum(px[i] for i in p) for p in parts]
    if px:
        assert max(loads) - min(loads) <= max(px)      # balance bound
    return loads


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("seed", [3, 11, 2024])
def test_uneven_mix_split(world, seed):
    px = uneven_mix(256, seed)
    parts = partition.balance_frames(px, world)
    loads = check_split(px, parts)
    assert partition.balance_frames(px, world) == parts  # deterministic
    # With 256 mixed frames the shares are far tighter than the bound.
    assert max(loads) - min(loads) <= 4096 * 3072


def test_equal_frames_split_evenly():
    px = [1920 * 1080] * 64
    for world in (1, 2, 4, 8):
        parts = partition.balance_frames(px, world)
        check_split(px, parts)
        assert {len(p) for p in parts} == {64 // world}


def test_more_ranks_than_frames_and_empty_batches():
    parts = partition.balance_frames([5, 7], 4)
    check_split([5, 7], parts)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]
    assert partition.balance_frames([], 3) == [[], [], []]
    check_split([0, 0, 9], partition.balance_frames([0, 0, 9], 2))


def test_bad_arguments():
    with pytest.raises(ValueError):
        partition.balance_frames([1], 0)
    with pytest.raises(ValueError):
        partition.balance_frames([-1], 2)
    with pytest.raises(ValueError):
        partition.rank_frames([1], 2, 2)


def test_brute_force_optimum_on_small_batches():
    """The greedy split is within the largest frame of the best possible split
    (brute force over all assignments of 8 frames to 2 ranks)."""
    import itertools
    rng = random.Random(5)
    for _ in range(20):
        px = [rng.randint(1, 100) for _ in range(8)]
        parts = partition.balance_frames(px, 2)
        got = max(sum(px[i] for i in p) for p in parts)
        best = min(max(sum(x for x, a in zip(px, asg) if a == 0), sum(x for x, a in zip(px, asg) if a == 1))
                   for asg in itertools.product((0, 1), repeat=8))
        assert got - best <= max(px)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2209_08241_gb300 import partition as part
    dist.init_process_group("gloo", rank=rank, world_size=world)
    px = uneven_mix(256, 3)                # every rank knows the batch description
    mine = part.rank_frames(px, rank, world)  # no communication needed for the split
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)   # only to check the result
    dist.destroy_process_group()
    q.put((rank, gathered))


def test_split_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got[0] == got[1]                  # both ranks see the same split
    px = uneven_mix(256, 3)
    check_split(px, got[0])
    assert got[0] == partition.balance_frames(px, 2)
