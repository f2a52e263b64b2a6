"""Frame-sharded batches over several GPUs, one process per GPU.

The method works on each organised depth map on its own: every output pixel
depends only on the depths of its own frame (Section 3.1, Eq. 4-6), so a batch
spread over N GPUs needs no exchange between them. Each rank takes a subset of
the frames and runs one batched launch over it on its own GPU; nothing on the
data path is communicated. The subsets are chosen to balance the pixel counts,
because a frame's cost is proportional to its pixels and frames of one batch
may differ in size by a factor of 160 (320 x 240 up to 4096 x 3072).

The split is a pure function of the frame sizes and the number of ranks, so
every rank computes the same split from the batch description alone.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def balance_frames(pixels: Sequence[int], world_size: int) -> list[list[int]]:
    """Splits frames 0 .. len(pixels) - 1 over ``world_size`` ranks.

    Largest frames first (ties: lower index first), each to the rank with the
    fewest pixels so far (ties: lower rank). Returns, per rank, its frame
    indices in increasing order. Every frame goes to exactly one rank, and the
    pixel counts of any two ranks differ by at most the largest frame's count:
    when the rank that ends with the most pixels received its last frame, it
    had the fewest, so its final excess over any other rank is at most that
    frame's size.
    """
    if world_size < 1:
        raise ValueError("world_size must be at least 1")
    px = [int(p) for p in pixels]
    if any(p < 0 for p in px):
        raise ValueError("pixel counts must be non-negative")
    order = sorted(range(len(px)), key=lambda i: (-px[i], i))
    heap = [(0, r) for r in range(world_size)]  # (pixels so far, rank)
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + px[i], r))
    return [sorted(p) for p in parts]


def rank_frames(pixels: Sequence[int], rank: int, world_size: int) -> list[int]:
    """The frame indices of ``rank`` in ``balance_frames(pixels, world_size)``."""
    if not 0 <= rank < world_size:
        raise ValueError("rank out of range")
    return balance_frames(pixels, world_size)[rank]


def shard(items: Sequence, rank: int, world_size: int) -> list:
    """This rank's frames of a batch of (depth, K) items (depth: an H x W tensor)."""
    px = [int(d.shape[-2]) * int(d.shape[-1]) for d, _ in items]
    return [items[i] for i in rank_frames(px, rank, world_size)]
