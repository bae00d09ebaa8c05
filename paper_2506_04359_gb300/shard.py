"""Sharding of independent bundle-adjustment windows across ranks (one GPU per rank).

Windows are independent problems (separate keyframes, landmarks and damping), so ranks
take disjoint subsets and solve them with no collective on the data path; results are
gathered once at the end.  A window's cost is estimated from its configuration before it
is generated: observations ~ landmarks x mean track length (linearisation, Schur), plus the
reduced-camera-system factorisation, whose dependent pivot chain grows with 6(K - 1).

Host logic only; the tests exercise it with `gloo` ranks on the CPU.
"""
from __future__ import annotations

import heapq


def window_cost(K: int, M: int, track_mean: float = 5.5) -> float:
    """Relative solve cost of one window: per-observation and per-pair work plus the
    factorisation's pivot chain (300 observation-equivalents per pivot)."""
    n_obs = 2.0 * M * track_mean                    # a stereo pair sees each tracked point twice
    n_c = 6 * max(K - 1, 0)
    return n_obs + 4.0 * M * track_mean + 300.0 * n_c


def partition(costs: list[float], world_size: int) -> list[list[int]]:
    """Balanced assignment of windows to ranks (longest processing time first: windows in
    decreasing cost, each to the least loaded rank; ties to the lower rank).  Returns, per
    rank, its window indices in increasing order.  Deterministic."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world_size)]
    heapq.heapify(heap)
    out: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(v) for v in out]


def gather(local: dict, world_size: int) -> dict:
    """All ranks' {window index: result} merged (torch.distributed all_gather_object on the
    current process group); with world_size 1 the local dict itself."""
    if world_size == 1:
        return dict(local)
    import torch.distributed as dist
    parts: list = [None] * world_size
    dist.all_gather_object(parts, local)
    merged: dict = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise ValueError(f"window {k} solved on two ranks")
            merged[k] = v
    return dict(sorted(merged.items()))
