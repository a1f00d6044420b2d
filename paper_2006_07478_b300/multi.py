"""One process per GPU: how work is split across ranks, and the one reduction the
multi-GPU run needs.

Regions are independent (an aggregate is per region, nothing flows between regions), so
the path shards with no data-path collective: a rank takes whole streams, or a
contiguous range of one stream's regions, and computes those regions' outputs alone.
The only collective is on timing: the step time of a multi-GPU run is the slowest
rank's, and the items processed are summed over ranks.
"""
from __future__ import annotations

import numpy as np


def shard_streams(n_streams: int, world: int, rank: int) -> range:
    """Contiguous block of stream indices for `rank` (sizes differ by at most one)."""
    lo = n_streams * rank // world
    hi = n_streams * (rank + 1) // world
    return range(lo, hi)


def shard_regions(lengths: np.ndarray, world: int, rank: int, region_cost: int = 1) -> tuple:
    """Contiguous region range [lo, hi) of one stream for `rank`, balanced on
    region_cost * regions + elements (the same merge-path cost the work units use), so
    ranks get equal work whatever the length distribution.  Ranges of consecutive ranks
    meet exactly: together they cover every region once."""
    L = np.asarray(lengths, dtype=np.int64)
    R = int(L.shape[0])
    if R == 0:
        return 0, 0
    # cost of regions [0, r): c r + elements before r; a rank's range starts at the first
    # region whose prefix cost reaches its share of the total
    prefix = region_cost * np.arange(R + 1, dtype=np.int64) + np.concatenate([[0], np.cumsum(L)])
    total = int(prefix[-1])

    def start(k: int) -> int:
        if k <= 0:
            return 0
        if k >= world:
            return R
        target = (total * k) // world
        return int(np.searchsorted(prefix, target, side="left"))

    return start(rank), start(rank + 1)


def shard_stream(stream: dict, world: int, rank: int, region_cost: int = 1) -> dict:
    """The part of a host stream (numpy arrays) that `rank` runs: its contiguous region
    range from `shard_regions`, with the matching lengths or CSR offsets, context words,
    parent ids (the global region ordinal when the stream has none, so hashed elements are
    unchanged) and element slice.  Regions are independent, so the shards' per-region
    results, concatenated in rank order, are the whole stream's."""
    if stream.get("len") is not None:
        L = np.asarray(stream["len"], dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(L)])
    else:
        o = np.asarray(stream["offsets"], dtype=np.int64)
        off = o - o[0]
        L = np.diff(o)
    lo, hi = shard_regions(L, world, rank, region_cost)
    out = {"R": hi - lo, "len": None, "offsets": None, "parents": None, "elements": None, "ctx": None,
           "shard": (lo, hi)}
    if stream.get("len") is not None:
        out["len"] = np.ascontiguousarray(stream["len"][lo:hi])
    else:
        out["offsets"] = np.ascontiguousarray((off[lo:hi + 1] - off[lo]).astype(np.uint32))
    if stream.get("parents") is not None:
        out["parents"] = np.ascontiguousarray(stream["parents"][lo:hi])
    else:
        out["parents"] = np.arange(lo, hi, dtype=np.uint64).astype(np.uint32)
    if stream.get("ctx") is not None:
        out["ctx"] = np.ascontiguousarray(stream["ctx"][lo:hi])
    if stream.get("elements") is not None:
        out["elements"] = np.ascontiguousarray(stream["elements"][off[lo]:off[hi]])
    return out


def reduce_step(elapsed_ms: float, items: int, device=None) -> tuple:
    """(slowest rank's time, items over all ranks) by torch.distributed all-reduces;
    the identity when no process group is initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_ms), int(items)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([int(items)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())
