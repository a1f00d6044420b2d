"""The multi-GPU path's host logic on CPU, two ranks over gloo: how regions and streams
are split across ranks (no data-path collective: each rank's shard computes its regions'
outputs alone) and the step reduction (slowest rank's time, items summed)."""
import os
import socket

import numpy as np
import pytest

from paper_2006_07478_b300 import multi
from paper_2006_07478_b300 import workloads as wl


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = wl.cascade_stream(n_total=1 << 15, mean=9, seed=5)
        lo, hi = multi.shard_regions(s["len"], world, rank)
        off = np.concatenate([[0], np.cumsum(s["len"].astype(np.int64))]).astype(np.uint32)
        # the rank's shard is a stream of its own: offsets into the same element array
        shard = wl.make_stream(offsets=off[lo:hi + 1], elements=s["elements"], ctx=s["ctx"][lo:hi])
        got = oracle.run(wl.pipeline_cascade(), shard)
        ms, items = multi.reduce_step(10.0 + rank, int(off[hi] - off[lo]))
        q.put((rank, lo, hi, got["count"].tolist(), got["sum"].tolist(), ms, items,
               list(multi.shard_streams(5, world, rank))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_exactly_and_reduce():
    import torch.multiprocessing as mp
    from oracle import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = wl.cascade_stream(n_total=1 << 15, mean=9, seed=5)
    want = oracle.run(wl.pipeline_cascade(), s)
    (r0, lo0, hi0, c0, s0, ms0, n0, st0), (r1, lo1, hi1, c1, s1, ms1, n1, st1) = res
    assert (lo0, hi1) == (0, s["R"]) and hi0 == lo1          # the shards partition the regions
    assert np.array_equal(np.array(c0 + c1, dtype=np.uint32), want["count"])
    assert np.array_equal(np.array(s0 + s1, dtype=np.uint64), want["sum"])
    assert ms0 == ms1 == 11.0                                   # the slowest rank's time
    assert n0 == n1 == 1 << 15                                  # items over both ranks
    assert st0 + st1 == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_region_shards_balance_merge_path_cost(world):
    rng = np.random.default_rng(world)
    L = rng.geometric(1 / 50, 20_000).astype(np.int64) - 1
    L[100] = 500_000                                            # one hub region
    cuts = [multi.shard_regions(L, world, k) for k in range(world)]
    assert cuts[0][0] == 0 and cuts[-1][1] == len(L)
    assert all(cuts[k][1] == cuts[k + 1][0] for k in range(world - 1))
    cost = np.array([(hi - lo) + L[lo:hi].sum() for lo, hi in cuts])
    # balanced up to the one region a cut cannot split
    assert cost.max() - cost.min() <= 2 * (L.max() + 1)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_stream_shards_concatenate_to_the_whole(world):
    """Each rank's shard (regions, lengths or offsets, context, parent ids, elements) run by
    the oracle; the results, concatenated in rank order, are the whole stream's."""
    from oracle import oracle
    cases = [(wl.pipeline_cascade(), wl.cascade_stream(n_total=1 << 16, mean=6, seed=3)),
             (wl.pipeline_graph_edges(), wl.graph_stream(V=4000, E=40000, cap=3000, seed=7)),
             (wl.pipeline_hash_filter_map(), wl.hashed_uniform_stream(3000, 64, 4))]
    for pipe, s in cases:
        whole = oracle.run(pipe, s)
        parts = [oracle.run(pipe, multi.shard_stream(s, world, r)) for r in range(world)]
        for k in ("count", "sum", "min"):
            assert np.array_equal(np.concatenate([p[k] for p in parts]), whole[k]), k
