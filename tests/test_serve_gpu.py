"""Serving form (continuous batching) on the GPU: every request's result equals the
oracle's, whether it ran in a mix with many others or alone, including when a small
arena forces requests to wait for memory.  Bit-exact (integer results)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2006_07478_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2006_07478_b300 import rs as _rs
    _rs.lib()
    return _rs


def _drain(srv, n, budget_s=60.0):
    import time
    done = []
    t0 = time.time()
    while len(done) < n:
        srv.progress()
        done += srv.poll()
        assert time.time() - t0 < budget_s, srv.stats()
    return done


def _check(rs, req, stream, pipe):
    want = oracle.run(pipe, stream)
    got = rs.results_to_numpy({k: req[k] for k in ("count", "sum", "min")})
    for k in got:
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("strategy", ["tag", "signal"])
def test_mix_equals_alone(rs, strategy):
    pipe = wl.pipeline_hash_filter_map()
    streams = wl.batched_streams(n_streams=40, median=2 ** 10, sigma=1.5, cap=1 << 14, seed=21)
    srv = rs.Server(pipe, arena_bytes=64 << 20, strategy=strategy)
    reqs = [rs.host_request(s) for s in streams]
    ids = [srv.submit(r) for r in reqs]
    done = _drain(srv, len(ids))
    assert sorted(done) == sorted(ids)
    st = srv.stats()
    assert st["completed"] == len(ids) and st["arena_live"] == 0
    assert st["per_array"] == 0                      # the arena had room for every gather
    for r, s in zip(reqs, streams):
        _check(rs, r, s, pipe)
    # the same stream alone in its own batch gives the same result
    alone = rs.host_request(streams[7])
    srv.submit(alone)
    _drain(srv, 1)
    for k in ("count", "sum", "min"):
        assert np.array_equal(alone[k].numpy(), reqs[7][k].numpy()), k
    srv.close()


def test_small_arena_admission_waits_for_memory(rs):
    """An arena that holds only a few requests at a time: later requests wait until
    earlier batches release their space, and all finish correctly."""
    pipe = wl.pipeline_cascade()
    streams = [wl.cascade_stream(n_total=1 << 15, mean=16, seed=30 + i) for i in range(24)]
    srv = rs.Server(pipe, arena_bytes=1 << 20, strategy="tag")
    reqs = [rs.host_request(s, outputs=("count", "sum")) for s in streams]
    ids = [srv.submit(r) for r in reqs]
    _drain(srv, len(ids))
    st = srv.stats()
    assert st["arena_peak"] <= 1 << 20 and st["batches"] > 1
    for r, s in zip(reqs, streams):
        want = oracle.run(pipe, s)
        got = rs.results_to_numpy({"count": r["count"], "sum": r["sum"]})
        for k in got:
            assert np.array_equal(got[k], want[k]), k
    srv.close()


def test_requests_arriving_during_a_batch_join_the_next(rs):
    import time
    pipe = wl.pipeline_hash_filter_map()
    streams = wl.batched_streams(n_streams=64, median=2 ** 12, sigma=1.0, cap=1 << 16, seed=5)
    srv = rs.Server(pipe, arena_bytes=256 << 20, strategy="tag", max_inflight=2)
    reqs = [rs.host_request(s) for s in streams]
    done = []
    for i, r in enumerate(reqs):
        srv.submit(r)
        if i % 8 == 7:
            srv.progress()
            done += srv.poll()
    done += _drain(srv, len(reqs) - len(done))
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["batches"] >= 2
    for r, s in zip(reqs, streams):
        _check(rs, r, s, pipe)
    srv.close()


def test_results_copied_per_array_when_the_arena_is_full(rs):
    """An arena sized so that requests fill it: launches find no room for the
    gathered-results region and copy each output array back on its own, with the
    oracle's results (the gathered path is checked in test_mix_equals_alone)."""
    pipe = wl.pipeline_hash_filter_map()
    streams = [wl.hashed_uniform_stream(4000, 64, 40 + i) for i in range(30)]
    reqs = [rs.host_request(s) for s in streams]
    srv = rs.Server(pipe, arena_bytes=192 << 10, strategy="tag", max_inflight=1)
    ids = [srv.submit(r) for r in reqs]
    _drain(srv, len(ids))
    st = srv.stats()
    assert st["completed"] == len(ids) and st["arena_live"] == 0
    assert st["per_array"] > 0, st
    for r, s in zip(reqs, streams):
        _check(rs, r, s, pipe)
    srv.close()


@pytest.mark.parametrize("slice_units", [1, 4, 0])
def test_mix_equals_alone_any_slice_budget(rs, slice_units):
    """Every slice budget (one unit per launch, a few, whole requests) gives each request
    the oracle's result, loaded streams with resident planning state included."""
    pipe = wl.pipeline_cascade()
    streams = [wl.cascade_stream(n_total=n, mean=m, seed=60 + i)
               for i, (n, m) in enumerate(((1 << 16, 8), (1 << 13, 1), (1 << 17, 300), (1 << 15, 30)))]
    srv = rs.Server(pipe, arena_bytes=64 << 20, strategy="tag", slice_units=slice_units)
    reqs = [rs.host_request(s, outputs=("count", "sum")) for s in streams]
    ids = [srv.submit(r) for r in reqs]
    _drain(srv, len(ids))
    for r, s in zip(reqs, streams):
        want = oracle.run(pipe, s)
        got = rs.results_to_numpy({"count": r["count"], "sum": r["sum"]})
        for k in got:
            assert np.array_equal(got[k], want[k]), (slice_units, k)
    assert srv.stats()["arena_live"] == 0
    srv.close()


def test_short_requests_are_not_held_back_by_a_long_one(rs):
    """Continuous batching over resident state: a long request (hundreds of work units)
    is running when short ones (one unit each) arrive; they join the next launches and
    all finish before it, each with the oracle's result."""
    pipe = wl.pipeline_hash_filter_map()
    big = wl.batched_streams(n_streams=1, median=2 ** 21, sigma=0.01, cap=1 << 22, seed=70)[0]
    small = wl.batched_streams(n_streams=24, median=2 ** 9, sigma=0.5, cap=1 << 11, seed=71)
    srv = rs.Server(pipe, arena_bytes=512 << 20, strategy="tag", slice_units=2, max_inflight=2)
    rb = rs.host_request(big)
    big_id = srv.submit(rb)
    srv.progress()                 # the long request starts
    rss = [rs.host_request(s) for s in small]
    small_ids = [srv.submit(r) for r in rss]
    order = _drain(srv, 1 + len(small_ids), budget_s=120.0)
    assert set(order) == set(small_ids) | {big_id}
    assert order.index(big_id) == len(order) - 1, order
    _check(rs, rb, big, pipe)
    for r, s in zip(rss, small):
        _check(rs, r, s, pipe)
    srv.close()

