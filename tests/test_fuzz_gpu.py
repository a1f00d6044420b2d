"""Seeded random pipelines on the GPU vs the CPU oracle, bit-exact.

Each case draws a linear stage list (loaded or hashed enumeration; one to three element
stages among the modulus, context-hash and weight filters, the multiply-add map and the
expansion; an aggregate or an emit sink), a strategy, a boundary mode per edge, an ensemble
width and a unit shape, and a stream of geometric region lengths (empty regions included),
then compares every region's results (a random subset of count, sum and min) with oracle.run /
oracle.run_emit.  A drawn combination the library rejects at creation (an illegal mode
sequence, say) is drawn again; every case runs."""
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


def _stream(rng, hashed, want_offsets):
    mean = float(rng.choice([0.5, 2, 9, 40, 300]))
    R = int(rng.integers(50, 3000))
    L = rng.geometric(1.0 / (1.0 + mean), size=R).astype(np.int64) - 1   # support from 0
    L = np.minimum(L, 5000).astype(np.uint32)
    N = int(L.sum())
    parents = rng.integers(0, 1 << 32, size=R, dtype=np.uint64).astype(np.uint32)
    ctx = rng.integers(0, 1 << 32, size=R, dtype=np.uint64).astype(np.uint32)
    elements = None if hashed else rng.integers(0, 1 << 32, size=max(N, 1), dtype=np.uint64).astype(np.uint32)[:N]
    if want_offsets:
        off = np.concatenate(([0], np.cumsum(L.astype(np.int64)))).astype(np.uint32)
        return wl.make_stream(offsets=off, parents=parents, elements=elements, ctx=ctx)
    return wl.make_stream(L, parents=parents, elements=elements, ctx=ctx)


def _stage(rng, k):
    kind = rng.choice(["mod", "hctx", "weight", "map", "expand"])
    salt = int(rng.integers(1, 1 << 31))
    if kind == "mod":
        m = int(rng.choice([2, 3, 4, 7, 16]))
        return ("filter_mod", m, int(rng.integers(0, m)))
    if kind == "hctx":
        return ("filter_hash_ctx", salt, int(rng.integers(1 << 29, 1 << 32)))
    if kind == "weight":
        return ("filter_weight_lt", salt)
    if kind == "map":
        return ("map_mul", int(rng.integers(1, 1 << 32)), int(rng.integers(0, 1 << 32)))
    return ("expand", int(rng.integers(0, 4)), salt)


def _modes(rng, n_stages, stages):
    modes, tagged = {}, False
    for e in range(1, n_stages):
        if tagged:
            m = "tag"
        else:
            choices = ["signal", "tag"] + ([] if stages[e][0] == "expand" else ["lane"])
            m = str(rng.choice(choices))
        tagged = tagged or m == "tag"
        modes[e] = m
    return modes


def _draw(rng):
    hashed = bool(rng.random() < 0.3)
    emit = bool(rng.random() < 0.3)
    stages = [("enum_hash",) if hashed else ("enum_load",)]
    for k in range(int(rng.integers(1, 4))):
        stages.append(_stage(rng, k))
    stages.append(("emit",) if emit else ("aggregate",))
    strategy = str(rng.choice(["tag", "signal"]))
    opts = {"ensemble_width": int(rng.choice([64, 128, 256] if strategy == "tag" else [32, 64, 128]))}
    if rng.random() < 0.5:
        opts["regions_per_unit"] = int(rng.choice([16, 128, 512] if strategy == "signal" else [64, 1024, 8192]))
    if strategy == "signal" and rng.random() < 0.6:
        opts["boundary_modes"] = _modes(rng, len(stages), stages)
    if rng.random() < 0.5:
        # the rest of the option space (the library rejects what does not fit; redrawn)
        opts["region_cost"] = int(rng.choice([1, 2, 4, 16, 64]))
        opts["warps_per_block"] = int(rng.choice([0, 1, 2, 3, 4, 8]))
        opts["grid"] = int(rng.choice([0, 0, 1, 5, 37]))
        if strategy == "signal":
            opts["tiles_in_flight"] = int(rng.choice([0, 2, 4]))
            opts["tile_elements"] = int(rng.choice([128, 256, 1024]))
            opts["signal_capacity"] = int(rng.choice([4, 8, 32, 256]))
        if rng.random() < 0.5:
            opts["queue_capacity"] = int(rng.choice([256, 512, 1024, 2048]))
    return stages, strategy, opts, hashed, emit


@pytest.mark.parametrize("seed", range(96))
def test_random_pipeline_matches_oracle(rs, seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(50):
        stages, strategy, opts, hashed, emit = _draw(rng)
        try:
            rs.Pipeline(stages, strategy=strategy, **opts).close()
        except rs.RsError:
            continue   # a combination the library rejects: draw again
        break
    else:
        pytest.fail("no accepted combination drawn")
    s = _stream(rng, hashed, want_offsets=emit)
    case = (stages, strategy, opts)
    if emit:
        want = oracle.run_emit(stages, s)
        got, st = rs.run_stream(stages, s, strategy=strategy, **opts)
        assert st["device_status"] == 0, (case, st)
        assert np.array_equal(got["count"], want["count"]), case
        start = want["start"]
        for r in np.flatnonzero(want["count"]):
            a = np.sort(got["values"][start[r]:start[r] + int(want["count"][r])])
            b = np.sort(want["values"][start[r]:start[r] + int(want["count"][r])])
            assert np.array_equal(a, b), (case, r)
    else:
        # a random subset of the outputs (the kernels size and use per-parent minima only
        # when a stream asks for them)
        outputs = [("count", "sum", "min"), ("count", "sum"), ("count",), ("sum", "min")][int(rng.integers(0, 4))]
        want = oracle.run(stages, s)
        got, st = rs.run_stream(stages, s, strategy=strategy, outputs=outputs, **opts)
        assert st["device_status"] == 0, (case, st)
        for k in outputs:
            bad = np.flatnonzero(got[k] != want[k])
            assert bad.size == 0, (case, k, bad[:5])


@pytest.mark.parametrize("seed", range(48))
def test_random_region_sum_matches_oracle(rs, seed):
    """Enumeration straight into the sink (the region-sum pipeline, and its emit form):
    random region-length mixes from all-short to a few thousand elements, random unit
    shapes, grids and output subsets (the minimum among them takes the general window
    path), at the ensemble width the specialised kernels are compiled for and at others."""
    rng = np.random.default_rng(5000 + seed)
    emit = bool(rng.random() < 0.2)
    stages = [("enum_load",), ("emit",) if emit else ("aggregate",)]
    strategy = str(rng.choice(["tag", "signal"]))
    widths = [64, 128, 128, 128, 256] if strategy == "tag" else [32, 64, 128, 128, 128]
    opts = {"ensemble_width": int(rng.choice(widths))}
    if rng.random() < 0.6:
        opts["regions_per_unit"] = int(rng.choice([1, 16, 128, 512] if strategy == "signal" else [16, 64, 1024, 8192]))
        opts["region_cost"] = int(rng.choice([1, 2, 4, 16, 64]))
        opts["warps_per_block"] = int(rng.choice([0, 1, 2, 4, 8]))
        opts["grid"] = int(rng.choice([0, 0, 1, 5, 37]))
        if rng.random() < 0.3:
            opts["flags"] = rs.FLAG_UNBALANCED_UNITS
    mean = float(rng.choice([0.5, 3, 16, 127, 600, 2500]))
    R = int(rng.integers(20, max(40, int(2_000_000 / (mean + 1)))))
    R = min(R, 20000)
    L = rng.geometric(1.0 / (1.0 + mean), size=R).astype(np.int64) - 1
    if rng.random() < 0.3:
        L = np.full(R, int(rng.choice([1, 31, 128, 129, 1000])), dtype=np.int64)   # fixed sizes
    L = L.astype(np.uint32)
    N = int(L.sum())
    elements = rng.integers(0, 1 << 32, size=max(N, 1), dtype=np.uint64).astype(np.uint32)[:N]
    case = (stages, strategy, opts, mean, R)
    if emit:
        off = np.concatenate(([0], np.cumsum(L.astype(np.int64)))).astype(np.uint32)
        s = wl.make_stream(offsets=off, elements=elements)
        want = oracle.run_emit(stages, s)
        got, st = rs.run_stream(stages, s, strategy=strategy, **opts)
        assert st["device_status"] == 0, (case, st)
        assert np.array_equal(got["count"], want["count"]), case
        start = want["start"]
        for r in np.flatnonzero(want["count"])[:2000]:
            a = np.sort(got["values"][start[r]:start[r] + int(want["count"][r])])
            b = np.sort(want["values"][start[r]:start[r] + int(want["count"][r])])
            assert np.array_equal(a, b), (case, r)
        return
    s = wl.make_stream(L, elements=elements)
    outputs = [("count", "sum"), ("count", "sum"), ("sum",), ("count", "sum", "min"), ("count",)][int(rng.integers(0, 5))]
    want = oracle.run(stages, s)
    got, st = rs.run_stream(stages, s, strategy=strategy, outputs=outputs, **opts)
    assert st["device_status"] == 0, (case, st)
    for k in outputs:
        bad = np.flatnonzero(got[k] != want[k])
        assert bad.size == 0, (case, k, bad[:5])


def _draw_tree(rng):
    """A tree (Figure 1(b)): the enumeration feeds one element stage; below it two
    branches of zero to two element stages each end in an aggregate, forking at a random
    element stage of the trunk."""
    hashed = bool(rng.random() < 0.4)
    stages = [("enum_hash",) if hashed else ("enum_load",)]
    inputs = [0]
    trunk = [len(stages)]
    stages.append(_stage(rng, 0))
    inputs.append(0)
    for _ in range(int(rng.integers(0, 2))):
        inputs.append(len(stages) - 1)
        trunk.append(len(stages))
        stages.append(_stage(rng, 0))
    fork = int(rng.choice(trunk))
    for _ in range(2):
        prev = fork
        for _ in range(int(rng.integers(0, 3))):
            inputs.append(prev)
            prev = len(stages)
            stages.append(_stage(rng, 0))
        inputs.append(prev)
        stages.append(("aggregate",))
    modes, tagged = {}, set()
    for c in range(1, len(stages)):
        if inputs[c] in tagged and inputs[c] != 0:
            m = "tag"
        else:
            m = str(rng.choice(["signal", "tag"] + ([] if stages[c][0] == "expand" else ["lane"])))
        if m == "tag":
            tagged.add(c)
        modes[c] = m
    if rng.random() < 0.25:
        modes = {c: "signal" for c in range(1, len(stages))}
    return stages, inputs, modes, hashed


@pytest.mark.parametrize("seed", range(48))
def test_random_tree_matches_oracle(rs, seed):
    rng = np.random.default_rng(5000 + seed)
    for _ in range(50):
        stages, inputs, modes, hashed = _draw_tree(rng)
        w = int(rng.choice([32, 64, 128]))
        try:
            rs.Pipeline(stages, strategy="signal", inputs=inputs, boundary_modes=modes, ensemble_width=w).close()
        except rs.RsError:
            continue
        break
    else:
        pytest.fail("no accepted tree drawn")
    s = _stream(rng, hashed, want_offsets=False)
    outputs = [("count", "sum", "min"), ("count", "sum"), ("min",)][int(rng.integers(0, 3))]
    case = (stages, inputs, modes, w)
    want = oracle.run_tree(stages, inputs, s)
    got, st = rs.run_stream(stages, s, strategy="signal", inputs=inputs, boundary_modes=modes, ensemble_width=w,
                            outputs=outputs)
    assert st["device_status"] == 0, (case, st)
    for k in outputs:
        assert np.array_equal(got[k], want[0][k]), (case, k, 0)
        assert np.array_equal(got[k + "2"], want[1][k]), (case, k, 1)


@pytest.mark.parametrize("seed", range(32))
def test_random_pipeline_sliced_matches_oracle(rs, seed):
    """The same random linear pipelines (aggregate sinks) run a few work units per launch
    over resident per-stream state until done: the results equal the oracle's."""
    import torch
    rng = np.random.default_rng(9000 + seed)
    for _ in range(50):
        stages, strategy, opts, hashed, emit = _draw(rng)
        if emit:
            continue
        try:
            rs.Pipeline(stages, strategy=strategy, **opts).close()
        except rs.RsError:
            continue
        break
    else:
        pytest.fail("no accepted combination drawn")
    s = _stream(rng, hashed, want_offsets=bool(rng.random() < 0.5))
    budget = int(rng.integers(1, 5))
    outputs = ("count", "sum", "min")
    case = (stages, strategy, opts, budget)
    want = oracle.run(stages, s)
    p = rs.Pipeline(stages, strategy=strategy, **opts)
    dev = rs.to_device(s)
    out = p.submit(dev, outputs=outputs)
    for k in outputs:
        out[k].fill_(0x5A5A5A5A)
    nbytes, units = p.state_size(dev)
    state = torch.empty(max(256, nbytes) + 256, dtype=torch.uint8, device="cuda")
    state = state[(-state.data_ptr()) % 256:]
    begin = 0
    while begin < units:
        p.clear()
        p.submit(dev, out=out, state=state, unit_begin=begin, unit_count=budget)
        p.run()
        st = p.stats()
        assert st["device_status"] == 0, (case, st)
        begin += budget
    torch.cuda.synchronize()
    got = rs.results_to_numpy(out)
    for k in outputs:
        bad = np.flatnonzero(got[k] != want[k])
        assert bad.size == 0, (case, k, bad[:5])
    p.close()


@pytest.mark.parametrize("seed", range(16))
def test_random_pipeline_served_matches_oracle(rs, seed):
    """Random linear pipelines (aggregate sinks) served: a dozen random streams submitted to
    the continuous-batching server with a random slice budget, each result equal to the
    oracle's."""
    import time
    rng = np.random.default_rng(13000 + seed)
    for _ in range(50):
        stages, strategy, opts, hashed, emit = _draw(rng)
        opts.pop("boundary_modes", None)
        if emit:
            continue
        try:
            rs.Pipeline(stages, strategy=strategy, **opts).close()
        except rs.RsError:
            continue
        break
    else:
        pytest.fail("no accepted combination drawn")
    streams = [_stream(rng, hashed, want_offsets=False) for _ in range(12)]
    slice_units = int(rng.choice([0, 1, 4, 64]))
    srv = rs.Server(stages, arena_bytes=256 << 20, strategy=strategy, slice_units=slice_units, **opts)
    reqs = [rs.host_request(s) for s in streams]
    ids = [srv.submit(r) for r in reqs]
    done, t0 = [], time.time()
    while len(done) < len(ids):
        srv.progress()
        done += srv.poll()
        assert time.time() - t0 < 60.0, srv.stats()
    srv.close()
    for r, s in zip(reqs, streams):
        want = oracle.run(stages, s)
        got = rs.results_to_numpy({k: r[k] for k in ("count", "sum", "min")})
        for k in got:
            bad = np.flatnonzero(got[k] != want[k])
            assert bad.size == 0, (stages, strategy, opts, slice_units, k, bad[:5])


def _check_results(got, want, outputs, case):
    for k in outputs:
        bad = np.flatnonzero(got[k] != want[k])
        assert bad.size == 0, (case, k, bad[:5])


@pytest.mark.parametrize("seed", range(24))
def test_random_batch_graph_replay_and_noalloc_match_oracle(rs, seed):
    """Random linear pipelines (aggregate or emit sinks) over two to six random streams in one
    launch: the plain run, two replays of a captured CUDA graph (on a side stream, outputs
    clobbered before) and the workspace-free entry point all give the oracle's results for
    every stream."""
    import torch
    rng = np.random.default_rng(17000 + seed)
    for _ in range(50):
        stages, strategy, opts, hashed, emit = _draw(rng)
        try:
            rs.Pipeline(stages, strategy=strategy, **opts).close()
        except rs.RsError:
            continue
        break
    else:
        pytest.fail("no accepted combination drawn")
    streams = [_stream(rng, hashed, want_offsets=emit or bool(rng.random() < 0.5))
               for _ in range(int(rng.integers(2, 7)))]
    outputs = ("count", "values") if emit else ("count", "sum", "min")
    case = (stages, strategy, opts, len(streams))
    wants = [oracle.run_emit(stages, s) if emit else oracle.run(stages, s) for s in streams]
    p = rs.Pipeline(stages, strategy=strategy, **opts)
    outs = [p.submit(rs.to_device(s), outputs=outputs) for s in streams]

    def clobber():
        for o in outs:
            for k in outputs:
                o[k].fill_(0x5A5A5A5A)

    def verify():
        torch.cuda.synchronize()
        for o, want in zip(outs, wants):
            got = rs.results_to_numpy(o)
            if not emit:
                _check_results(got, want, outputs, case)
                continue
            assert np.array_equal(got["count"], want["count"]), case
            start = want["start"]
            for r in np.flatnonzero(want["count"]):
                a = np.sort(got["values"][start[r]:start[r] + int(want["count"][r])])
                b = np.sort(want["values"][start[r]:start[r] + int(want["count"][r])])
                assert np.array_equal(a, b), (case, r)

    clobber()
    p.run()
    assert p.stats()["device_status"] == 0, case
    verify()
    clobber()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        p.graph_capture()
        p.graph_launch()
        p.graph_launch()
    side.synchronize()
    verify()
    p.graph_release()
    clobber()
    try:
        p.run_noalloc()
    except rs.RsError as e:
        # beyond the fixed scratch array (16 MiB, 64 streams): refused, nothing ran
        assert e.status == rs.RS_ERR_CAPACITY, (case, e)
    else:
        verify()
    p.close()
