"""Sliced runs over resident per-stream state (bounded launches) on the GPU, bit-exact
against the CPU oracle.

A stream's units run a slice at a time: its planning state (unit records, planner words,
merge slots) stays in a device buffer of its own between launches, and the region
results fold across launches.  One unit per launch, repeated until the stream is done,
must give exactly the one-shot result (and the oracle's); several streams may advance
in the same launch by different amounts, and new ones may join later."""
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


def _sliced(rs, p, dev, out, budget):
    """Run `dev` on pipeline p in slices of `budget` units until it is done; returns the
    number of launches."""
    import torch
    nbytes, units = p.state_size(dev)
    state = torch.empty(max(256, nbytes) + 256, dtype=torch.uint8, device="cuda")
    state = state[(-state.data_ptr()) % 256:]
    launches, begin = 0, 0
    while begin < units:
        p.clear()
        p.submit(dev, out=out, state=state, unit_begin=begin, unit_count=budget)
        p.run()
        st = p.stats()
        assert st["device_status"] == 0, st
        begin += budget
        launches += 1
    torch.cuda.synchronize()
    return launches


CASES = [
    ("cascade", lambda: wl.cascade_stream(n_total=1 << 17, mean=32, seed=7), ("count", "sum")),
    ("cascade1", lambda: wl.cascade_stream(n_total=1 << 16, mean=1, seed=7), ("count", "sum")),
    ("hashed", lambda: wl.hashed_uniform_stream(3000, 64, 2), ("count", "sum", "min")),
    ("graph", lambda: wl.graph_stream(V=1 << 11, E=1 << 16, cap=1 << 12, seed=7), ("count", "min")),
]


def _pipe(name):
    return {"cascade": wl.pipeline_cascade(), "cascade1": wl.pipeline_cascade(),
            "hashed": wl.pipeline_hash_filter_map(), "graph": wl.pipeline_graph_edges()}[name]


@pytest.mark.parametrize("strategy", ["tag", "signal"])
@pytest.mark.parametrize("budget", [1, 3])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_one_unit_per_launch_equals_one_shot(rs, ci, budget, strategy):
    name, make, outputs = CASES[ci]
    s = make()
    pipe = _pipe(name)
    want = oracle.run(pipe, s)
    p = rs.Pipeline(pipe, strategy=strategy)
    dev = rs.to_device(s)
    out = p.submit(dev, outputs=outputs)      # allocates the outputs
    for k in outputs:
        out[k].fill_(0x5A5A5A5A)
    n = _sliced(rs, p, dev, out, budget)
    assert n >= 2
    got = rs.results_to_numpy(out)
    for k in outputs:
        bad = np.flatnonzero(got[k] != want[k])
        assert bad.size == 0, (name, k, bad[:5])
    p.close()


def test_streams_advance_together_and_join_late(rs):
    """Three streams share every launch, each with its own budget; a fourth joins after
    the others have started; all end exactly as the oracle says."""
    import torch
    pipe = wl.pipeline_cascade()
    streams = [wl.cascade_stream(n_total=n, mean=m, seed=sd) for n, m, sd in
               ((1 << 17, 16, 1), (1 << 15, 4, 2), (1 << 18, 300, 3), (1 << 16, 40, 4))]
    p = rs.Pipeline(pipe, strategy="tag")
    devs = [rs.to_device(s) for s in streams]
    outs, states, units, nxt = [], [], [], []
    for d in devs:
        o = p.submit(d, outputs=("count", "sum"))
        o["count"].fill_(-1)
        outs.append(o)
        b, u = p.state_size(d)
        t = torch.empty(b + 512, dtype=torch.uint8, device="cuda")
        states.append(t[(-t.data_ptr()) % 256:])
        units.append(u)
        nxt.append(0)
    budgets = [1, 2, 5, 3]
    step = 0
    while any(nxt[i] < units[i] for i in range(4)):
        p.clear()
        for i in range(4):
            if i == 3 and step < 3:
                continue                      # joins at the fourth launch
            if nxt[i] < units[i]:
                p.submit(devs[i], out=outs[i], state=states[i], unit_begin=nxt[i], unit_count=budgets[i])
                nxt[i] += budgets[i]
        p.run()
        assert p.stats()["device_status"] == 0
        step += 1
    torch.cuda.synchronize()
    for s, o in zip(streams, outs):
        want = oracle.run(pipe, s)
        got = rs.results_to_numpy(o)
        for k in ("count", "sum"):
            assert np.array_equal(got[k], want[k]), k
    p.close()


def test_state_too_small_is_refused(rs):
    import torch
    s = wl.cascade_stream(n_total=1 << 16, mean=8, seed=5)
    p = rs.Pipeline(wl.pipeline_cascade(), strategy="tag")
    dev = rs.to_device(s)
    out = p.submit(dev, outputs=("count", "sum"))
    b, u = p.state_size(dev)
    assert b > 256 and u > 1
    small = torch.empty(b - 256, dtype=torch.uint8, device="cuda")
    small = small[(-small.data_ptr()) % 256:]
    p.clear()
    p.submit(dev, out=out, state=small, unit_begin=0, unit_count=1)
    with pytest.raises(rs.RsError) as e:
        p.run()
    assert e.value.status == rs.RS_ERR_CAPACITY
    with pytest.raises(rs.RsError):          # a slice is not captured in a graph
        p.graph_capture()
    p.close()
