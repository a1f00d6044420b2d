"""The paper's protocol, modelled step by step (oracle/protosim.py), against its
own lemmas and the Figure 2(b) example, and against the C oracle (CPU only)."""
import os

import numpy as np
import pytest

from oracle import oracle, protosim
from paper_2006_07478_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig2b():
    data, signals, expect = [], [], None
    with open(os.path.join(GOLDEN, "fig2b_credit.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "data":
                data = tok[1:]
            elif tok[0] == "signal":
                signals.append((tok[1], int(tok[2])))
            elif tok[0] == "expect":
                expect = " ".join(tok[1:])
    return data, signals, expect


def _fmt(trace):
    out = []
    for t in trace:
        out.append("[" + " ".join(t) + "]" if isinstance(t, list) else t)
    return " ".join(out)


def test_fig2b_receiver_rules():
    data, signals, expect = _read_fig2b()
    assert _fmt(protosim.receiver_trace(data, signals, W=8)) == expect
    # ensembles narrower than the credit split the data but keep the signal positions
    assert _fmt(protosim.receiver_trace(data, signals, W=1)) == "[d1] s1 [d2] [d3] s2"


def test_sender_rules():
    e = protosim.Edge(cap_q=8, cap_s=4)
    e.push_item((10, 0, None))
    e.push_item((11, 0, None))
    e.push_signal("E", 0)          # rule 1: S empty -> credit = |Q| = 2
    e.push_signal("B", 1)          # rule 2: nothing emitted since -> 0
    e.push_item((12, 1, None))
    e.push_signal("E", 1)          # rule 2: one item since the last signal
    assert [s[2] for s in e.s] == [2, 0, 1]
    e.q.popleft()                  # receiver drains an item: rule 1 uses the live |Q|
    e2 = protosim.Edge(cap_q=8, cap_s=4)
    e2.push_item((1, 0, None))
    e2.push_item((2, 0, None))
    e2.push_item((3, 0, None))
    e2.emitted = 0                 # an earlier signal was emitted and consumed already
    e2.q.popleft()
    e2.push_signal("E", 0)
    assert e2.s[0][2] == 2


def _random_stream(rng, R, max_len, load):
    L = rng.integers(0, max_len + 1, R)
    if load:
        n = int(L.sum())
        return wl.make_stream(L, elements=rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32),
                              ctx=rng.integers(0, 1 << 32, R, dtype=np.uint64).astype(np.uint32),
                              parents=rng.integers(0, 1 << 32, R, dtype=np.uint64).astype(np.uint32))
    return wl.make_stream(L, parents=rng.integers(0, 1 << 32, R, dtype=np.uint64).astype(np.uint32))


PIPES = [
    wl.pipeline_hash_filter_map(),
    [("enum_load",), ("filter_hash_ctx", 1, 2147483648), ("filter_hash_ctx", 2, 3000000000),
     ("aggregate",)],
    [("enum_load",), ("filter_weight_lt", 0x5EED), ("aggregate",)],
    [("enum_hash",), ("expand", 3, 77), ("filter_mod", 3, 1), ("aggregate",)],
    [("enum_load",), ("expand", 2, 5), ("map_mul", 7, 1), ("expand", 2, 9), ("aggregate",)],
]


@pytest.mark.parametrize("strategy", ["signal", "tag"])
@pytest.mark.parametrize("pi", range(len(PIPES)))
def test_protosim_equals_oracle_random_schedules(strategy, pi):
    pipe = PIPES[pi]
    rng = np.random.default_rng(100 + pi)
    load = pipe[0][0] == "enum_load"
    for trial in range(6):
        s = _random_stream(rng, int(rng.integers(0, 12)), int(rng.integers(0, 9)), load)
        W = int(rng.choice([1, 2, 3, 4]))
        k = max([protosim.max_fanout(x) for x in pipe[1:-1]] + [1])
        cap_q = W * k + int(rng.integers(0, 4))
        sim = protosim.Sim(pipe, s, W=W, cap_q=cap_q, cap_s=int(rng.integers(2, 5)),
                           K=int(rng.integers(1, 4)), n_proc=int(rng.integers(1, 4)),
                           strategy=strategy, seed=trial).run()
        assert not sim.violations, sim.violations[:3]
        assert sim.edge_logs_match()                       # Lemma 1: precise delivery
        assert all(c == 1 for c in sim.result_writes)      # one aggregate per region
        got = sim.aggregates()
        want = oracle.run(pipe, s)
        for key in ("count", "sum", "min"):
            assert np.array_equal(got[key], want[key]), (key, trial)


def test_exhaustive_tiny_length_sequences():
    """Every length sequence with R <= 3, L <= 4, for W in {1,2,4} and tight queues."""
    import itertools
    pipe = [("enum_load",), ("filter_mod", 2, 1), ("aggregate",)]
    cases = 0
    for R in range(0, 4):
        for L in itertools.product(range(5), repeat=R):
            n = sum(L)
            s = wl.make_stream(np.array(L, dtype=np.uint32), elements=np.arange(1, n + 1, dtype=np.uint32))
            want = oracle.run(pipe, s)
            for W in (1, 2, 4):
                for cap_q in (W, W + 1):
                    sim = protosim.Sim(pipe, s, W=W, cap_q=cap_q, cap_s=2, K=1, seed=R * 7 + W).run()
                    assert not sim.violations and sim.edge_logs_match()
                    got = sim.aggregates()
                    for key in ("count", "sum", "min"):
                        assert np.array_equal(got[key], want[key])
                    cases += 1
    assert cases > 500


def test_signal_ensembles_respect_region_bound():
    """With signals, stage 1 fires at least sum_r ceil(L_r / W) ensembles (no
    ensemble spans a region boundary); tags can do it in ceil(N / W)."""
    rng = np.random.default_rng(3)
    L = rng.integers(1, 10, 30)
    s = wl.make_stream(L, elements=np.arange(int(L.sum()), dtype=np.uint32))
    pipe = [("enum_load",), ("filter_mod", 1, 0), ("aggregate",)]
    W = 4
    sig = protosim.Sim(pipe, s, W=W, cap_q=64, cap_s=64, K=30, strategy="signal", seed=1).run()
    lower = int(np.sum((L + W - 1) // W))
    assert len(sig.ensemble_sizes(1)) >= lower
    assert sum(sig.ensemble_sizes(1)) == int(L.sum())      # item conservation
    tag = protosim.Sim(pipe, s, W=W, cap_q=64, cap_s=64, K=30, strategy="tag", seed=1).run()
    assert sum(tag.ensemble_sizes(1)) == int(L.sum())
    assert len(tag.ensemble_sizes(1)) < lower


def test_termination_and_empty_queues_on_many_seeds():
    rng = np.random.default_rng(9)
    pipe = PIPES[3]
    for seed in range(30):
        s = _random_stream(rng, 6, 5, False)
        sim = protosim.Sim(pipe, s, W=2, cap_q=6, cap_s=2, K=2, n_proc=2, seed=seed).run()
        assert not sim.violations
        assert sim.steps < 100000
