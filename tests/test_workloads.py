"""Seeded workload generators: determinism, sizes and distribution shapes (CPU only)."""
import numpy as np

from paper_2006_07478_b300 import workloads as wl


def test_xorshift64_definition_and_lockstep_agree():
    # Marsaglia's (13, 7, 17) step, applied by hand to a few states
    seq = wl.xorshift64_sequence(1, 3)
    x = 1
    for v in seq:
        x ^= (x << 13) & wl.MASK64
        x ^= x >> 7
        x ^= (x << 17) & wl.MASK64
        assert int(v) == x
    st = np.array([1, 2, 3], dtype=np.uint64)
    wl.xorshift64_lockstep(st)
    assert [int(v) for v in st] == [int(wl.xorshift64_sequence(s, 1)[0]) for s in (1, 2, 3)]


def test_splitmix64_counter_matches_scalar_steps():
    seed = 12345
    vals = wl.splitmix64_counter(seed, 0, 4)
    state = seed
    for v in vals:
        assert int(v) == wl.splitmix64_scalar(state)
        state = (state + wl.GAMMA) & wl.MASK64


def test_hashed_uniform_shape():
    s = wl.hashed_uniform_stream()
    assert s["R"] == 10_000 and s["parents"] is None
    L = s["len"]
    assert L.min() >= 1 and L.max() <= 64
    assert abs(L.mean() - 32.5) < 1.0
    s2 = wl.hashed_uniform_stream()
    assert np.array_equal(L, s2["len"])


def test_geometric_lengths_total_and_mean():
    for mu in (1, 4, 32, 256):
        L = wl.geometric_lengths(1 << 20, mu, 7)
        assert int(L.astype(np.int64).sum()) == 1 << 20
        m = L[:-1].mean()
        assert abs(m - mu) < 6 * mu / np.sqrt(len(L)) + 0.05 * mu
        if mu == 1:
            assert abs((L == 0).mean() - 0.5) < 0.01


def test_graph_degrees_exact_and_capped():
    g = wl.graph_stream(V=1 << 12, E=1 << 16, cap=1 << 10, seed=7)
    deg = np.diff(g["offsets"].astype(np.int64))
    assert int(deg.sum()) == 1 << 16
    assert deg.max() <= 1 << 10
    assert g["elements"].max() < 1 << 12
    # heavy tail: the largest degree is far above the mean
    assert deg.max() > 20 * deg.mean()


def test_batched_streams_sizes():
    ss = wl.batched_streams(n_streams=64, seed=3)
    assert len(ss) == 64
    sizes = np.array([wl.n_elements(s) for s in ss])
    want = wl.lognormal_stream_sizes(64, 2 ** 14, 1.5, 1 << 22, 3)
    assert np.array_equal(sizes, want)
    for s in ss:
        assert s["len"].max() <= 512 and s["len"].min() >= 1
    # parent ids are globally unique across the batch
    allp = np.concatenate([s["parents"] for s in ss])
    assert len(np.unique(allp)) == len(allp)


def test_poisson_arrivals_rate():
    t = wl.poisson_arrivals(20000.0, 2.0, 1)
    assert abs(len(t) - 40000) < 5 * np.sqrt(40000)
    assert (np.diff(t) > 0).all()


def test_sized_region_lengths():
    """Region-sum streams: the lengths total n_total; fixed sizes are `size` except a
    shorter last region; variable sizes stay in 0..size with mean near size / 2; the
    draws are deterministic in the seed."""
    from paper_2006_07478_b300 import workloads as wl
    n = 100_003
    for size in (1, 7, 128, 129, 4096):
        L = wl.sized_lengths(n, size, seed=3).astype(np.int64)
        assert L.sum() == n
        assert np.all(L[:-1] == size) and 1 <= L[-1] <= size
    for size in (64, 513):
        L = wl.sized_lengths(n, size, seed=3, variable=True).astype(np.int64)
        assert L.sum() == n and L.min() >= 0 and L.max() <= size
        assert abs(L[:-1].mean() - size / 2) < 0.05 * size
        assert np.array_equal(L, wl.sized_lengths(n, size, seed=3, variable=True))
        assert not np.array_equal(L[:100], wl.sized_lengths(n, size, seed=4, variable=True)[:100])
    s = wl.sized_region_stream(n, 33, seed=5)
    assert s["R"] == (n + 32) // 33 and s["elements"].shape[0] == n and s["elements"].dtype == np.uint32
