"""Pins of the CPU oracle to facts outside itself (CPU only).

* fmix32 against published MurmurHash3_x86_32 vectors and its algebraic inverse;
* ora_run against closed forms (loaded arange elements), algebraic invariants of
  the aggregate (region splitting, permutation inside a region, threshold
  monotonicity, empty regions), thread-count invariance and sampled == full;
* filter pass rates against the probabilities the thresholds encode.
The independent protocol model (protosim) is compared with the oracle in
test_protosim.py.
"""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2006_07478_b300 import workloads as wl

M32 = 0xFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rotl(x, r):
    return ((x << r) | (x >> (32 - r))) & M32


def murmur3_x86_32(key: bytes, seed: int) -> int:
    """MurmurHash3_x86_32 body (block mix, tail, length) with the ORACLE's fmix32 as
    the final step, so a published vector pins the oracle's finalizer."""
    c1, c2 = 0xCC9E2D51, 0x1B873593
    h = seed
    nb = len(key) // 4
    for i in range(nb):
        k = int.from_bytes(key[4 * i:4 * i + 4], "little")
        k = (k * c1) & M32
        k = _rotl(k, 15)
        k = (k * c2) & M32
        h ^= k
        h = _rotl(h, 13)
        h = (h * 5 + 0xE6546B64) & M32
    tail = key[4 * nb:]
    k = 0
    if len(tail) >= 3:
        k ^= tail[2] << 16
    if len(tail) >= 2:
        k ^= tail[1] << 8
    if len(tail) >= 1:
        k ^= tail[0]
        k = (k * c1) & M32
        k = _rotl(k, 15)
        k = (k * c2) & M32
        h ^= k
    h ^= len(key)
    return oracle.fmix32(h)


def test_fmix32_published_vectors():
    n = 0
    with open(os.path.join(GOLDEN, "murmur3_x86_32_vectors.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key_hex, seed_hex, want_hex = line.split()
            key = b"" if key_hex == "-" else bytes.fromhex(key_hex)
            assert murmur3_x86_32(key, int(seed_hex, 16)) == int(want_hex, 16), line
            n += 1
    assert n >= 8


def test_fmix32_is_inverted_by_its_algebraic_inverse():
    # undo xor-shift k by re-applying it until the shifted-in bits are exhausted;
    # undo the multiplications with modular inverses mod 2^32
    inv1 = pow(0x85EBCA6B, -1, 1 << 32)
    inv2 = pow(0xC2B2AE35, -1, 1 << 32)

    def unxorshift(y, k):
        x = y
        for _ in range(32 // k + 1):
            x = y ^ (x >> k)
        return x

    def unfmix(h):
        h = unxorshift(h, 16)
        h = (h * inv2) & M32
        h = unxorshift(h, 13)
        h = (h * inv1) & M32
        h = unxorshift(h, 16)
        return h

    rng = np.random.default_rng(5)
    for x in [0, 1, M32, 0x80000000] + [int(v) for v in rng.integers(0, 1 << 32, 2000)]:
        assert unfmix(oracle.fmix32(x)) == x


def test_hash32_is_a_bijection_in_its_first_argument():
    # fmix32 is a bijection, so for fixed b, a -> fmix32(a ^ c_b) must be injective
    b = 0x5EED
    vals = {oracle.hash32(a, b) for a in range(20000)}
    assert len(vals) == 20000


def _identity_pipeline():
    return [("enum_load",), ("filter_mod", 1, 0), ("map_mul", 1, 0), ("aggregate",)]


def _arange_stream(lengths):
    L = np.asarray(lengths, dtype=np.uint32)
    n = int(L.astype(np.int64).sum())
    return wl.make_stream(L, elements=np.arange(n, dtype=np.uint32))


def test_closed_form_loaded_arange():
    rng = np.random.default_rng(11)
    L = rng.integers(0, 40, 500)
    L[::7] = 0
    s = _arange_stream(L)
    res = oracle.run(_identity_pipeline(), s)
    off = np.concatenate(([0], np.cumsum(L)[:-1])).astype(np.int64)
    Ls = L.astype(np.int64)
    assert np.array_equal(res["count"], Ls.astype(np.uint32))
    assert np.array_equal(res["sum"], (Ls * off + Ls * (Ls - 1) // 2).astype(np.uint64))
    want_min = np.where(Ls > 0, off, M32).astype(np.uint32)
    assert np.array_equal(res["min"], want_min)


def test_closed_form_map_and_mod_filter():
    rng = np.random.default_rng(12)
    L = rng.integers(0, 50, 300)
    s = _arange_stream(L)
    off = np.concatenate(([0], np.cumsum(L)[:-1])).astype(np.int64)
    # map x -> 3x + 5 (no wrap at these sizes)
    pipe = [("enum_load",), ("map_mul", 3, 5), ("aggregate",)]
    res = oracle.run(pipe, s)
    Ls = L.astype(np.int64)
    sx = Ls * off + Ls * (Ls - 1) // 2
    assert np.array_equal(res["sum"], (3 * sx + 5 * Ls).astype(np.uint64))
    # keep x mod 3 == 1: count of such x in [off, off+L)
    pipe = [("enum_load",), ("filter_mod", 3, 1), ("aggregate",)]
    res = oracle.run(pipe, s)

    def upto(n):  # number of x in [0, n) with x % 3 == 1
        return (n + 1) // 3
    want = upto(off + Ls) - upto(off)
    assert np.array_equal(res["count"], want.astype(np.uint32))


def test_map_wraps_mod_2_32():
    s = _arange_stream([3])
    s["elements"] = np.array([M32, 0x80000000, 7], dtype=np.uint32)
    res = oracle.run([("enum_load",), ("map_mul", 2, 1), ("aggregate",)], s)
    assert int(res["sum"][0]) == ((2 * M32 + 1) & M32) + 1 + 15
    assert int(res["min"][0]) == 1


def test_empty_regions_and_threshold_extremes():
    s = wl.cascade_stream(n_total=5000, mean=4, seed=3)
    none = [("enum_load",), ("filter_hash_ctx", 1, 0), ("aggregate",)]
    res = oracle.run(none, s)
    assert not res["count"].any() and not res["sum"].any() and (res["min"] == M32).all()
    allp = [("enum_load",), ("filter_hash_ctx", 1, M32), ("aggregate",)]
    res = oracle.run(allp, s)
    # keeps every element except the ones with (h ^ t) == 2^32 - 1 (about 5000 / 2^32)
    assert int(res["count"].astype(np.int64).sum()) == 5000
    zero_len = s["len"] == 0
    assert zero_len.any()
    assert (res["count"][zero_len] == 0).all() and (res["min"][zero_len] == M32).all()


def test_expand_with_zero_fanout_emits_nothing():
    s = wl.hashed_uniform_stream(200, 16, 2)
    res = oracle.run([("enum_hash",), ("expand", 0, 9), ("aggregate",)], s)
    assert not res["count"].any()


def test_region_split_merges():
    """Cutting a region in two (same parent context) splits its aggregate."""
    rng = np.random.default_rng(13)
    L = rng.integers(1, 60, 200)
    n = int(L.sum())
    elems = wl.to_u32(wl.splitmix64_counter(99, 0, n))
    ctx = wl.to_u32(wl.splitmix64_counter(98, 0, 200))
    pipe = wl.pipeline_cascade()
    pipe[1] = ("filter_hash_ctx", 1, 3000000000)   # looser thresholds keep more items
    pipe[2] = ("filter_hash_ctx", 2, 3000000000)
    pipe[3] = ("filter_hash_ctx", 3, 3000000000)
    whole = oracle.run(pipe, wl.make_stream(L, elements=elems, ctx=ctx))
    cut = rng.integers(0, L + 1)
    L2 = np.stack([cut, L - cut], axis=1).reshape(-1)
    ctx2 = np.repeat(ctx, 2)
    parts = oracle.run(pipe, wl.make_stream(L2, elements=elems, ctx=ctx2))
    assert np.array_equal(parts["count"][0::2] + parts["count"][1::2], whole["count"])
    assert np.array_equal(parts["sum"][0::2] + parts["sum"][1::2], whole["sum"])
    assert np.array_equal(np.minimum(parts["min"][0::2], parts["min"][1::2]), whole["min"])
    assert whole["count"].sum() > 0


def test_permutation_inside_region_invariance():
    rng = np.random.default_rng(14)
    s = wl.cascade_stream(n_total=20000, mean=32, seed=5)
    pipe = wl.pipeline_cascade()
    a = oracle.run(pipe, s)
    e = s["elements"].copy()
    off = np.concatenate(([0], np.cumsum(s["len"].astype(np.int64))))
    for r in range(s["R"]):
        seg = e[off[r]:off[r + 1]]
        rng.shuffle(seg)
    s2 = dict(s, elements=e)
    b = oracle.run(pipe, s2)
    for k in ("count", "sum", "min"):
        assert np.array_equal(a[k], b[k])


def test_threshold_monotonicity():
    s = wl.cascade_stream(n_total=30000, mean=16, seed=6)
    prev = None
    for theta in (0, 1 << 28, 1 << 30, 1 << 31, 3 << 30, M32):
        c = oracle.run([("enum_load",), ("filter_hash_ctx", 1, theta), ("aggregate",)], s)["count"]
        if prev is not None:
            assert (c >= prev).all()
        prev = c


def test_threads_and_sampling_do_not_change_results():
    s = wl.cascade_stream(n_total=200000, mean=8, seed=7)
    pipe = wl.pipeline_cascade()
    a = oracle.run(pipe, s, threads=1)
    b = oracle.run(pipe, s, threads=5)
    for k in ("count", "sum", "min"):
        assert np.array_equal(a[k], b[k])
    idx = np.array([0, 1, 17, s["R"] // 2, s["R"] - 1], dtype=np.uint64)
    c = oracle.run_sampled(pipe, s, idx)
    for k in ("count", "sum", "min"):
        assert np.array_equal(c[k], a[k][idx.astype(np.int64)])


def test_csr_offsets_equal_lengths():
    g = wl.graph_stream(V=2000, E=20000, cap=1000, seed=7)
    pipe = wl.pipeline_graph_edges()
    a = oracle.run(pipe, g)
    L = np.diff(g["offsets"].astype(np.int64)).astype(np.uint32)
    b = oracle.run(pipe, dict(g, offsets=None, len=L))
    for k in ("count", "sum", "min"):
        assert np.array_equal(a[k], b[k])


def test_pass_rates_match_thresholds():
    # hashed elements, keep even: each element survives with probability 1/2
    s = wl.hashed_uniform_stream()
    res = oracle.run(wl.pipeline_hash_filter_map(), s)
    N = int(s["len"].astype(np.int64).sum())
    frac = res["count"].astype(np.int64).sum() / N
    assert abs(frac - 0.5) < 5 * np.sqrt(0.25 / N)
    # cascade: survival 0.5 * 0.3 * 0.1 = 0.015
    s = wl.cascade_stream(n_total=1 << 20, mean=32, seed=7)
    res = oracle.run(wl.pipeline_cascade(), s, threads=4)
    p = 0.5 * 0.3 * 0.1
    frac = res["count"].astype(np.int64).sum() / (1 << 20)
    assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / (1 << 20))


def test_invalid_pipelines_rejected():
    s = wl.hashed_uniform_stream(10, 4, 1)
    with pytest.raises(ValueError):
        oracle.run([("aggregate",)], s)
    with pytest.raises(ValueError):
        oracle.run([("enum_hash",), ("filter_mod", 0, 0), ("aggregate",)], s)
    with pytest.raises(ValueError):
        oracle.run([("enum_hash",), ("map_mul", 1, 0)], s)


# ---------------------------------------------------------------------------
# filter_weight_lt (keep edge u -> v iff w(v) < w(u), w(v) = hash32(v, salt)): pinned by
# what a strict comparison of a bijective weight must satisfy, and tied to the pinned
# direction of the threshold filter


def _edge_stream(src, dst):
    """One region per directed edge: parent id = source vertex, its only element = dst."""
    src = np.asarray(src, dtype=np.uint32)
    return wl.make_stream(np.ones(src.shape[0], dtype=np.uint32), parents=src,
                          elements=np.asarray(dst, dtype=np.uint32))


WPIPE = [("enum_load",), ("filter_weight_lt", wl.WEIGHT_SALT), ("aggregate",)]


def test_weight_filter_self_loops_never_survive():
    v = np.arange(5000, dtype=np.uint32) * 7919
    res = oracle.run(WPIPE, _edge_stream(v, v))
    assert not res["count"].any() and (res["min"] == M32).all()


def test_weight_filter_is_antisymmetric_with_pass_rate_one_half():
    rng = np.random.default_rng(21)
    n = 40000
    u = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    v = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    v[u == v] ^= 1
    fwd = oracle.run(WPIPE, _edge_stream(u, v))["count"].astype(np.int64)
    bwd = oracle.run(WPIPE, _edge_stream(v, u))["count"].astype(np.int64)
    # hash32 is a bijection in its first argument, so w(u) != w(v): exactly one direction
    assert np.array_equal(fwd + bwd, np.ones(n, dtype=np.int64))
    assert abs(fwd.mean() - 0.5) < 5 * np.sqrt(0.25 / n)


def test_weight_filter_ranks_a_complete_digraph():
    """Every vertex of a complete digraph (no self-loops) keeps the out-edges to the
    vertices of smaller weight: the counts are the weight ranks, a permutation of
    0..n-1 (a strict total order), and min dst is the smallest id of lower rank."""
    n = 300
    ids = (np.arange(n, dtype=np.uint64) * 2654435761 % (1 << 32)).astype(np.uint32)
    L = np.full(n, n - 1, dtype=np.uint32)
    dst = np.concatenate([np.delete(ids, i) for i in range(n)])
    res = oracle.run(WPIPE, wl.make_stream(L, parents=ids, elements=dst))
    rank = res["count"].astype(np.int64)
    assert np.array_equal(np.sort(rank), np.arange(n))
    for i in range(n):
        lower = ids[rank < rank[i]]
        want = int(lower.min()) if lower.size else M32
        assert int(res["min"][i]) == want


def test_weight_filter_is_the_threshold_filter_at_the_parents_weight():
    """keep w(x) < w(p) is the context-free threshold filter keep hash32(x, salt) < theta
    with theta = w(p): the threshold filter's direction and rates are pinned above."""
    rng = np.random.default_rng(22)
    for p in (0, 1, 12345, M32, int(rng.integers(0, 1 << 32))):
        x = rng.integers(0, 1 << 32, 3000, dtype=np.uint64).astype(np.uint32)
        a = oracle.run(WPIPE, _edge_stream(np.full(x.shape[0], p), x))["count"]
        theta = oracle.hash32(p, wl.WEIGHT_SALT)
        b = oracle.run([("enum_load",), ("filter_hash_ctx", wl.WEIGHT_SALT, theta), ("aggregate",)],
                       wl.make_stream(np.ones(x.shape[0], dtype=np.uint32), elements=x))["count"]
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# expand (n = hash32(x, salt) mod (k + 1) outputs hash32(x, salt + 1 + j), j < n): pinned
# by bounds, the uniform law of n, the modular relation between fan-outs, and the
# independence of the output values from n


def _single_items(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    return wl.make_stream(np.ones(n, dtype=np.uint32), elements=x)


def _expand_counts(s, k, salt=9):
    return oracle.run([("enum_load",), ("expand", k, salt), ("aggregate",)], s)


def test_expand_outputs_are_bounded_and_uniform_in_number():
    n = 60000
    s = _single_items(n, 23)
    for k in (1, 2, 3, 5, 8):
        c = _expand_counts(s, k)["count"].astype(np.int64)
        assert c.min() >= 0 and c.max() <= k
        # n = h mod (k + 1) of a uniform 32-bit h: every value 0..k about n / (k + 1) times
        freq = np.bincount(c, minlength=k + 1)
        p = 1.0 / (k + 1)
        assert np.all(np.abs(freq - n * p) < 5 * np.sqrt(n * p * (1 - p))), (k, freq)
        # mean yield k / 2 (variance ((k + 1)^2 - 1) / 12 per item)
        sd = np.sqrt(((k + 1) ** 2 - 1) / 12.0 / n)
        assert abs(c.mean() - k / 2.0) < 5 * sd


def test_expand_counts_follow_the_modulus():
    """h mod 2 = (h mod 4) mod 2 and h mod 4 = (h mod 8) mod 4: the counts at fan-outs 1,
    3 and 7 are reductions of one another (a wrong modulus breaks this)."""
    s = _single_items(30000, 24)
    c1 = _expand_counts(s, 1)["count"].astype(np.int64)
    c3 = _expand_counts(s, 3)["count"].astype(np.int64)
    c7 = _expand_counts(s, 7)["count"].astype(np.int64)
    assert np.array_equal(c1, c3 % 2)
    assert np.array_equal(c3, c7 % 4)


def test_expand_output_values_do_not_depend_on_the_count():
    """The j-th output is the same value at every fan-out (the output sequence does not
    depend on k), and it is drawn with a salt other than the count's: among items with
    one output, that output's residue mod (k + 1) is 1 only about 1 / (k + 1) of the time."""
    n = 40000
    s = _single_items(n, 25)
    r1, r3 = _expand_counts(s, 1), _expand_counts(s, 3)
    one = (r1["count"] == 1) & (r3["count"] >= 1)
    assert one.sum() > n // 4
    # with one output at fan-out 1 the sum is y_0; at fan-out 3 the min is <= y_0 and
    # with exactly one output there it equals y_0
    assert np.all(r3["min"][one].astype(np.int64) <= r1["sum"][one].astype(np.int64))
    both1 = (r1["count"] == 1) & (r3["count"] == 1)
    assert np.array_equal(r1["sum"][both1], r3["sum"][both1])
    k = 3
    y0 = r3["sum"][r3["count"] == 1].astype(np.int64)
    rate = np.mean(y0 % (k + 1) == 1)
    p = 1.0 / (k + 1)
    assert abs(rate - p) < 5 * np.sqrt(p * (1 - p) / y0.size)


def test_expand_then_keep_all_adds_up_exactly():
    s = wl.hashed_uniform_stream(3000, 40, 3)
    a = oracle.run([("enum_hash",), ("expand", 4, 17), ("aggregate",)], s)
    b = oracle.run([("enum_hash",), ("expand", 4, 17), ("filter_mod", 1, 0), ("aggregate",)], s)
    for key in ("count", "sum", "min"):
        assert np.array_equal(a[key], b[key])
    # every region's count is at most k times its length
    assert np.all(a["count"].astype(np.int64) <= 4 * s["len"].astype(np.int64))


# ---------------------------------------------------------------------------
# emit sink (element results stripped of their parent, Section 4): pinned by the closed
# form of the identity pipeline and by the aggregate's pinned count / sum / min


def _as_emit(pipe):
    return list(pipe[:-1]) + [("emit",)]


def test_emit_identity_pipeline_returns_each_region_in_order():
    rng = np.random.default_rng(31)
    L = rng.integers(0, 30, 400)
    L[::9] = 0
    n = int(L.sum())
    el = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    s = wl.make_stream(L, elements=el)
    res = oracle.run_emit([("enum_load",), ("emit",)], s)
    assert np.array_equal(res["count"], L.astype(np.uint32))
    assert np.array_equal(res["values"][:n], el)       # F = 1: the segments tile the array
    assert np.array_equal(res["start"], np.concatenate(([0], np.cumsum(L))))


def _segments(res):
    return [res["values"][res["start"][r]:res["start"][r] + int(res["count"][r])] for r in range(len(res["count"]))]


@pytest.mark.parametrize("which", ["cascade", "hashed", "expand", "graph"])
def test_emit_agrees_with_the_aggregate(which):
    if which == "cascade":
        pipe, s = wl.pipeline_cascade(), wl.cascade_stream(n_total=40000, mean=24, seed=3)
    elif which == "hashed":
        pipe, s = wl.pipeline_hash_filter_map(), wl.hashed_uniform_stream(2000, 64, 5)
    elif which == "expand":
        pipe = [("enum_hash",), ("expand", 3, 5), ("filter_mod", 3, 1), ("expand", 2, 8), ("aggregate",)]
        s = wl.hashed_uniform_stream(1500, 20, 6)
    else:
        pipe, s = wl.pipeline_graph_edges(), wl.graph_stream(V=3000, E=30000, cap=2000, seed=7)
    agg = oracle.run(pipe, s)
    em = oracle.run_emit(_as_emit(pipe), s)
    assert np.array_equal(em["count"], agg["count"])
    F = oracle.fanout_product(pipe)
    L = np.diff(em["start"]) // F
    assert np.all(em["count"].astype(np.int64) <= F * L)
    segs = _segments(em)
    sums = np.array([int(x.astype(np.uint64).sum()) for x in segs], dtype=np.uint64)
    mins = np.array([int(x.min()) if x.size else M32 for x in segs], dtype=np.uint32)
    assert np.array_equal(sums, agg["sum"])
    assert np.array_equal(mins, agg["min"])
    # the slots past each region's count are untouched
    used = np.zeros(em["values"].shape[0], dtype=bool)
    for r in range(s["R"]):
        used[em["start"][r]:em["start"][r] + int(em["count"][r])] = True
    assert not em["values"][~used].any()


# ---------------------------------------------------------------------------
# tree topologies (Figure 1(b)): the stream is replicated at a branch, so each leaf's
# results are the linear pipeline along the root-to-leaf path (pinned above)


def _path(pipeline, inputs, leaf):
    path = [leaf]
    while path[-1] != 0:
        path.append(inputs[path[-1]])
    return [pipeline[i] for i in reversed(path)]


TREES = [
    # enumerate -> A -> {B -> sink, sink}
    ([("enum_load",), ("filter_hash_ctx", 1, 2147483648), ("filter_hash_ctx", 2, 1288490188), ("aggregate",),
      ("aggregate",)], [0, 0, 1, 2, 1]),
    # enumerate -> map -> {filter -> sink, expand -> sink}
    ([("enum_hash",), ("map_mul", 2654435761, 7), ("filter_mod", 2, 0), ("aggregate",), ("expand", 3, 11),
      ("aggregate",)], [0, 0, 1, 2, 1, 4]),
    # enumerate -> expand -> {sink, sink} (the same expanded stream twice)
    ([("enum_hash",), ("expand", 2, 5), ("aggregate",), ("aggregate",)], [0, 0, 1, 1]),
]


@pytest.mark.parametrize("ti", range(len(TREES)))
def test_tree_leaves_are_their_root_to_leaf_pipelines(ti):
    pipe, inputs = TREES[ti]
    if pipe[0][0] == "enum_load":
        s = wl.cascade_stream(n_total=30000, mean=12, seed=4)
    else:
        s = wl.hashed_uniform_stream(2000, 48, 8)
    res = oracle.run_tree(pipe, inputs, s)
    leaves = [i for i, st in enumerate(pipe) if st[0] == "aggregate"]
    assert len(res) == len(leaves)
    for k, leaf in enumerate(leaves):
        want = oracle.run(_path(pipe, inputs, leaf), s)
        for key in ("count", "sum", "min"):
            assert np.array_equal(res[k][key], want[key]), (ti, leaf, key)
    if ti == 2:
        for key in ("count", "sum", "min"):
            assert np.array_equal(res[0][key], res[1][key])


def test_tree_validation():
    s = wl.hashed_uniform_stream(10, 4, 1)
    with pytest.raises(ValueError):          # a sink with a child
        oracle.run_tree([("enum_hash",), ("aggregate",), ("aggregate",)], [0, 0, 1], s)
    with pytest.raises(ValueError):          # an element stage without children
        oracle.run_tree([("enum_hash",), ("filter_mod", 2, 0), ("map_mul", 1, 0), ("aggregate",)], [0, 0, 1, 1], s)
    with pytest.raises(ValueError):          # an input that is not upstream
        oracle.run_tree([("enum_hash",), ("filter_mod", 2, 0), ("aggregate",)], [0, 0, 2], s)
