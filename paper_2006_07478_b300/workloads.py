"""Seeded synthetic workloads for region-segmented streaming pipelines.

This module only draws inputs: region lengths, parent ids, element arrays,
per-region context words, CSR graphs and arrival times.  It holds none of the
pipeline's arithmetic (no hash32, no filter or map, no aggregation), so both the
CUDA path and the CPU oracle can be fed from it without sharing method code.

Generators (published definitions, written here from those definitions):
  * xorshift64 -- Marsaglia, "Xorshift RNGs" (2003), shift triple (13, 7, 17);
    state = seed (non-zero), each call returns the new state.
  * splitmix64 -- Steele, Lea & Flood, "Fast splittable pseudorandom number
    generators" (2014): state advances by 0x9E3779B97F4A7C15 and is mixed by
    (x ^ x>>30)*0xBF58476D1CE4E5B9, (x ^ x>>27)*0x94D049BB133111EB, x ^ x>>31.
    Used counter-style: value j of substream s is mix(s + (j+1)*gamma), so whole
    arrays vectorise.

A stream is a dict with keys R, parents, len, offsets, elements, ctx (numpy
uint32 arrays or None) plus descriptive metadata.  A pipeline is a list of
plain tuples naming stage operations; each executing side maps the names to
its own implementation.
"""
from __future__ import annotations

import math

import numpy as np

U64 = np.uint64
MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15

# ---------------------------------------------------------------------------
# generators


def splitmix64_scalar(x: int) -> int:
    """One splitmix64 step from state x: returns the mixed output of x + gamma."""
    z = (x + GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def substream_seed(seed: int, tag: int) -> int:
    """Seed of an independent substream: splitmix64(seed XOR tag), never zero."""
    s = splitmix64_scalar((seed ^ tag) & MASK64)
    return s if s != 0 else 1


def splitmix64_counter(seed: int, start: int, n: int) -> np.ndarray:
    """Values start..start+n-1 of the splitmix64 sequence seeded with `seed`."""
    with np.errstate(over="ignore"):
        j = np.arange(start + 1, start + n + 1, dtype=U64)
        z = U64(seed) + j * U64(GAMMA)
        z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
        return z ^ (z >> U64(31))


def xorshift64_sequence(seed: int, n: int) -> np.ndarray:
    """First n outputs of xorshift64 (13, 7, 17) started from state `seed`."""
    x = seed & MASK64
    if x == 0:
        raise ValueError("xorshift64 needs a non-zero seed")
    out = np.empty(n, dtype=U64)
    for i in range(n):
        x ^= (x << 13) & MASK64
        x ^= x >> 7
        x ^= (x << 17) & MASK64
        out[i] = x
    return out


def xorshift64_lockstep(states: np.ndarray) -> np.ndarray:
    """Advance a vector of independent xorshift64 states by one step (in place)."""
    with np.errstate(over="ignore"):
        states ^= states << U64(13)
        states ^= states >> U64(7)
        states ^= states << U64(17)
    return states


def uniform_int(draws: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """lo + draw mod (hi-lo+1): exact for power-of-two ranges, negligible bias otherwise."""
    span = U64(hi - lo + 1)
    return (draws % span).astype(np.int64) + lo


def to_u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64) & U64(0xFFFFFFFF)).astype(np.uint32)


# ---------------------------------------------------------------------------
# pipelines (plain descriptions; no arithmetic here)

HASH_MAP_MUL = 2654435761
CASCADE_SALTS = (1, 2, 3)
CASCADE_THETAS = (2147483648, 1288490188, 429496729)   # floor(0.5, 0.3, 0.1 * 2^32)
WEIGHT_SALT = 0x5EED


def pipeline_hash_filter_map() -> list:
    """enumerate (hashed elements) -> keep even -> multiply -> aggregate per region."""
    return [("enum_hash",), ("filter_mod", 2, 0), ("map_mul", HASH_MAP_MUL, 0), ("aggregate",)]


def pipeline_cascade() -> list:
    """enumerate (loaded elements) -> three context-dependent hash filters -> aggregate."""
    st = [("enum_load",)]
    for salt, theta in zip(CASCADE_SALTS, CASCADE_THETAS):
        st.append(("filter_hash_ctx", salt, theta))
    st.append(("aggregate",))
    return st


def pipeline_graph_edges() -> list:
    """enumerate a vertex's out-edges -> keep w(dst) < w(src) -> aggregate count and min dst."""
    return [("enum_load",), ("filter_weight_lt", WEIGHT_SALT), ("aggregate",)]


# ---------------------------------------------------------------------------
# streams


def make_stream(lengths=None, *, parents=None, offsets=None, elements=None, ctx=None, **meta) -> dict:
    if lengths is None and offsets is None:
        raise ValueError("need lengths or offsets")
    if lengths is not None:
        lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
        R = int(lengths.shape[0])
    else:
        offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        R = int(offsets.shape[0]) - 1
    s = {
        "R": R,
        "len": lengths,
        "offsets": offsets,
        "parents": None if parents is None else np.ascontiguousarray(parents, dtype=np.uint32),
        "elements": None if elements is None else np.ascontiguousarray(elements, dtype=np.uint32),
        "ctx": None if ctx is None else np.ascontiguousarray(ctx, dtype=np.uint32),
    }
    s.update(meta)
    return s


def n_elements(stream: dict) -> int:
    if stream["offsets"] is not None:
        o = stream["offsets"]
        return int(o[-1]) - int(o[0])
    return int(stream["len"].astype(np.uint64).sum())


def hashed_uniform_stream(n_regions: int = 10_000, max_len: int = 64, seed: int = 1) -> dict:
    """10^4 parents p_r = r with lengths 1..max_len drawn by xorshift64 (the small
    hashed-element workload)."""
    draws = xorshift64_sequence(seed, n_regions)
    lengths = uniform_int(draws, 1, max_len)
    return make_stream(lengths, parents=None, workload=f"hash-uniform R={n_regions} L=U[1,{max_len}] seed={seed}")


def geometric_lengths(n_total: int, mean: float, seed: int, support_from_zero: bool = True) -> np.ndarray:
    """Region lengths drawn as the gaps of a Bernoulli process with success
    probability p = 1/(mean+1) on {0,1,...} (mean exactly `mean`), or 1/mean on
    {1,2,...}; drawn until the total reaches n_total and the last one truncated."""
    p_den = mean + 1.0 if support_from_zero else float(mean)
    thresh = int((1 << 64) / p_den) if p_den > 1.0 else MASK64
    T = U64(min(thresh, MASK64))
    sub = substream_seed(seed, 0x1E9)
    out = []
    total = 0
    start = 0
    prev = -1  # index of the previous success
    chunk = 1 << 24
    while total < n_total:
        u = splitmix64_counter(sub, start, chunk)
        succ = np.flatnonzero(u < T) + start
        if succ.size:
            gaps = np.diff(np.concatenate(([prev], succ))) - 1   # failures before each success
            if not support_from_zero:
                gaps = gaps + 1
            out.append(gaps)
            total += int(gaps.sum())
            prev = int(succ[-1])
        start += chunk
    lengths = np.concatenate(out).astype(np.int64)
    csum = np.cumsum(lengths)
    last = int(np.searchsorted(csum, n_total))          # first index with csum >= n_total
    lengths = lengths[: last + 1].copy()
    lengths[-1] -= int(csum[last]) - n_total
    return lengths.astype(np.uint32)


def cascade_stream(n_total: int = 1 << 26, mean: float = 32, seed: int = 7,
                   support_from_zero: bool = True) -> dict:
    """Loaded-element stream for the three-filter cascade: n_total uint32 elements
    cut into geometric regions of mean `mean`, with a uniform context word t_r per
    region."""
    lengths = geometric_lengths(n_total, mean, seed, support_from_zero)
    R = lengths.shape[0]
    elements = to_u32(splitmix64_counter(substream_seed(seed, 0xE1E), 0, n_total))
    ctx = to_u32(splitmix64_counter(substream_seed(seed, 0xC7C), 0, R))
    return make_stream(lengths, parents=None, elements=elements, ctx=ctx,
                       workload=f"cascade N={n_total} mean={mean} seed={seed}")


def pipeline_lines() -> list:
    """The stand-in for the paper's taxi application (Section 5): lines of text are
    enumerated into characters; stage 1 keeps the characters that may open a coordinate
    pair (a context-dependent test passing about 45 of a line's 1,397 characters); stage
    2 verifies each candidate (keeps 90%) and stage 3 parses it (a map); the aggregate
    reduces each line's parsed pairs."""
    return [("enum_load",), ("filter_hash_ctx", 11, LINE_THETA_OPEN), ("filter_hash_ctx", 12, LINE_THETA_VERIFY),
            ("map_mul", 2654435761, 12345), ("aggregate",)]


LINE_MEAN = 1397                                  # characters per line (taxi input, Section 5)
LINE_PAIRS = 45                                   # coordinate pairs per line
LINE_THETA_OPEN = (LINE_PAIRS << 32) // LINE_MEAN  # pass rate 45 / 1397
LINE_THETA_VERIFY = 3865470566                    # floor(0.9 * 2^32)


def lines_stream(n_total: int = 1 << 26, seed: int = 13) -> dict:
    """n_total characters (splitmix64 words) cut into lines of U{1..2 * 1397 - 1}
    characters (mean 1397), the last one truncated; one context word per line."""
    m = int(n_total / LINE_MEAN * 1.2) + 16
    L = uniform_int(splitmix64_counter(substream_seed(seed, 0x11E), 0, m), 1, 2 * LINE_MEAN - 1)
    cs = np.cumsum(L)
    last = int(np.searchsorted(cs, n_total))
    L = L[: last + 1].copy()
    L[-1] -= int(cs[last]) - int(n_total)
    R = L.shape[0]
    elements = to_u32(splitmix64_counter(substream_seed(seed, 0xC4A), 0, n_total))
    ctx = to_u32(splitmix64_counter(substream_seed(seed, 0xC7B), 0, R))
    return make_stream(L.astype(np.uint32), elements=elements, ctx=ctx,
                       workload=f"lines N={n_total} L=U[1,{2 * LINE_MEAN - 1}] seed={seed}")


def pipeline_region_sum() -> list:
    """The paper's region-sum benchmark (Section 5, Figures figFixed and figVariable):
    enumerate each region of an integer array and reduce it to its sum (and count)."""
    return [("enum_load",), ("aggregate",)]


def sized_lengths(n_total: int, size: int, seed: int = 11, variable: bool = False) -> np.ndarray:
    """Region lengths totalling n_total: `size` each (the last one shorter), or, with
    `variable`, uniform on 0..size (splitmix64 draws), the last one truncated."""
    if variable:
        sub = substream_seed(seed, 0x5A5)
        n_est = 2 * n_total // max(size, 1) + 1024
        lengths = (splitmix64_counter(sub, 0, n_est) % U64(size + 1)).astype(np.int64)
        csum = np.cumsum(lengths)
        while csum[-1] < n_total:   # draw more (never in practice: n_est is twice the mean)
            more = (splitmix64_counter(sub, lengths.shape[0], n_est) % U64(size + 1)).astype(np.int64)
            lengths = np.concatenate([lengths, more])
            csum = np.cumsum(lengths)
        last = int(np.searchsorted(csum, n_total))
        lengths = lengths[: last + 1].copy()
        lengths[-1] -= int(csum[last]) - n_total
    else:
        R = (n_total + size - 1) // size
        lengths = np.full(R, size, dtype=np.int64)
        lengths[-1] = n_total - size * (R - 1)
    return lengths.astype(np.uint32)


def sized_region_stream(n_total: int, size: int, seed: int = 11, variable: bool = False) -> dict:
    """n_total uint32 elements (splitmix64) cut into regions by `sized_lengths`."""
    elements = to_u32(splitmix64_counter(substream_seed(seed, 0xE1E), 0, n_total))
    kind = "U{0.." + str(size) + "}" if variable else str(size)
    return make_stream(sized_lengths(n_total, size, seed, variable), parents=None, elements=elements,
                       workload=f"region-sum N={n_total} size={kind} seed={seed}")


def zipf_degrees(V: int, E: int, s: float, cap: int, seed: int) -> np.ndarray:
    """Out-degrees with a Zipf(s) shape on 1..cap, rescaled so they sum to exactly E
    with none above cap."""
    k = np.arange(1, cap + 1, dtype=np.float64)
    pmf = k ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = (splitmix64_counter(substream_seed(seed, 0x21F), 0, V) >> U64(11)).astype(np.float64) / float(1 << 53)
    kv = np.searchsorted(cdf, u, side="right") + 1
    kv = np.minimum(kv, cap).astype(np.int64)
    d = np.floor(kv.astype(np.float64) * (E / float(kv.sum()))).astype(np.int64)
    d = np.clip(d, 0, cap)
    short = E - int(d.sum())
    perm_keys = splitmix64_counter(substream_seed(seed, 0x9E5), 0, V)
    order = np.argsort(perm_keys, kind="stable")
    while short > 0:
        room = order[d[order] < cap]
        take = room[:short]
        d[take] += 1
        short -= take.shape[0]
    while short < 0:   # cannot happen with floor scaling, kept for completeness
        big = order[d[order] > 0][: -short]
        d[big] -= 1
        short += big.shape[0]
    return d


def graph_stream(V: int = 1 << 22, E: int = 1 << 26, s: float = 2.1, cap: int = 1 << 16, seed: int = 7) -> dict:
    """CSR out-edge stream: region v = vertex v's out-edges, elements = dst ids
    uniform in [0, V)."""
    deg = zipf_degrees(V, E, s, min(cap, E), seed)
    offsets = np.zeros(V + 1, dtype=np.uint64)
    np.cumsum(deg, out=offsets[1:])
    dst = (splitmix64_counter(substream_seed(seed, 0xD57), 0, E) % U64(V)).astype(np.uint32)
    return make_stream(None, parents=None, offsets=offsets.astype(np.uint32), elements=dst,
                       workload=f"graph V={V} E={E} zipf={s} cap={cap} seed={seed}")


def lognormal_stream_sizes(n_streams: int, median: float, sigma: float, cap: int, seed: int) -> np.ndarray:
    """Stream sizes round(exp(ln median + sigma*z)) clipped to [1, cap], z standard
    normal by Box-Muller from splitmix64 doubles."""
    u = splitmix64_counter(substream_seed(seed, 0x106), 0, 2 * n_streams)
    u = ((u >> U64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    z = np.sqrt(-2.0 * np.log(u[0::2])) * np.cos(2.0 * math.pi * u[1::2])
    n = np.rint(np.exp(math.log(median) + sigma * z))
    return np.clip(n, 1, cap).astype(np.int64)


def uniform_region_lengths(sizes: np.ndarray, lo: int, hi: int, seed: int) -> list:
    """Per stream, region lengths U{lo..hi} drawn from that stream's own splitmix64
    substream (counter-based, so each stream vectorises) until its size is reached;
    the last region is truncated."""
    out = []
    mean = 0.5 * (lo + hi)
    for i, n in enumerate(sizes.astype(np.int64)):
        sub = substream_seed(seed, 0x5000 + i)
        m = int(n / mean * 1.25) + 32
        while True:
            L = uniform_int(splitmix64_counter(sub, 0, m), lo, hi)
            cs = np.cumsum(L)
            if cs[-1] >= n:
                break
            m *= 2
        last = int(np.searchsorted(cs, n))
        L = L[: last + 1].copy()
        L[-1] -= int(cs[last]) - int(n)
        out.append(L.astype(np.uint32))
    return out


def batched_streams(n_streams: int = 4096, median: float = 2 ** 14, sigma: float = 1.5,
                    cap: int = 1 << 22, lo: int = 1, hi: int = 512, seed: int = 3) -> list:
    """Many independent hashed-element streams with lognormal sizes; parent ids are
    the global region ordinal across the batch so streams do not repeat."""
    sizes = lognormal_stream_sizes(n_streams, median, sigma, cap, seed)
    lens = uniform_region_lengths(sizes, lo, hi, seed)
    streams = []
    base = 0
    for i, L in enumerate(lens):
        R = L.shape[0]
        parents = np.arange(base, base + R, dtype=np.uint64).astype(np.uint32)
        streams.append(make_stream(L, parents=parents, workload=f"batched stream {i}"))
        base += R
    return streams


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Open-loop Poisson arrival times (seconds) on [0, duration)."""
    n_guess = int(rate_per_s * duration_s * 1.2) + 64
    u = splitmix64_counter(substream_seed(seed, 0xA77), 0, n_guess)
    u = ((u >> U64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    t = np.cumsum(-np.log(u) / rate_per_s)
    return t[t < duration_s]
