"""Per-edge boundary modes and tree topologies on the GPU vs the CPU oracle, bit-exact.

* Per-stage strategy mixing (Section 5, the taxi application): signals on the edges into
  the first stages, tags after a filter has shrunk the regions.
* Per-lane state selection (Section 6): edges that carry signals with credits while the
  consumer's ensembles span them, each lane picking its own item's context.
* Tree topologies (Section 2.1, Figure 1(b)): a stage's output stream -- and with it every
  region boundary -- replicated to each of its children, one aggregate per leaf.

Every mode combination gives the plain definition's results (Lemma 1: the delivery
mechanism does not change which items meet which context), so each case is compared
element by element with oracle.run / oracle.run_tree on the same seeded input."""
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


def _check(rs, pipe, stream, modes, outputs=("count", "sum", "min"), strategy="signal", **opts):
    want = oracle.run(pipe, stream)
    got, st = rs.run_stream(pipe, stream, strategy=strategy, outputs=outputs, boundary_modes=modes, **opts)
    assert st["device_status"] == 0, st
    for k in outputs:
        bad = np.flatnonzero(got[k] != want[k])
        assert bad.size == 0, (k, modes, bad[:5], got[k][bad[:5]], want[k][bad[:5]])
    return st


# (boundary mode per stage 1..4) for the cascade's four edges
CASCADE_MODES = [
    {1: "signal", 2: "tag", 3: "tag", 4: "tag"},       # tags from the first filter on
    {1: "signal", 2: "signal", 3: "tag", 4: "tag"},    # ... from the second
    {1: "signal", 2: "signal", 3: "signal", 4: "tag"},  # ... only into the aggregate
    {1: "signal", 2: "signal", 3: "signal", 4: "signal"},  # every edge signalled (per-edge kernel)
    {1: "tag", 2: "tag", 3: "tag", 4: "tag"},          # every edge tagged (per-edge kernel)
    {1: "lane", 2: "lane", 3: "lane", 4: "lane"},      # per-lane selection everywhere
    {1: "lane", 2: "signal", 3: "lane", 4: "tag"},
    {1: "signal", 2: "lane", 3: "signal", 4: "lane"},
]


@pytest.mark.parametrize("mi", range(len(CASCADE_MODES)))
@pytest.mark.parametrize("mean", [1, 4, 32, 300])
def test_cascade_per_edge_modes(rs, mi, mean):
    # 128 items per ensemble: the per-edge kernel specialised for the cascade's ops
    s = wl.cascade_stream(n_total=1 << 18, mean=mean, seed=7)
    st = _check(rs, wl.pipeline_cascade(), s, CASCADE_MODES[mi], outputs=("count", "sum"))
    assert st["items"][1] == 1 << 18


@pytest.mark.parametrize("mi", [0, 5, 6])
def test_cascade_per_edge_modes_generic_kernel(rs, mi):
    # 64 items per ensemble: the generic per-edge kernel on the same stage list
    s = wl.cascade_stream(n_total=1 << 17, mean=24, seed=8)
    _check(rs, wl.pipeline_cascade(), s, CASCADE_MODES[mi], outputs=("count", "sum"), ensemble_width=64)


@pytest.mark.parametrize("W", [32, 64, 128])
@pytest.mark.parametrize("modes", [{1: "lane", 2: "lane", 3: "lane"}, {1: "signal", 2: "tag", 3: "tag"},
                                   {1: "lane", 2: "tag", 3: "tag"}])
def test_hashed_per_edge_modes_and_widths(rs, W, modes):
    s = wl.hashed_uniform_stream()
    st = _check(rs, wl.pipeline_hash_filter_map(), s, modes, ensemble_width=W)
    if W >= 64 and all(v == "lane" for v in modes.values()):
        # ensembles are not cut at region boundaries: node 1 fires fewer ensembles than
        # any signal-delimited schedule can (one per W elements of each region, rounded up)
        L = s["len"].astype(np.int64)
        assert st["ensembles"][1] < int(np.sum((L + W - 1) // W))


@pytest.mark.parametrize("modes", [{1: "lane", 2: "lane"}, {1: "signal", 2: "tag"}, {1: "tag", 2: "tag"}])
def test_graph_per_edge_modes(rs, modes):
    g = wl.graph_stream(V=1 << 13, E=1 << 17, cap=1 << 12, seed=7)
    _check(rs, wl.pipeline_graph_edges(), g, modes, outputs=("count", "min"))


def test_lane_selection_with_tiny_and_empty_regions(rs):
    """Many zero-credit signals per ensemble (empty regions, one-element regions), more
    than 32 signals inside one ensemble, and signal rings of minimum size."""
    rng = np.random.default_rng(5)
    L = rng.choice([0, 0, 0, 1, 2], size=50000).astype(np.uint32)
    n = int(L.sum())
    s = wl.make_stream(L, elements=wl.to_u32(wl.splitmix64_counter(3, 0, n)),
                       ctx=wl.to_u32(wl.splitmix64_counter(4, 0, L.shape[0])))
    pipe = [("enum_load",), ("filter_hash_ctx", 1, 3 << 30), ("map_mul", 3, 1), ("aggregate",)]
    for sc in (4, 32):
        _check(rs, pipe, s, {1: "lane", 2: "lane", 3: "lane"}, signal_capacity=sc)
        _check(rs, pipe, s, {1: "lane", 2: "signal", 3: "lane"}, signal_capacity=sc)


def test_expand_with_signal_and_tag_edges(rs):
    pipe = [("enum_hash",), ("expand", 3, 5), ("filter_mod", 3, 1), ("expand", 2, 8), ("aggregate",)]
    s = wl.hashed_uniform_stream(3000, 40, 6)
    _check(rs, pipe, s, {1: "signal", 2: "signal", 3: "tag", 4: "tag"})
    _check(rs, pipe, s, {1: "signal", 2: "lane", 3: "tag", 4: "tag"})


def test_lane_into_an_expansion_is_rejected(rs):
    pipe = [("enum_hash",), ("expand", 3, 5), ("aggregate",)]
    with pytest.raises(rs.RsError):
        rs.Pipeline(pipe, strategy="signal", boundary_modes={1: "lane"})
    with pytest.raises(rs.RsError):   # signals below a tagged edge
        rs.Pipeline(wl.pipeline_cascade(), strategy="signal",
                    boundary_modes={1: "tag", 2: "signal", 3: "tag", 4: "tag"})


@pytest.mark.parametrize("modes", [{1: "lane", 2: "lane"}, {1: "signal", 2: "tag"}, {1: "tag", 2: "tag"}])
def test_emit_sink_fed_by_lane_and_tag_edges(rs, modes):
    pipe = [("enum_load",), ("filter_hash_ctx", 1, 3 << 30), ("emit",)]
    s = wl.cascade_stream(n_total=1 << 17, mean=20, seed=3)
    L = s["len"].astype(np.int64)
    s = dict(s, len=None, offsets=np.concatenate(([0], np.cumsum(L))).astype(np.uint32))
    want = oracle.run_emit(pipe, s)
    got, st = rs.run_stream(pipe, s, strategy="signal", boundary_modes=modes)
    assert st["device_status"] == 0
    assert np.array_equal(got["count"], want["count"])
    for r in np.flatnonzero(want["count"]):
        a, b = want["start"][r], want["start"][r] + int(want["count"][r])
        assert np.array_equal(np.sort(got["values"][a:b]), np.sort(want["values"][a:b]))


TREES = [
    ([("enum_load",), ("filter_hash_ctx", 1, 2147483648), ("filter_hash_ctx", 2, 1288490188), ("aggregate",),
      ("aggregate",)], [0, 0, 1, 2, 1]),
    ([("enum_hash",), ("map_mul", 2654435761, 7), ("filter_mod", 2, 0), ("aggregate",), ("expand", 3, 11),
      ("aggregate",)], [0, 0, 1, 2, 1, 4]),
    ([("enum_hash",), ("expand", 2, 5), ("aggregate",), ("aggregate",)], [0, 0, 1, 1]),
]
TREE_MODES = [None, "signal", "tag", "lane_signal", "lane_tag"]


def _tree_modes(pipe, inputs, kind):
    if kind is None:
        return 0
    m = {}
    for c in range(1, len(pipe)):
        if kind == "signal":
            m[c] = "signal"
        elif kind == "tag":
            m[c] = "tag"
        elif kind == "lane_signal":
            # per-lane selection wherever the consumer is not an expansion
            m[c] = "signal" if pipe[c][0] == "expand" else "lane"
        else:
            # signals (or lane selection) into stage 1, tags below it
            m[c] = ("signal" if pipe[c][0] == "expand" else "lane") if c == 1 else "tag"
    return m


@pytest.mark.parametrize("mk", TREE_MODES)
@pytest.mark.parametrize("ti", range(len(TREES)))
def test_tree_topologies(rs, ti, mk):
    pipe, inputs = TREES[ti]
    s = wl.cascade_stream(n_total=1 << 17, mean=12, seed=4) if pipe[0][0] == "enum_load" else \
        wl.hashed_uniform_stream(4000, 48, 8)
    want = oracle.run_tree(pipe, inputs, s)
    got, st = rs.run_stream(pipe, s, strategy="signal", inputs=inputs, boundary_modes=_tree_modes(pipe, inputs, mk))
    assert st["device_status"] == 0
    for k in ("count", "sum", "min"):
        assert np.array_equal(got[k], want[0][k]), (k, 0)
        assert np.array_equal(got[k + "2"], want[1][k]), (k, 1)
    if mk in (None, "signal"):
        # Begin and End reach every node of the tree: both branches get every signal (a
        # region split between work units gets a pair in each piece)
        R = s["R"]
        for node in range(1, len(pipe)):
            assert st["signals"][node] == st["signals"][1], node
        assert st["signals"][1] >= 2 * R
        if pipe[0][0] == "enum_hash":
            assert st["signals"][1] == 2 * R      # whole-parent units: exactly one pair each


def test_lines_workload_all_variants(rs):
    """The taxi stand-in (lines of about 1,397 characters, about 45 candidates each) under
    the paper's three variants and per-lane selection: identical results."""
    s = wl.lines_stream(1 << 20)
    pipe = wl.pipeline_lines()
    for modes in ({1: "signal", 2: "signal", 3: "signal", 4: "signal"},
                  {1: "signal", 2: "tag", 3: "tag", 4: "tag"},
                  {1: "tag", 2: "tag", 3: "tag", 4: "tag"},
                  {1: "lane", 2: "lane", 3: "lane", 4: "lane"}):
        _check(rs, pipe, s, modes)
