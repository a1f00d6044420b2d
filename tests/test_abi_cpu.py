"""The C ABI without a GPU: the library loads, exports every symbol include/rs.h
declares, and its host-side validation behaves as documented (no kernel runs)."""
import ctypes
import os
import re

import pytest

from paper_2006_07478_b300 import rs
from paper_2006_07478_b300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported():
    L = rs.lib()
    declared = _declared()
    assert "rs_run" in declared and "rs_pipeline_create" in declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(rs.EXPORTS) <= declared


def test_struct_mirrors_match_the_c_layout():
    """rs.lib() refuses a library whose structs differ from the ctypes mirrors; check the
    sizes it compared directly as well."""
    L = rs.lib()
    sizes = (ctypes.c_uint64 * 8)()
    assert L.rs_struct_sizes(sizes, 8) == 7
    assert list(sizes)[:7] == [ctypes.sizeof(c) for c in (rs.StageDesc, rs.Opts, rs.StreamDesc, rs.RegionResults,
                                                         rs.Stats, rs.Request, rs.ServerStats)]
    assert sizes[7] == 0                                   # nothing written past the known count
    assert L.rs_struct_sizes(None, 0) == 7


def test_version_and_status_strings():
    assert rs.lib().rs_version() >= 1
    assert rs.status_string(rs.RS_OK) == "ok"
    assert "invalid" in rs.status_string(rs.RS_ERR_INVALID)


def _create(stages, **opts):
    arr = (rs.StageDesc * len(stages))(*[rs.stage_desc(s) for s in stages])
    o = rs.make_opts(**opts)
    h = ctypes.c_void_p()
    st = rs.lib().rs_pipeline_create(arr, len(stages), ctypes.byref(o), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("pipe", [wl.pipeline_hash_filter_map(), wl.pipeline_cascade(), wl.pipeline_graph_edges(),
                                  [("enum_hash",), ("expand", 3, 7), ("aggregate",)]])
def test_valid_pipelines_create(pipe):
    st, h = _create(pipe)
    assert st == rs.RS_OK
    assert rs.lib().rs_pipeline_destroy(h) == rs.RS_OK


@pytest.mark.parametrize("pipe", [
    [("aggregate",)],                                                    # too short
    [("enum_hash",), ("filter_mod", 2, 0)],                              # no aggregate last
    [("filter_mod", 2, 0), ("aggregate",)],                              # no enumeration first
    [("enum_hash",), ("filter_mod", 0, 0), ("aggregate",)],              # modulus 0
    [("enum_hash",)] + [("map_mul", 1, 0)] * 5 + [("aggregate",)],       # too many stages
    [("enum_hash",), ("expand", 9, 1), ("aggregate",)],                  # fan-out > 8
])
def test_invalid_pipelines_rejected(pipe):
    st, h = _create(pipe)
    assert st == rs.RS_ERR_INVALID


def test_queue_capacity_must_hold_worst_case_output():
    # fan-out 4 at W = 128 needs >= 128 * 5 slots; 512 is too small, 1024 is fine
    st, _ = _create([("enum_hash",), ("expand", 4, 1), ("aggregate",)], queue_capacity=512)
    assert st == rs.RS_ERR_INVALID
    st, h = _create([("enum_hash",), ("expand", 4, 1), ("aggregate",)], queue_capacity=1024)
    assert st == rs.RS_OK
    rs.lib().rs_pipeline_destroy(h)
    st, _ = _create(wl.pipeline_cascade(), queue_capacity=96)      # not a power of two
    assert st == rs.RS_ERR_INVALID
    st, _ = _create(wl.pipeline_cascade(), tiles_in_flight=3)
    assert st == rs.RS_ERR_INVALID
    st, _ = _create(wl.pipeline_cascade(), ensemble_width=48)
    assert st == rs.RS_ERR_INVALID
    st, _ = _create(wl.pipeline_cascade(), ensemble_width=128, tile_elements=64)   # tile < W
    assert st == rs.RS_ERR_INVALID
    st, _ = _create(wl.pipeline_cascade(), region_cost=24)                          # not a power of two
    assert st == rs.RS_ERR_INVALID
    st, _ = _create(wl.pipeline_cascade(), region_cost=512)                         # above 256
    assert st == rs.RS_ERR_INVALID
    st, h = _create(wl.pipeline_cascade(), region_cost=1, regions_per_unit=256)
    assert st == rs.RS_OK
    rs.lib().rs_pipeline_destroy(h)
    # flags: RS_FLAG_UNBALANCED_UNITS | RS_FLAG_PRIVATE_WORKSPACE, nothing else
    st, h = _create(wl.pipeline_cascade(), flags=rs.FLAG_UNBALANCED_UNITS | rs.FLAG_PRIVATE_WORKSPACE)
    assert st == rs.RS_OK
    rs.lib().rs_pipeline_destroy(h)
    st, _ = _create(wl.pipeline_cascade(), flags=4)
    assert st == rs.RS_ERR_INVALID


def test_stream_submit_validation_and_workspace_size():
    st, h = _create(wl.pipeline_cascade())
    assert st == rs.RS_OK
    L = rs.lib()
    d = rs.StreamDesc()
    d.n_regions = 10
    sid = ctypes.c_uint64()
    # no lengths and no offsets
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_ERR_INVALID
    d.region_len = ctypes.c_void_p(0x1000)
    # loading enumeration without elements
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_ERR_INVALID
    d.elements = ctypes.c_void_p(0x2000)
    d.n_elements = 1 << 32
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_ERR_CAPACITY
    d.n_elements = 1000
    d.out_count = ctypes.c_void_p(0x3000)
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_OK
    assert sid.value == 0
    n = ctypes.c_uint64()
    assert L.rs_workspace_size(h, ctypes.byref(n)) == rs.RS_OK
    # header + one look-back word per unit + the stream table, each 256-byte aligned
    assert n.value >= 256 and n.value % 256 == 0
    # running without a workspace is an argument error, caught before any CUDA call
    assert L.rs_run(h, None, 0, None) == rs.RS_ERR_INVALID
    assert L.rs_clear_streams(h) == rs.RS_OK
    assert L.rs_graph_launch(h, None) == rs.RS_ERR_NOT_READY
    assert L.rs_pipeline_destroy(h) == rs.RS_OK


def test_calibration_argument_checks_without_gpu():
    L = rs.lib()
    s3 = (ctypes.c_uint32 * 3)(1, 2, 3)
    # no output array, or elements missing for n > 0: argument errors before any CUDA call
    assert L.rs_calibrate_cascade(None, 0, 0, s3, s3, None, None) == rs.RS_ERR_INVALID
    assert L.rs_calibrate_cascade(None, 10, 0, s3, s3, ctypes.c_void_p(0x1000), None) == rs.RS_ERR_INVALID
    assert L.rs_calibrate_cascade(ctypes.c_void_p(0x2000), 10, 0, s3, s3, ctypes.c_void_p(0x1004), None) == \
        rs.RS_ERR_INVALID


def test_opts_round_trip():
    p = rs.Pipeline(wl.pipeline_cascade(), strategy="signal", queue_capacity=512, regions_per_unit=16)
    o = p.opts
    assert o["strategy"] == 0 and o["queue_capacity"] == 512 and o["regions_per_unit"] == 16
    p.set_opts(strategy="tag", warps_per_block=8)
    assert p.opts["strategy"] == 1 and p.opts["warps_per_block"] == 8
    # the binding's workspace is the pipeline's own tensor: the flag stays set
    assert p.opts["flags"] == rs.FLAG_PRIVATE_WORKSPACE
    p.set_opts(flags=rs.FLAG_UNBALANCED_UNITS)
    assert p.opts["flags"] == rs.FLAG_UNBALANCED_UNITS | rs.FLAG_PRIVATE_WORKSPACE
    with pytest.raises(rs.RsError):
        p.set_opts(warps_per_block=16)
    with pytest.raises(rs.RsError):
        p.set_opts(regions_per_unit=70000)
    p.close()


def test_server_argument_checks_without_gpu():
    L = rs.lib()
    pipe = wl.pipeline_hash_filter_map()
    arr = (rs.StageDesc * len(pipe))(*[rs.stage_desc(s) for s in pipe])
    o = rs.make_opts()
    h = ctypes.c_void_p()
    # no arena / unaligned arena / too small arena
    assert L.rs_server_create(arr, len(pipe), ctypes.byref(o), None, 1 << 20, 0, 0, None, ctypes.byref(h)) == \
        rs.RS_ERR_INVALID
    assert L.rs_server_create(arr, len(pipe), ctypes.byref(o), ctypes.c_void_p(0x1001), 1 << 20, 0, 0, None,
                              ctypes.byref(h)) == rs.RS_ERR_INVALID
    assert L.rs_server_create(arr, len(pipe), ctypes.byref(o), ctypes.c_void_p(0x1000), 1024, 0, 0, None,
                              ctypes.byref(h)) == rs.RS_ERR_INVALID
    # a valid server (the arena address is never touched without work)
    assert L.rs_server_create(arr, len(pipe), ctypes.byref(o), ctypes.c_void_p(0x100000), 1 << 20, 0, 0, None,
                              ctypes.byref(h)) == rs.RS_OK
    r = rs.Request()
    r.n_regions = 1 << 20          # needs more than half the arena
    r.region_len = ctypes.c_void_p(0x2000)
    r.out_count = ctypes.c_void_p(0x3000)
    rid = ctypes.c_uint64()
    assert L.rs_server_submit(h, ctypes.byref(r), ctypes.byref(rid)) == rs.RS_ERR_CAPACITY
    r.n_regions = 16
    assert L.rs_server_submit(h, ctypes.byref(r), ctypes.byref(rid)) == rs.RS_OK
    st = rs.ServerStats()
    assert L.rs_server_get_stats(h, ctypes.byref(st)) == rs.RS_OK and st.submitted == 1


def test_emit_sink_pipelines_and_streams():
    """An emit sink is a legal last stage; its streams need CSR offsets, counts and a
    value array; the server does not take emit pipelines (its requests carry per-region
    outputs only)."""
    pipe = wl.pipeline_cascade()[:-1] + [("emit",)]
    st, h = _create(pipe)
    assert st == rs.RS_OK
    L = rs.lib()
    d = rs.StreamDesc()
    d.n_regions = 10
    d.region_len = ctypes.c_void_p(0x1000)
    d.elements = ctypes.c_void_p(0x2000)
    d.n_elements = 1000
    d.out_count = ctypes.c_void_p(0x3000)
    sid = ctypes.c_uint64()
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_ERR_INVALID   # no offsets
    d.region_offsets = ctypes.c_void_p(0x4000)
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_ERR_INVALID   # no values
    d.out_values = ctypes.c_void_p(0x5000)
    d.out_values_len = 1000
    assert L.rs_stream_submit(h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_OK
    assert L.rs_pipeline_destroy(h) == rs.RS_OK
    st, h = _create([("enum_load",), ("emit",), ("aggregate",)])                             # emit is last only
    assert st == rs.RS_ERR_INVALID
    arr = (rs.StageDesc * len(pipe))(*[rs.stage_desc(s) for s in pipe])
    srv = ctypes.c_void_p()
    assert L.rs_server_create(arr, len(pipe), None, ctypes.c_void_p(0x10000), 1 << 20, 0, 0, None,
                              ctypes.byref(srv)) == rs.RS_ERR_INVALID


def test_tree_topologies_and_boundary_modes_are_validated():
    tree = [("enum_load",), ("filter_hash_ctx", 1, 5), ("filter_hash_ctx", 2, 5), ("aggregate",), ("aggregate",)]

    def create(stages, inputs, **opts):
        descs = [rs.stage_desc(s) for s in stages]
        for i in range(1, len(descs)):
            descs[i].input = inputs[i]
        arr = (rs.StageDesc * len(stages))(*descs)
        o = rs.make_opts("signal", **opts)
        h = ctypes.c_void_p()
        st = rs.lib().rs_pipeline_create(arr, len(stages), ctypes.byref(o), ctypes.byref(h))
        if st == rs.RS_OK:
            rs.lib().rs_pipeline_destroy(h)
        return st

    assert create(tree, [0, 0, 1, 2, 1]) == rs.RS_OK
    assert create(tree, [0, 0, 1, 2, 3]) == rs.RS_ERR_INVALID       # reads a sink
    assert create(tree, [0, 0, 1, 1, 1]) == rs.RS_ERR_INVALID       # stage 2 is a leaf but not a sink
    assert create(tree, [0, 2, 1, 2, 1]) == rs.RS_ERR_INVALID       # stage 1 must read the enumeration
    three = tree[:4] + [("aggregate",), ("aggregate",)]
    assert create(three, [0, 0, 1, 2, 1, 1]) == rs.RS_ERR_INVALID   # more than RS_MAX_SINKS leaves
    emit_tree = tree[:4] + [("emit",)]
    assert create(emit_tree, [0, 0, 1, 2, 1]) == rs.RS_ERR_INVALID  # an emit sink ends a linear pipeline
    cas = wl.pipeline_cascade()
    lin = [0, 0, 1, 2, 3]
    assert create(cas, lin, boundary_modes=rs.boundary_modes({1: "signal", 2: "tag", 3: "tag", 4: "tag"})) == rs.RS_OK
    assert create(cas, lin, boundary_modes=rs.boundary_modes({1: "lane", 2: "lane", 3: "lane", 4: "lane"})) == rs.RS_OK
    assert create(cas, lin, boundary_modes=rs.boundary_modes({1: "tag", 2: "signal", 3: "tag", 4: "tag"})) == \
        rs.RS_ERR_INVALID                                           # signals below a tagged edge
    assert create(cas, lin, boundary_modes=1) == rs.RS_ERR_INVALID  # the enumeration has no input edge
    ex = [("enum_hash",), ("expand", 3, 1), ("aggregate",)]
    assert create(ex, [0, 0, 1], boundary_modes=rs.boundary_modes({1: "lane"})) == rs.RS_ERR_INVALID
    assert create(ex, [0, 0, 1], boundary_modes=rs.boundary_modes({1: "tag", 2: "tag"})) == rs.RS_OK
    arr = (rs.StageDesc * 5)(*[rs.stage_desc(s) for s in tree])
    arr[4].input = 1
    srv = ctypes.c_void_p()
    assert rs.lib().rs_server_create(arr, 5, None, ctypes.c_void_p(0x10000), 1 << 20, 0, 0, None,
                                     ctypes.byref(srv)) == rs.RS_ERR_INVALID   # the server serves linear pipelines
