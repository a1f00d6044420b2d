"""rs_run_noalloc, the workspace-free entry point, through the C ABI (GPU).

Some callers cannot allocate device memory when they run a pipeline: an application
that owns the whole device-memory budget through its own allocator or a hard cap, or
a latency-critical loop in which an allocation could synchronise the device.
rs_run_noalloc serves them: it runs the same kernels as rs_run, with the scratch
memory in a fixed 16 MiB array inside the library, and allocates nothing.  Its
per-region results must equal rs_run's exactly (all arithmetic is integer, the
tolerance of every parity test here), on two calls in a row, since the second call
finds the previous call's contents in the shared array.
"""
import ctypes

import numpy as np
import pytest

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


CASES = [
    (wl.pipeline_cascade(), lambda: wl.cascade_stream(n_total=1 << 20, mean=32, seed=7), ("count", "sum"), "tag"),
    (wl.pipeline_cascade(), lambda: wl.cascade_stream(n_total=1 << 19, mean=2000, seed=3), ("count", "sum"), "signal"),
    (wl.pipeline_hash_filter_map(), lambda: wl.hashed_uniform_stream(), ("count", "sum", "min"), "signal"),
    (wl.pipeline_graph_edges(), lambda: wl.graph_stream(V=1 << 12, E=1 << 17, cap=1 << 12, seed=7),
     ("count", "min"), "tag"),
]


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_noalloc_equals_run_on_two_calls(rs, ci):
    import torch
    pipe, make, outputs, strategy = CASES[ci]
    p = rs.Pipeline(pipe, strategy=strategy)
    out = p.submit(rs.to_device(make()), outputs=outputs)
    p.run()
    torch.cuda.synchronize()
    want = rs.results_to_numpy(out)
    for _ in range(2):
        for k in outputs:
            out[k].fill_(-1)
        p.run_noalloc()
        torch.cuda.synchronize()
        got = rs.results_to_numpy(out)
        for k in outputs:
            assert np.array_equal(got[k], want[k]), k
    p.close()


def test_noalloc_scratch_need_is_reported_without_a_run(rs):
    """The size rule on the host alone: a loaded stream of 2^31 parents needs more than
    the fixed 16 MiB of scratch under any unit shape (its planner alone keeps one 8-byte
    look-back word per 1024 parents).  Only host-side calls see this descriptor, whose
    pointers are placeholders; nothing is run with it."""
    p = rs.Pipeline(wl.pipeline_cascade(), strategy="tag")
    d = rs.StreamDesc()
    d.n_regions = 1 << 31
    d.region_len = ctypes.c_void_p(0x1000)
    d.elements = ctypes.c_void_p(0x2000)
    d.n_elements = 1 << 27
    d.out_count = ctypes.c_void_p(0x3000)
    sid = ctypes.c_uint64()
    assert rs.lib().rs_stream_submit(p._h, ctypes.byref(d), ctypes.byref(sid)) == rs.RS_OK
    assert p.workspace_bytes() > 16 << 20
    p.close()


def test_noalloc_rejects_scratch_beyond_its_fixed_size(rs):
    """A real stream whose scratch needs more than the fixed 16 MiB: 2^21 regions of 8
    elements cut into merge-path units of one step each (2^21 * 9 units of 16 bytes of
    unit records, about 300 MB).  The call returns RS_ERR_CAPACITY with nothing enqueued,
    and the outputs keep their sentinel."""
    import torch
    R = 1 << 21
    lens = np.full(R, 8, dtype=np.uint32)
    s = wl.make_stream(lens, elements=np.arange(8 * R, dtype=np.uint32), ctx=np.zeros(R, dtype=np.uint32))
    p = rs.Pipeline(wl.pipeline_cascade(), strategy="tag", regions_per_unit=1, region_cost=1)
    out = p.submit(rs.to_device(s), outputs=("count", "sum"))
    out["count"].fill_(-7)
    assert p.workspace_bytes() > 16 << 20
    assert rs.lib().rs_run_noalloc(p._h, None) == rs.RS_ERR_CAPACITY
    torch.cuda.synchronize()
    assert bool((out["count"] == -7).all())
    p.close()
