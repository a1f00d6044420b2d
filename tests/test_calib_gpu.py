"""The calibration kernel (rs_calibrate_cascade) against the CPU oracle, bit-exact: the
cascade's three context-hash filters over ONE region are the cascade pipeline on a stream
of one region with that context word (Section 5's cascade; an aggregate's count and sum of
the survivors).  Sizes span many windows, a ragged tail, an unaligned start and no
elements at all."""
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


def _one_region(el, ctx):
    return wl.make_stream(np.array([el.shape[0]], dtype=np.uint32), elements=el,
                          ctx=np.array([ctx], dtype=np.uint32))


@pytest.mark.parametrize("n,offset", [(1 << 20, 0), ((1 << 20) + 37, 0), (100_003, 1), (300, 3), (1, 0), (0, 0)])
def test_calibration_equals_one_region_pipeline(rs, n, offset):
    import torch
    base = wl.cascade_stream(n_total=(1 << 20) + 64, mean=4096, seed=5)["elements"]
    el = np.ascontiguousarray(base[offset:offset + n])
    ctx = 0x1234ABCD
    pipe = wl.pipeline_cascade()
    want = oracle.run(pipe, _one_region(el, ctx)) if n else {"count": np.zeros(1), "sum": np.zeros(1)}
    dev = torch.from_numpy(base.view(np.int32).copy()).cuda()[offset:offset + n]   # offset: unaligned start
    salts = [st[1] for st in pipe[1:4]]
    thetas = [st[2] for st in pipe[1:4]]
    out = rs.calibrate_cascade(dev, ctx, salts, thetas)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.uint64)
    assert int(got[0]) == int(want["count"][0]) and int(got[1]) == int(want["sum"][0]), (got, want)
    if n >= 1 << 20:
        # the pipeline kernels on the same one-region stream agree: one region spans
        # hundreds of work units, whose records the planner's warp writes together
        for strategy in ("tag", "signal"):
            res, st = rs.run_stream(pipe, _one_region(el, ctx), strategy=strategy, outputs=("count", "sum"))
            assert st["device_status"] == 0, st
            assert int(res["count"][0]) == int(got[0]) and int(res["sum"][0]) == int(got[1]), strategy


@pytest.mark.parametrize("strategy", ["tag", "signal"])
def test_long_regions_among_short_ones(rs, strategy):
    """Regions of up to 2^18 elements (hundreds of units each) between short ones, as
    lengths and as CSR offsets: the planner writes a long region's unit records with the
    whole warp, a short one's with its lane."""
    rng = np.random.default_rng(17)
    L = rng.integers(0, 40, size=3000).astype(np.uint32)
    L[[5, 6, 700, 2999]] = [1 << 18, 100_000, 77_777, 1 << 17]
    el = wl.cascade_stream(n_total=int(L.sum()), mean=4096, seed=6)["elements"]
    ctx = rng.integers(0, 1 << 32, size=L.shape[0], dtype=np.uint64).astype(np.uint32)
    s = wl.make_stream(L, elements=el, ctx=ctx)
    pipe = wl.pipeline_cascade()
    want = oracle.run(pipe, s)
    off = np.concatenate(([0], np.cumsum(L.astype(np.int64)))).astype(np.uint32)
    for stream in (s, wl.make_stream(offsets=off, elements=el, ctx=ctx)):
        for rpu in ((64, 1024) if strategy == "tag" else (64, 256)):
            res, st = rs.run_stream(pipe, stream, strategy=strategy, outputs=("count", "sum"), regions_per_unit=rpu)
            assert st["device_status"] == 0, st
            for k in ("count", "sum"):
                assert np.array_equal(res[k], want[k]), (k, rpu)


def test_calibration_argument_checks(rs):
    import torch
    el = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(rs.RsError):
        rs.calibrate_cascade(el, 0, [1, 2, 3], [1, 2, 3], out=out[1:].view(torch.int32)[1:])   # misaligned out
