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
        # the pipeline kernel on the same one-region stream agrees
        res, st = rs.run_stream(pipe, _one_region(el, ctx), strategy="tag", outputs=("count", "sum"))
        assert int(res["count"][0]) == int(got[0]) and int(res["sum"][0]) == int(got[1])


def test_calibration_argument_checks(rs):
    import torch
    el = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(rs.RsError):
        rs.calibrate_cascade(el, 0, [1, 2, 3], [1, 2, 3], out=out[1:].view(torch.int32)[1:])   # misaligned out
