"""The committed ncu summaries that bench.py reads: the DRAM-traffic file parses, names the
kernel sources it was taken on, and holds one row per mean region length of the cascade."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_file_parses():
    path = os.path.join(ROOT, "profiles", "dram_traffic_cascade.txt")
    src, rows = None, {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("kernel_source"):
                src = line.split()[1]
            elif line.startswith("mean="):
                kv = dict(tok.split("=", 1) for tok in line.split())
                rows[int(kv["mean"])] = kv
    assert src and len(src) == 16
    assert sorted(rows) == [1, 4, 32, 256, 4096]
    for m, kv in rows.items():
        dram = int(kv["dram_bytes"])
        assert dram == int(kv["read"]) + int(kv["write"])
        assert dram == int(kv["planner_bytes"]) + int(kv["kernel_bytes"])
        # at least the algorithmic bytes of a 2^26-element run moved, and not wildly more
        assert 0.95 <= float(kv["ratio_to_alg"]) <= 3.0


def test_bench_reads_traffic_when_sources_match():
    rows = bench.read_traffic()
    if rows is None:          # kernel sources changed since the capture: bench reports null
        return
    assert sorted(m for m, _ in rows) == [1, 4, 32, 256, 4096]
    assert all(v > 4 * (1 << 26) for v in rows.values())
