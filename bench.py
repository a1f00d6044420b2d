"""Benchmark: input items/s of the region-segmented cascade on B300, with the
fraction of HBM peak per mean region size.

One step = one pass of the pipeline (enumerate -> three context-dependent hash
filters -> per-region count+sum) over five seeded streams of 2^26 uint32 elements
each, cut into geometric regions of mean 1, 4, 32, 256 and 4096 (seed 7); each
stream runs with the region strategy and unit size the library's autotuner picked
for it.  Inputs are device-resident and each stream's 256 MiB element array is
larger than L2, and the five streams alternate, so no launch reuses the previous
launch's lines.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs the same five streams on
its own GPU (weak scaling, no data-path collective); value = all ranks' items /
the slowest rank's time.  `--impl reference` times the CPU oracle (the plain
sequential definition) on the host cores instead.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2006_07478_b300 import workloads as wl  # noqa: E402

METRIC = "input items/s & fraction of HBM peak vs mean region size; p50/p99 stream latency"
MEANS = (1, 4, 32, 256, 4096)
N_ELEM = 1 << 26
SEED = 7
SPEC_HBM_GBS = 8000.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def alg_bytes(stream) -> int:
    """Algorithmic HBM bytes of one pass: every element read once (4 B), and per
    region its length and context word read and its count (4 B) and sum (8 B)
    written."""
    return 4 * wl.n_elements(stream) + 20 * int(stream["R"])


def make_streams():
    return [wl.cascade_stream(n_total=N_ELEM, mean=m, seed=SEED) for m in MEANS]


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._reader, daemon=True)
        self.thread.start()

    def _reader(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float) -> dict:
        rows = []
        for t, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            rows.append((t, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1]
        used = inside if inside else [r for r in rows if t0 - 0.5 <= r[0] <= t1 + 0.5]
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(p[0]) for _, p in used if p[0].replace(".", "", 1).isdigit()]
        smax = [float(p[1]) for _, p in used if p[1].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, p in used:
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(used), "samples_in_timed_region": len(inside)}


# ---------------------------------------------------------------------------
# the oracle on the host cores

def time_oracle(streams, threads: int, budget_s: float = 20.0):
    """Run the CPU oracle over the streams (whole streams, in order) until the
    budget is spent; returns (items, seconds, streams_done)."""
    from oracle import oracle
    pipe = wl.pipeline_cascade()
    items, secs, done = 0, 0.0, 0
    for s in streams:
        t = time.perf_counter()
        oracle.run(pipe, s, threads=threads)
        secs += time.perf_counter() - t
        items += N_ELEM
        done += 1
        if secs > budget_s:
            break
    return items, secs, done


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    streams = make_streams()
    threads = os.cpu_count() or 1
    from oracle import oracle
    oracle.build()
    for _ in range(args.warmup):
        time_oracle(streams[:1], threads, budget_s=0.0)
    times, items = [], 0
    for _ in range(args.steps):
        it, secs, done = time_oracle(streams, threads, budget_s=1e9)
        times.append(secs)
        items += it
    total = sum(times)
    value = items / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "items/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded)",
        "config": {"workload": "cascade: 5 streams x 2^26 u32 elements, geometric regions mean 1/4/32/256/4096, "
                               "3 context hash filters (pass 0.5/0.3/0.1), count+sum per region", "seed": SEED},
        "cpu_baseline": {"value": value, "unit": "items/s", "cores": threads, "kind": "oracle",
                         "sample": "the whole workload each step (5 x 2^26 elements)"},
        "e2e": {"value": value, "unit": "items/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for fn in ("rs_tag.cuh", "rs_tag.cu", "rs_tag2.cu", "rs_kernel.cu", "rs_device.cuh", "rs_internal.h", "rs_api.cu"):
        with open(os.path.join(ROOT, "paper_2006_07478_b300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_traffic():
    """DRAM bytes of one run (planner + pipeline kernel, the pair the roofline times) per
    mean, from the committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_cascade.txt")
    try:
        rows = {}
        src = None
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line.startswith("kernel_source"):
                    src = line.split()[1]
                elif line.startswith("mean="):
                    kv = dict(tok.split("=", 1) for tok in line.split())
                    rows[(int(kv["mean"]), kv["strategy"])] = float(kv["dram_bytes"])
        if src != kernel_source_hash():
            return None
        return rows
    except Exception:
        return None


def bench_graph(rs, torch, peak):
    """Graph-edge stream: 2^22 vertices, 2^26 edges (Zipf hubs); items = edges."""
    g = wl.graph_stream()
    E, V = wl.n_elements(g), g["R"]
    p = rs.Pipeline(wl.pipeline_graph_edges(), strategy="auto")
    out = p.submit(rs.to_device(g), outputs=("count", "min"))
    best, _ = p.autotune(trials=2)
    p.timing_enable(16)
    for _ in range(3):
        p.run()
    torch.cuda.synchronize()
    p.timing_read()
    for _ in range(7):
        p.run()
    kms = statistics.median(p.timing_read())
    st = p.stats()
    # invariants of the result (exactness against the oracle is tested in tests/): no vertex
    # keeps more edges than it has, the counts add up to the items the aggregate consumed,
    # and min dst is a vertex id exactly where an edge survived
    got = rs.results_to_numpy(out)
    deg = np.diff(g["offsets"].astype(np.int64))
    cnt = got["count"].astype(np.int64)
    mn = got["min"].astype(np.uint32)
    inv = bool(np.all(cnt <= deg) and int(cnt.sum()) == st["items"][-1] and
               np.all((mn == 0xFFFFFFFF) == (cnt == 0)) and np.all(mn[cnt > 0] < V))
    ab = 4 * E + 4 * (V + 1) + 8 * V
    p.close()
    return {"workload": "graph: 2^22 vertices, 2^26 edges, Zipf(2.1) out-degree capped at 2^16; keep w(dst)<w(src); "
                        "count and min dst per vertex",
            "kernel_ms": kms, "items_per_s": E / (kms * 1e-3), "alg_gbs": ab / (kms * 1e-3) / 1e9,
            "frac_of_measured_hbm": ab / (kms * 1e-3) / 1e9 / peak, "max_degree": int(np.diff(g["offsets"]).max()),
            "chosen": {"strategy": "signal" if best["strategy"] == 0 else "tag",
                       "regions_per_unit": best["regions_per_unit"], "ensemble_width": best["ensemble_width"]},
            "active_lane_fraction": [round(x, 4) for x in st["active_lane_fraction"]],
            "invariants_ok": inv}


def bench_region_sizes(rs, torch):
    """The paper's region-sum benchmark (Section 5, Figures figFixed and figVariable): one
    2^26-element array, enumerate + sum per region, regions of a fixed size or of sizes
    uniform on 0..max; both strategies at their default options.  Per size: time per run,
    items/s and node 1's active-lane fraction (signals cut ensembles at region boundaries,
    tags do not).  With no filter every region's count is its length, and the sums add up
    to the sum of the array."""
    n = N_ELEM
    base = wl.sized_region_stream(n, 128, seed=11)
    dev_el = torch.from_numpy(base["elements"].view(np.int32)).cuda()
    pipe = wl.pipeline_region_sum()
    sizes = [(s, False) for s in (16, 32, 64, 96, 127, 128, 129, 192, 256, 257, 384, 512, 1024, 2048)]
    sizes += [(s, True) for s in (64, 256, 1024)]
    rows, inv = [], True
    total = int(base["elements"].astype(np.uint64).sum())
    for size, variable in sizes:
        L = wl.sized_lengths(n, size, 11, variable)
        dev = {"R": int(L.shape[0]), "len": torch.from_numpy(L.view(np.int32)).cuda(), "elements": dev_el}
        row = {"size": size, "variable": variable, "regions": int(L.shape[0])}
        for strat in ("tag", "signal"):
            p = rs.Pipeline(pipe, strategy=strat)
            out = p.submit(dev, outputs=("count", "sum"))
            p.timing_enable(8)
            for _ in range(3):
                p.run()
            torch.cuda.synchronize()
            p.timing_read()
            for _ in range(5):
                p.run()
            ms = statistics.median(p.timing_read())
            st = p.stats()
            row[strat] = {"ms": ms, "items_per_s": n / (ms * 1e-3),
                          "active_lane_fraction_node1": st["active_lane_fraction"][1]}
            got = rs.results_to_numpy(out)
            inv &= bool(np.array_equal(got["count"], L) and int(got["sum"].astype(np.uint64).sum()) == total)
            p.close()
        rows.append(row)
    return {"workload": "region sum: 2^26 u32 elements, fixed region sizes 16..2048 and sizes U{0..64/256/1024}; "
                        "enumerate -> aggregate (count, sum); default options",
            "rows": rows, "invariants_ok": inv}


def _timed(p, torch, warm=2, reps=5):
    """Median kernel time (planner + pipeline kernel + finalize, CUDA events on the
    launching stream) of `reps` runs after `warm`, and the last run's statistics."""
    p.timing_enable(warm + reps + 2)
    for _ in range(warm):
        p.run()
    torch.cuda.synchronize()
    p.timing_read()
    for _ in range(reps):
        p.run()
    ms = statistics.median(p.timing_read())
    return ms, p.stats()


LANE4 = {1: "lane", 2: "lane", 3: "lane", 4: "lane"}
SIG4 = {1: "signal", 2: "signal", 3: "signal", 4: "signal"}
TAG4 = {1: "tag", 2: "tag", 3: "tag", 4: "tag"}


def bench_modes(rs, torch, cascades):
    """Per-stage strategy mixing (Section 5, the taxi application), per-lane state
    selection (Section 6), a tree topology (Figure 1(b)) and the emit sink (Section 4).
    Every variant of a workload must give the same results (compared here; exactness
    against the oracle is tested in tests/)."""
    res = {}
    # ---- lines: the taxi stand-in, the paper's three variants and per-lane selection ----
    s = wl.lines_stream(N_ELEM)
    pipe = wl.pipeline_lines()
    dev = rs.to_device(s)
    variants = [
        ("both stages enumerated: signals on every edge", "signal", SIG4),
        ("stage 1 enumerated, tags after it (mixed)", "signal", {1: "signal", 2: "tag", 3: "tag", 4: "tag"}),
        ("neither stage enumerated: tags on every edge", "signal", TAG4),
        ("per-lane selection on every edge", "signal", LANE4),
        ("per-lane selection into stage 1, tags after it", "signal", {1: "lane", 2: "tag", 3: "tag", 4: "tag"}),
        ("tag kernel (linear pipelines, every edge tagged)", "tag", None),
        ("signal kernel (linear pipelines, every edge signalled)", "signal", None),
    ]
    rows, ref, same = [], None, True
    for name, strat, modes in variants:
        p = rs.Pipeline(pipe, strategy=strat, boundary_modes=modes or 0)
        o = p.submit(dev)
        ms, st = _timed(p, torch)
        got = rs.results_to_numpy(o)
        if ref is None:
            ref = got
        same &= all(np.array_equal(got[k], ref[k]) for k in ref)
        rows.append({"variant": name, "kernel_ms": ms, "items_per_s": N_ELEM / (ms * 1e-3),
                     "active_lane_fraction": [round(x, 4) for x in st["active_lane_fraction"]],
                     "ensembles": st["ensembles"], "signals": st["signals"]})
        p.close()
    p = rs.Pipeline(pipe, strategy="auto")
    p.submit(dev)
    best, best_ms = p.autotune(trials=2)
    p.close()
    res["lines"] = {"workload": f"{s['R']} lines of U{{1..2793}} characters (mean 1397), 2^26 in all; "
                                "keep ~45 candidates per line (context hash), verify 90%, parse (map); "
                                "count/sum/min per line",
                    "variants": rows, "results_identical": bool(same),
                    "autotuned": {"strategy": best["strategy"], "boundary_modes": best["boundary_modes"],
                                  "ensemble_width": best["ensemble_width"], "ms": best_ms}}
    # ---- occupancy against overhead by mean region size, on the per-edge kernel ----
    sweep = []
    for m, cs in cascades:
        dv = rs.to_device(cs)
        row, ref = {"mean": m}, None
        for name, modes in (("signal", SIG4), ("lane", LANE4), ("tag", TAG4)):
            p = rs.Pipeline(wl.pipeline_cascade(), strategy="signal", boundary_modes=modes)
            o = p.submit(dv, outputs=("count", "sum"))
            ms, st = _timed(p, torch, reps=3)
            got = rs.results_to_numpy(o)
            ref = got if ref is None else ref
            row[name] = {"kernel_ms": ms, "items_per_s": N_ELEM / (ms * 1e-3),
                         "active_lane_fraction_node1": round(st["active_lane_fraction"][1], 4),
                         "identical": bool(all(np.array_equal(got[k], ref[k]) for k in ref))}
            p.close()
        sweep.append(row)
        del dv
    res["mean_sweep_per_edge_kernel"] = sweep
    # ---- a tree: one filter feeding a second filter's aggregate and an aggregate of its own ----
    m, cs = cascades[1]
    dv = rs.to_device(cs)
    tree = [("enum_load",), ("filter_hash_ctx", 1, wl.CASCADE_THETAS[0]), ("filter_hash_ctx", 2, wl.CASCADE_THETAS[1]),
            ("aggregate",), ("aggregate",)]
    inputs = [0, 0, 1, 2, 1]
    trow, ref = {"mean": m, "inputs": inputs}, None
    for name, modes in (("signal", SIG4), ("lane", LANE4), ("tag", TAG4)):
        p = rs.Pipeline(tree, strategy="signal", inputs=inputs, boundary_modes=modes)
        o = p.submit(dv, outputs=("count", "sum"))
        ms, st = _timed(p, torch, reps=3)
        got = rs.results_to_numpy(o)
        ref = got if ref is None else ref
        trow[name] = {"kernel_ms": ms, "items_per_s": N_ELEM / (ms * 1e-3),
                      "signals_per_node": st["signals"],
                      "identical": bool(all(np.array_equal(got[k], ref[k]) for k in ref))}
        p.close()
    res["tree"] = trow
    # ---- the emit sink against the aggregate (tag kernel), CSR offsets ----
    L = cs["len"].astype(np.int64)
    csr = dict(cs, len=None, offsets=np.concatenate(([0], np.cumsum(L))).astype(np.uint32))
    dvc = rs.to_device(csr)
    erow = {"mean": m}
    for name, pp in (("aggregate", wl.pipeline_cascade()), ("emit", wl.pipeline_cascade()[:-1] + [("emit",)])):
        p = rs.Pipeline(pp, strategy="tag")
        o = p.submit(dvc, outputs=("count", "sum"))
        ms, st = _timed(p, torch, reps=3)
        erow[name] = {"kernel_ms": ms, "items_per_s": N_ELEM / (ms * 1e-3)}
        if name == "emit":
            got = rs.results_to_numpy(o)
            erow["emit_count_total"] = int(got["count"].astype(np.int64).sum())
        else:
            erow["aggregate_count_total"] = int(rs.results_to_numpy(o)["count"].astype(np.int64).sum())
        p.close()
    res["emit"] = erow
    return res


def bench_calibration(rs, torch, dev, peak, tag_ms_4096):
    """The calibration kernel (rs_calibrate_cascade): the cascade's three filters, queues
    and compaction on the bench's 2^26 elements as ONE region, with no region handling --
    an upper bound for the pipeline kernels on these elements -- beside the tag kernel on
    the same one-region stream and on the mean-4096 stream."""
    el = dev["elements"]
    n = int(el.numel())
    pipe = wl.pipeline_cascade()
    salts = [st[1] for st in pipe[1:4]]
    thetas = [st[2] for st in pipe[1:4]]
    ctx = 0x1234ABCD
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        rs.calibrate_cascade(el, ctx, salts, thetas, out=out)
    ms = []
    for _ in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs.calibrate_cascade(el, ctx, salts, thetas, out=out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    cal_ms = statistics.median(ms)
    cal = out.cpu().numpy().astype(np.uint64)
    # the tag kernel on the same elements as one region with the same context word
    one = {"R": 1, "len": torch.tensor([n], dtype=torch.int32, device="cuda"), "offsets": None, "parents": None,
           "elements": el, "ctx": torch.tensor([ctx - (1 << 32) if ctx >= 1 << 31 else ctx], dtype=torch.int32,
                                               device="cuda"), "total_elements": n}
    p = rs.Pipeline(pipe, strategy="tag")
    o = p.submit(one, outputs=("count", "sum"))
    p.autotune(trials=2)
    one_ms, _ = _timed(p, torch, reps=5)
    got = rs.results_to_numpy(o)
    p.close()
    b = 4 * n
    return {"elements": n, "ctx": ctx,
            "calibration_ms": cal_ms, "calibration_gbs": b / (cal_ms * 1e-3) / 1e9,
            "calibration_frac_of_measured_hbm": b / (cal_ms * 1e-3) / 1e9 / peak,
            "tag_kernel_one_region_ms": one_ms,
            "tag_kernel_one_region_gbs": b / (one_ms * 1e-3) / 1e9,
            "tag_kernel_mean4096_ms": tag_ms_4096,
            "same_results": bool(int(cal[0]) == int(got["count"][0]) and int(cal[1]) == int(got["sum"][0]))}


def bench_batched(rs, torch):
    """4,096 independent hashed streams (lognormal sizes): one persistent launch for all
    of them replayed from a CUDA graph, against one launch per stream."""
    streams = wl.batched_streams()
    pipe = wl.pipeline_hash_filter_map()
    items = sum(wl.n_elements(s) for s in streams)
    devs = [rs.to_device(s) for s in streams]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        p = rs.Pipeline(pipe, strategy="auto")
        outs = [p.submit(d) for d in devs]
        best, _ = p.autotune(trials=1)
        p.graph_capture()
        for _ in range(3):
            p.graph_launch()
        side.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(side)
        for _ in range(reps):
            p.graph_launch()
        e1.record(side)
        side.synchronize()
        one_ms = e0.elapsed_time(e1) / reps
        # one launch per stream: the same work, a pipeline (and workspace) per stream
        singles = []
        for d in devs:
            q = rs.Pipeline(pipe, strategy=("signal" if best["strategy"] == 0 else "tag"),
                            regions_per_unit=best["regions_per_unit"], ensemble_width=best["ensemble_width"])
            q.submit(d)
            q.workspace()
            singles.append(q)
        for q in singles[:64]:
            q.run()
        side.synchronize()
        t0 = time.perf_counter()
        e0.record(side)
        for q in singles:
            q.run()
        e1.record(side)
        side.synchronize()
        per_ms = e0.elapsed_time(e1)
        per_wall = (time.perf_counter() - t0) * 1e3
        # the same one-launch-per-stream work with little host time between launches: each
        # stream's run captured in a graph of its own, the 4096 graphs replayed back to back
        for q in singles:
            q.graph_capture()
        for q in singles[:64]:
            q.graph_launch()
        side.synchronize()
        t1 = time.perf_counter()
        e0.record(side)
        for q in singles:
            q.graph_launch()
        e1.record(side)
        side.synchronize()
        per_graph_ms = e0.elapsed_time(e1)
        per_graph_wall = (time.perf_counter() - t1) * 1e3
        for q in singles:
            q.graph_release()
    # invariants of the results (exactness against the oracle is tested in tests/): no
    # region keeps more items than it has, and the counts over all streams add up to the
    # items the aggregate consumed in the last batched run
    p.graph_launch()
    torch.cuda.synchronize()
    st = p.stats()
    kept = 0
    exact = True
    for i, s in enumerate(streams):
        got = rs.results_to_numpy(outs[i])
        c = got["count"].astype(np.int64)
        exact &= bool(np.all(c <= s["len"].astype(np.int64)))
        kept += int(c.sum())
    exact &= kept == st["items"][-1]
    for q in singles:
        q.close()
    p.graph_release()
    p.close()
    return {"workload": "4096 hashed streams, sizes lognormal(median 2^14, sigma 1.5, cap 2^22), regions U{1..512}",
            "items": items, "batched_graph_ms": one_ms, "batched_items_per_s": items / (one_ms * 1e-3),
            "per_stream_launch_ms": per_ms, "per_stream_items_per_s": items / (per_ms * 1e-3),
            "per_stream_host_wall_ms": per_wall, "speedup": per_ms / one_ms,
            "per_stream_graphs_ms": per_graph_ms, "per_stream_graphs_host_wall_ms": per_graph_wall,
            "speedup_vs_per_stream_graphs": per_graph_ms / one_ms, "invariants_ok": bool(exact),
            "chosen": {"strategy": "signal" if best["strategy"] == 0 else "tag",
                       "regions_per_unit": best["regions_per_unit"], "ensemble_width": best["ensemble_width"]}}


def cgroup_cpu_stat() -> dict:
    """This process's cgroup CPU counters (cgroup v2 cpu.stat), {} where unavailable."""
    try:
        with open("/sys/fs/cgroup/cpu.stat") as f:
            return {k: int(v) for k, v in (line.split() for line in f if line.strip())}
    except Exception:
        return {}


def cgroup_cpu_quota():
    """The cgroup's CPU quota as 'max period' (cgroup v2 cpu.max), or None."""
    try:
        with open("/sys/fs/cgroup/cpu.max") as f:
            return f.read().strip()
    except Exception:
        return None


def bench_serving(rs, torch, seconds: float, rate: float = 20000.0, arena_gb: float = 40.0, slice_units: int = 64,
                  warm_requests: int = 64):
    """Open-loop Poisson arrivals of batched-size hashed streams into the
    continuous-batching server (requests advanced `slice_units` work units per launch over
    their resident state, admission by free arena memory); latency = scheduled arrival ->
    completion seen."""
    pool = wl.batched_streams()
    pipe = wl.pipeline_hash_filter_map()
    reqs = [rs.host_request(s) for s in pool]
    sizes = [wl.n_elements(s) for s in pool]
    busy = [False] * len(pool)
    arrivals = wl.poisson_arrivals(rate, seconds, seed=4)
    srv = rs.Server(pipe, arena_bytes=int(arena_gb * (1 << 30)), strategy="tag", slice_units=slice_units)
    # untimed warm-up: a few launches through the server (first launches, staging buffers)
    warm = [srv.submit(reqs[i]) for i in range(warm_requests)]
    left = set(warm)
    t_w = time.perf_counter()
    while left and time.perf_counter() - t_w < 30.0:
        srv.progress()
        left.difference_update(srv.poll())
    stamps, owner, lat, done_items = {}, {}, [], 0
    thr0 = cgroup_cpu_stat()
    # no garbage-collector pauses inside the timed loop (its objects are all still live)
    gc_was_enabled = gc.isenabled()
    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    a = 0
    pending = []
    while True:
        now = time.perf_counter() - t0
        while a < len(arrivals) and arrivals[a] <= now:
            pending.append(a)
            a += 1
        keep = []
        for j in pending:
            slot = j % len(pool)
            if busy[slot]:
                keep.append(j)
                continue
            busy[slot] = True
            rid = srv.submit(reqs[slot])
            stamps[rid] = arrivals[j]
            owner[rid] = slot
        pending = keep
        srv.progress()
        for rid in srv.poll():
            tdone = time.perf_counter() - t0
            lat.append((stamps[rid], tdone - stamps[rid], sizes[owner[rid]]))
            slot = owner.pop(rid)
            busy[slot] = False
            done_items += sizes[slot]
        if a >= len(arrivals) and not pending and not owner:
            break
        if now > seconds + 30:
            break
        if not owner and not pending and a < len(arrivals):
            # nothing in flight: sleep until shortly before the next arrival
            gap = arrivals[a] - (time.perf_counter() - t0)
            if gap > 2e-4:
                time.sleep(gap - 1e-4)
    wall = time.perf_counter() - t0
    thr1 = cgroup_cpu_stat()
    if gc_was_enabled:
        gc.enable()
    st = srv.stats()
    srv.close()
    L = np.array([x[1] for x in lat]) * 1e3
    Lw = np.array([x[1] for x in lat if x[0] >= 1.0]) * 1e3
    med = float(np.median(sizes))
    Ls = np.array([x[1] for x in lat if x[2] <= med]) * 1e3     # requests up to the median size
    return {"workload": f"Poisson {rate:.0f} streams/s for {seconds:.0f} s, batched-size hashed streams, "
                        f"arena {arena_gb:.0f} GiB, {slice_units} units per request per launch",
            "offered_items_per_s": rate * float(np.mean(sizes)),
            "launches": st["batches"], "largest_launch": st["largest_batch"],
            "requests": int(len(lat)), "items_per_s": done_items / wall,
            "p50_ms": float(np.percentile(L, 50)) if len(L) else None,
            "p99_ms": float(np.percentile(L, 99)) if len(L) else None,
            "p50_ms_after_1s": float(np.percentile(Lw, 50)) if len(Lw) else None,
            "p99_ms_after_1s": float(np.percentile(Lw, 99)) if len(Lw) else None,
            "p99_ms_requests_up_to_median_size": float(np.percentile(Ls, 99)) if len(Ls) else None,
            "max_ms": float(L.max()) if len(L) else None,
            "over_5ms": int((L > 5.0).sum()) if len(L) else 0,
            # completions of the requests over 5 ms, grouped by the 10-ms window they landed
            # in: few windows mean host stalls that delayed many requests at once
            "over_5ms_windows": int(len({int((x[0] + x[1]) * 100) for x in lat if x[1] > 5e-3})),
            "host_cpu": {"quota": cgroup_cpu_quota(),
                         "throttled_periods": (thr1.get("nr_throttled", 0) - thr0.get("nr_throttled", 0)) if thr0 else None,
                         "throttled_ms": ((thr1.get("throttled_usec", 0) - thr0.get("throttled_usec", 0)) / 1e3) if thr0 else None},
            "batches": st["batches"], "largest_batch": st["largest_batch"],
            "arena_peak_bytes": st["arena_peak"], "wall_s": wall}


def bench_serving_sweep(rs, torch, rates=(20000, 40000, 80000, 160000, 320000), seconds=3.0):
    """Arrival rates doubling from the configured 20,000 streams/s: throughput and p99 per
    rate; the saturation rate is the first whose p99 exceeds twice the lightest load's, or
    whose completions fall below 95% of the offered items."""
    rows = []
    for r in rates:
        x = bench_serving(rs, torch, seconds, rate=float(r), warm_requests=16)
        rows.append({"rate": r, "items_per_s": x["items_per_s"], "offered_items_per_s": x["offered_items_per_s"],
                     "p50_ms": x["p50_ms"], "p99_ms": x["p99_ms"],
                     "p99_ms_small": x["p99_ms_requests_up_to_median_size"], "launches": x["launches"]})
    base = rows[0]["p99_ms"] or 0.0
    sat = None
    for row in rows:
        if (row["p99_ms"] or 0.0) > 2 * base or row["items_per_s"] < 0.95 * row["offered_items_per_s"]:
            sat = row["rate"]
            break
    return {"seconds_per_rate": seconds, "rows": rows, "saturation_rate": sat}


def run_case(args, rs, torch):
    """One stream, one fixed strategy: warm-up launches then `steps` timed launches.
    Used to give profilers a small, fixed launch sequence."""
    parts = args.case.split(":")
    if parts[0] == "calib":
        # the calibration kernel on 2^lg elements of the cascade stream: calib:lg
        n = 1 << int(parts[1])
        el = rs.to_device(wl.cascade_stream(n_total=n, mean=4096, seed=SEED))["elements"]
        pipe = wl.pipeline_cascade()
        salts, thetas = [st[1] for st in pipe[1:4]], [st[2] for st in pipe[1:4]]
        out = torch.empty(2, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        for _ in range(args.warmup):
            rs.calibrate_cascade(el, 0x1234ABCD, salts, thetas, out=out)
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs.calibrate_cascade(el, 0x1234ABCD, salts, thetas, out=out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        kms = statistics.median(ms)
        print(json.dumps({"case": args.case, "n": n, "kernel_ms": kms, "items_per_s": n / (kms * 1e-3),
                          "gbs": 4 * n / (kms * 1e-3) / 1e9, "result": out.cpu().tolist()}), flush=True)
        return
    if parts[0] == "rsum":
        # the region-sum pipeline over 2^26 elements in regions of one size (rsum:SIZE:STRATEGY)
        # or of sizes uniform on 0..SIZE (rsum:USIZE:STRATEGY), as the region_sizes section cuts them
        variable = parts[1].startswith("U")
        size, strat = int(parts[1].lstrip("U")), parts[2]
        n = N_ELEM
        L = wl.sized_lengths(n, size, 11, variable)
        el = wl.sized_region_stream(n, 128, seed=11)["elements"]
        dev = {"R": int(L.shape[0]), "len": torch.from_numpy(L.view(np.int32)).cuda(),
               "elements": torch.from_numpy(el.view(np.int32)).cuda()}
        p = rs.Pipeline(wl.pipeline_region_sum(), strategy=strat)
        out = p.submit(dev, outputs=("count", "sum"))
        p.timing_enable(args.steps + args.warmup)
        for _ in range(args.warmup):
            p.run()
        torch.cuda.synchronize()
        p.timing_read()
        for _ in range(args.steps):
            p.run()
        kms = statistics.median(p.timing_read())
        got = rs.results_to_numpy(out)
        ok = bool(np.array_equal(got["count"], L) and
                  int(got["sum"].astype(np.uint64).sum()) == int(el.astype(np.uint64).sum()))
        print(json.dumps({"case": args.case, "n": n, "regions": int(L.shape[0]), "kernel_ms": kms,
                          "items_per_s": n / (kms * 1e-3), "opts": p.opts, "invariants_ok": ok}), flush=True)
        del out
        if not ok:
            raise SystemExit("rsum: counts or sums differ from the region lengths and the array's sum")
        return
    mean, strat = float(parts[0]), parts[1]
    n = 1 << int(parts[2]) if len(parts) > 2 and parts[2] else N_ELEM
    opts = {}
    if len(parts) > 3:
        for kv in parts[3].split(","):
            k, v = kv.split("=")
            opts[k] = int(v)
    s = wl.cascade_stream(n_total=n, mean=mean, seed=SEED)
    p = rs.Pipeline(wl.pipeline_cascade(), strategy=strat, **opts)
    out = p.submit(rs.to_device(s), outputs=("count", "sum"))
    p.timing_enable(args.steps + args.warmup)
    for _ in range(args.warmup):
        p.run()
    torch.cuda.synchronize()
    p.timing_read()
    for _ in range(args.steps):
        p.run()
    ms = p.timing_read()
    st = p.stats()
    kms = statistics.median(ms)
    ab = 4 * n + 20 * int(s["R"])
    print(json.dumps({"case": args.case, "n": n, "regions": int(s["R"]), "kernel_ms": kms,
                      "items_per_s": n / (kms * 1e-3), "alg_gbs": ab / (kms * 1e-3) / 1e9,
                      "opts": p.opts, "active_lane_fraction": st["active_lane_fraction"],
                      "ensembles": st["ensembles"], "firings": st["firings"], "cycles": st["cycles"]}),
          flush=True)
    del out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="also sweep arrival rates to find where p99 turns up (about 20 s more)")
    ap.add_argument("--no-extras", action="store_true", help="skip the graph, batched and serving sections")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split each stream's regions across the ranks (strong scaling) instead of "
                         "running the same five streams on every rank (weak scaling)")
    ap.add_argument("--case", default=None,
                    help="MEAN:STRATEGY[:N_LOG2[:OPT=V,...]] -- one cascade stream, fixed strategy and options; "
                         "calib:N_LOG2 -- the calibration kernel; rsum:SIZE:STRATEGY or rsum:USIZE:STRATEGY -- the "
                         "region-sum pipeline over 2^26 elements in regions of SIZE or of sizes U{0..SIZE} "
                         "(small fixed launch sequences for profilers)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2006_07478_b300 import multi, rs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.case:
        run_case(args, rs, torch)
        return

    streams = make_streams()
    if args.shard:
        # this rank's region range of every stream, balanced on merge-path cost; no data
        # crosses ranks (regions are independent), the step's items are summed over ranks
        streams = [multi.shard_stream(s, world, rank) for s in streams]
    pipe = wl.pipeline_cascade()

    # ---- device-resident inputs, one pipeline per stream, tuned per stream ----
    pipes, outs, tuned = [], [], []
    for s in streams:
        p = rs.Pipeline(pipe, strategy="auto")   # the autotuner picks the strategy too
        dev = rs.to_device(s)
        out = p.submit(dev, outputs=("count", "sum"))
        pipes.append(p)
        outs.append(out)
    per_mean = []
    for m, s, p in zip(MEANS, streams, pipes):
        best, best_ms = p.autotune(trials=3)
        tuned.append(best)
        row = {"mean": m, "regions": int(s["R"]), "alg_bytes": alg_bytes(s),
               "chosen": {"strategy": "signal" if best["strategy"] == 0 else "tag",
                          **{k: best[k] for k in ("ensemble_width", "regions_per_unit", "region_cost",
                                                  "tile_elements", "warps_per_block")}}}
        # both strategies, kernel-only event timing, each with the options the autotuner
        # finds for it (the other one searched alone, its strategy fixed)
        chosen = "signal" if best["strategy"] == 0 else "tag"
        for strat in ("tag", "signal"):
            if strat == chosen:
                p.set_opts(**{k: v for k, v in best.items() if k != "strategy"}, strategy=best["strategy"])
            else:
                p.set_opts(strategy=strat, regions_per_unit=0, region_cost=0, ensemble_width=128,
                           tile_elements=0, tiles_in_flight=0, warps_per_block=0, queue_capacity=0)
                other, _ = p.autotune(trials=2)
                row[strat + "_options"] = {k: other[k] for k in ("ensemble_width", "regions_per_unit",
                                                                "region_cost", "tile_elements", "warps_per_block")}
            p.timing_enable(8)
            for _ in range(2):
                p.run()
            torch.cuda.synchronize()
            p.timing_read()
            for _ in range(5):
                p.run()
            ms = p.timing_read()
            st = p.stats()
            kms = statistics.median(ms)
            gbs = alg_bytes(s) / (kms * 1e-3) / 1e9
            row[strat] = {"kernel_ms": kms, "items_per_s": wl.n_elements(s) / (kms * 1e-3), "alg_gbs": gbs,
                          "options": "tuned" if strat == chosen else "tuned for this strategy alone",
                          "active_lane_fraction": [round(x, 4) for x in st["active_lane_fraction"]],
                          "launch": st["launch"]}
        p.set_opts(**{k: v for k, v in best.items() if k != "strategy"}, strategy=best["strategy"])
        per_mean.append(row)

    # invariants of the tuned configuration's results (exactness against the oracle at this
    # size is tested in tests/): counts within the region lengths, adding up to the items
    # the aggregate consumed
    for s, p, out in zip(streams, pipes, outs):
        p.run()
        torch.cuda.synchronize()
        st = p.stats()
        c = rs.results_to_numpy(out)["count"].astype(np.int64)
        assert np.all(c <= s["len"].astype(np.int64)) and int(c.sum()) == st["items"][-1]

    for p in pipes:
        p.timing_enable(args.steps + 8)

    # ---- warm-up, then exactly K timed steps ----
    for _ in range(args.warmup):
        for p in pipes:
            p.run()
    torch.cuda.synchronize()
    for p in pipes:
        p.timing_read()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        for p in pipes:
            p.run()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    barrier()
    time.sleep(0.2)
    sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    kernel_ms = [p.timing_read() for p in pipes]
    statuses = [p.stats()["device_status"] for p in pipes]
    assert all(s == 0 for s in statuses), statuses
    # every rank runs the same five streams (weak scaling): the step time is the slowest
    # rank's, the items are summed over ranks
    items_step = sum(wl.n_elements(s) for s in streams)
    elapsed_ms, items_all = multi.reduce_step(elapsed_ms, items_step * args.steps, device="cuda")
    value = items_all / (elapsed_ms * 1e-3)

    # ---- roofline of the timed kernel: algorithmic bytes / kernel time, all launches ----
    peak, peak_kind = load_peaks()
    tot_bytes = sum(alg_bytes(s) * len(k) for s, k in zip(streams, kernel_ms))
    tot_kms = sum(sum(k) for k in kernel_ms)
    achieved = tot_bytes / (tot_kms * 1e-3) / 1e9
    traffic_rows = read_traffic()
    traffic = None
    if traffic_rows:
        try:
            traffic = sum(traffic_rows[(m, "signal" if t["strategy"] == 0 else "tag")]
                          for m, t in zip(MEANS, tuned)) / len(MEANS)
        except KeyError:
            traffic = None
    for row, k in zip(per_mean, kernel_ms):
        kms = statistics.median(k)
        row["timed_kernel_ms_median"] = kms
        row["timed_alg_gbs"] = row["alg_bytes"] / (kms * 1e-3) / 1e9
        row["frac_of_measured_hbm"] = row["timed_alg_gbs"] / peak
        row["frac_of_8tbs_spec"] = row["timed_alg_gbs"] / SPEC_HBM_GBS

    # ---- end to end: host buffers, copies inside the timed region ----
    e2e = None
    if args.e2e_steps > 0:
        host_in, dev_in = [], []
        for p in pipes:
            dev = p._keep[0][0]
            hi = {k: dev[k].cpu().pin_memory() for k in ("len", "elements", "ctx") if dev.get(k) is not None}
            host_in.append(hi)
            dev_in.append(dev)
        host_out = [{"count": torch.empty_like(o["count"], device="cpu").pin_memory(),
                     "sum": torch.empty_like(o["sum"], device="cpu").pin_memory()} for o in outs]
        h2d = sum(t.numel() * t.element_size() for hi in host_in for t in hi.values())
        d2h = sum(t.numel() * t.element_size() for ho in host_out for t in ho.values())
        # three CUDA streams so that a stream's copy-in, the previous stream's pipeline run
        # and an earlier stream's copy-out overlap; events order each stream's own copy-in
        # -> run -> copy-out and keep the next step's copies off buffers still in use
        s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        n = len(pipes)
        ev_in = [torch.cuda.Event() for _ in range(n)]
        ev_run = [torch.cuda.Event() for _ in range(n)]
        ev_out = [torch.cuda.Event() for _ in range(n)]
        started = [False] * n
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(args.e2e_steps + 1):
            if rep == 1:
                torch.cuda.synchronize()
                barrier()
                e0.record(s_in)
            for i, (p, hi, dev, out, ho) in enumerate(zip(pipes, host_in, dev_in, outs, host_out)):
                if started[i]:
                    s_in.wait_event(ev_run[i])     # the previous run of this stream has read its inputs
                with torch.cuda.stream(s_in):
                    p.upload(out["id"], hi)      # rs_stream_upload: host buffers -> the stream's arrays
                ev_in[i].record(s_in)
                s_run.wait_event(ev_in[i])
                if started[i]:
                    s_run.wait_event(ev_out[i])    # its previous results have been copied out
                with torch.cuda.stream(s_run):
                    p.run()
                ev_run[i].record(s_run)
                s_out.wait_event(ev_run[i])
                with torch.cuda.stream(s_out):
                    p.fetch(out["id"], count=ho["count"], sum=ho["sum"])
                ev_out[i].record(s_out)
                started[i] = True
        s_out.wait_event(ev_in[n - 1])
        e1.record(s_out)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
        e2e_ms, e2e_items = multi.reduce_step(e2e_ms, items_step, device="cuda")
        e2e = {"value": e2e_items / (e2e_ms * 1e-3), "unit": "items/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
               "overlap": "copy-in, run and copy-out on three CUDA streams",
               "path": "C ABI: rs_stream_upload -> rs_run -> rs_fetch_region_results, page-locked host buffers"}

    extras = {}
    if rank == 0 and not args.no_extras:
        for name, fn in (("calibration", lambda: bench_calibration(rs, torch, pipes[MEANS.index(4096)]._keep[0][0], peak,
                                                                   per_mean[MEANS.index(4096)]["timed_kernel_ms_median"])),
                         ("modes", lambda: bench_modes(rs, torch, [(m, s) for m, s in zip(MEANS, streams)
                                                                  if m in (4, 32, 256)])),
                         ("graph_edges", lambda: bench_graph(rs, torch, peak)),
                         ("region_sizes", lambda: bench_region_sizes(rs, torch)),
                         ("batched", lambda: bench_batched(rs, torch)),
                         ("serving", lambda: bench_serving(rs, torch, args.serve_seconds)),
                         ("serving_whole_requests",
                          lambda: bench_serving(rs, torch, min(10.0, args.serve_seconds), slice_units=0)),
                         ("serving_sweep", lambda: bench_serving_sweep(rs, torch) if args.serve_sweep else None)):
            try:
                extras[name] = fn()
            except Exception as exc:   # report, do not lose the main line
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- CPU baseline: the oracle on the host's cores (rank 0, N = 1), after the
    # GPU sections so that its host-memory churn does not overlap the serving loop ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        items, secs, done = time_oracle(streams, threads, budget_s=20.0)
        cpu = {"value": items / secs, "unit": "items/s", "cores": threads, "kind": "oracle",
               "sample": f"{done} of the 5 streams, whole ({items} elements), {threads} threads"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "items/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.shard else "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded)",
            "config": {"workload": "cascade: 5 streams x 2^26 u32 elements, geometric regions mean 1/4/32/256/4096, "
                                   "3 context hash filters (pass 0.5/0.3/0.1), count+sum per region",
                       "seed": SEED, "l2": "inputs larger than L2 (256 MiB per stream), streams alternate",
                       "parallelism": f"region shards x{world}" if args.shard else f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "frac_of_8tbs_spec": achieved / SPEC_HBM_GBS,
                         "kernel": "planner + pipeline kernel (rs_tag_kernel for the tag strategy) of "
                                   "every run in the timed region",
                         "kernel_source": kernel_source_hash()},
            "per_mean": per_mean,
            "clocks": sampler.summary(t_start, t_end),
            "e2e": e2e,
            "cpu_baseline": cpu,
            # per run: the tag strategy's unit sums + group scan (loaded streams of mean under 8)
            # or planner, and the pipeline kernel; the signal strategy's planner, pipeline
            # kernel and finalize kernel
            "gpu_launches": sum(len(k) * (3 if t["strategy"] != 1 or wl.n_elements(s) < 8 * s["R"] else 2)
                                for k, t, s in zip(kernel_ms, tuned, streams)),
            **extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
