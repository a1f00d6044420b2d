"""ctypes binding of librs (include/rs.h): argument marshalling only.

Every step of the pipeline runs in the CUDA library; this module turns stage
tuples into rs_stage_desc records, torch CUDA tensors into device pointers and
the current torch CUDA stream into an rs_cuda_stream.  torch is used for device
memory and streams only.  There is no CPU path: if librs.so is missing or no GPU
is present, calls raise.

Stage tuples (the same names the workload module uses):
    ("enum_hash",)                   element i of parent r = hash32(p_r, i)
    ("enum_load",)                   element i of parent r = elements[off_r + i]
    ("filter_mod", m, c)             keep x mod m == c
    ("filter_hash_ctx", salt, theta) keep (hash32(x, salt) ^ t_r) < theta
    ("filter_weight_lt", salt)       keep hash32(x, salt) < hash32(p_r, salt)
    ("map_mul", a, b)                x <- a*x + b mod 2^32
    ("expand", k, salt)              0..k outputs per input
    ("aggregate",)                   count / sum / min per region
    ("emit",)                        the survivors themselves, grouped by region (needs
                                     CSR offsets; outputs "count" and "values")
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RS_OK, RS_ERR_INVALID, RS_ERR_NOMEM, RS_ERR_CUDA, RS_ERR_NOT_READY = 0, 1, 2, 3, 4
RS_ERR_STALL, RS_ERR_CAPACITY, RS_ERR_STATE, RS_ERR_DEVICE_INPUT = 5, 6, 7, 8
RS_ENUM_HASH, RS_ENUM_LOAD, RS_FILTER, RS_MAP, RS_EXPAND, RS_AGGREGATE, RS_EMIT = 1, 2, 3, 4, 5, 6, 7
RS_OP_NONE, RS_OP_MOD_EQ, RS_OP_HASH_CTX_LT, RS_OP_WEIGHT_LT, RS_OP_MUL_ADD, RS_OP_HASH_FANOUT = 0, 1, 2, 3, 4, 5
STRATEGIES = {"signal": 0, "tag": 1, "auto": 2}
BOUNDARIES = {"default": 0, "signal": 1, "tag": 2, "lane": 3}


def boundary_modes(modes) -> int:
    """Pack per-stage boundary modes ({stage: "signal" | "tag" | "lane"}, or a list
    indexed by stage with None / "default" for the pipeline's strategy) into
    rs_pipeline_opts.boundary_modes."""
    if isinstance(modes, int):
        return modes
    items = modes.items() if isinstance(modes, dict) else enumerate(modes)
    v = 0
    for stage, m in items:
        if m is None:
            continue
        v |= BOUNDARIES[m] << (2 * int(stage))
    return v
RS_MAX_STAGES = 6

EXPORTS = [
    "rs_default_opts", "rs_pipeline_create", "rs_pipeline_destroy", "rs_pipeline_set_opts",
    "rs_pipeline_get_opts", "rs_stream_submit", "rs_clear_streams", "rs_workspace_size", "rs_run",
    "rs_stream_state_size", "rs_stream_submit_slice",
    "rs_fetch_region_results", "rs_stream_upload", "rs_get_stats", "rs_graph_capture", "rs_graph_launch",
    "rs_graph_release", "rs_autotune", "rs_timing_enable", "rs_timing_read", "rs_run_noalloc",
    "rs_server_create", "rs_server_set_slice_units", "rs_server_submit", "rs_server_progress", "rs_server_poll", "rs_server_get_stats",
    "rs_server_destroy", "rs_calibrate_cascade", "rs_status_string", "rs_last_cuda_error", "rs_version",
    "rs_struct_sizes",
]
# the ctypes mirrors, in the order rs_struct_sizes reports the C structs' sizes
_MIRRORS = ("StageDesc", "Opts", "StreamDesc", "RegionResults", "Stats", "Request", "ServerStats")


class StageDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("op", ctypes.c_uint32), ("max_fanout", ctypes.c_uint32),
                ("params", ctypes.c_uint32 * 4), ("input", ctypes.c_uint32)]


class Opts(ctypes.Structure):
    _fields_ = [("ensemble_width", ctypes.c_uint32), ("queue_capacity", ctypes.c_uint32),
                ("signal_capacity", ctypes.c_uint32), ("strategy", ctypes.c_uint32),
                ("regions_per_unit", ctypes.c_uint32), ("tile_elements", ctypes.c_uint32),
                ("tiles_in_flight", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("region_cost", ctypes.c_uint32),
                ("device_budget", ctypes.c_uint64), ("boundary_modes", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class StreamDesc(ctypes.Structure):
    _fields_ = [("n_regions", ctypes.c_uint64), ("parents", ctypes.c_void_p), ("region_len", ctypes.c_void_p),
                ("region_offsets", ctypes.c_void_p), ("elements", ctypes.c_void_p),
                ("n_elements", ctypes.c_uint64), ("ctx", ctypes.c_void_p), ("out_count", ctypes.c_void_p),
                ("out_sum", ctypes.c_void_p), ("out_min", ctypes.c_void_p),
                ("total_elements_hint", ctypes.c_uint64), ("out_values", ctypes.c_void_p),
                ("out_values_len", ctypes.c_uint64), ("out2_count", ctypes.c_void_p),
                ("out2_sum", ctypes.c_void_p), ("out2_min", ctypes.c_void_p)]


class HostInputs(ctypes.Structure):
    _fields_ = [("parents", ctypes.c_void_p), ("region_len", ctypes.c_void_p), ("region_offsets", ctypes.c_void_p),
                ("elements", ctypes.c_void_p), ("ctx", ctypes.c_void_p)]


class RegionResults(ctypes.Structure):
    _fields_ = [("count", ctypes.c_void_p), ("sum", ctypes.c_void_p), ("min", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("device_status", ctypes.c_uint32), ("n_nodes", ctypes.c_uint32), ("units", ctypes.c_uint64),
                ("ensembles", ctypes.c_uint64 * RS_MAX_STAGES), ("items", ctypes.c_uint64 * RS_MAX_STAGES),
                ("signals", ctypes.c_uint64 * RS_MAX_STAGES), ("firings", ctypes.c_uint64 * RS_MAX_STAGES),
                ("cycles", ctypes.c_uint64 * 16), ("grid", ctypes.c_uint32), ("block", ctypes.c_uint32),
                ("smem_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("chunk_parents", ctypes.c_uint32)]
    CYCLE_SLOTS = ("setup", "lookback", "tile_wait", "enumerate", "node1", "node2", "node3", "node4",
                   "node5", "flush", "total")

    def as_dict(self, W: int = 32):
        """Counters as lists per node; active-lane fraction = items / (W * ensembles)."""
        n = self.n_nodes
        ens = list(self.ensembles)[:n]
        items = list(self.items)[:n]
        return {
            "device_status": self.device_status, "units": self.units,
            "ensembles": ens, "items": items,
            "signals": list(self.signals)[:n], "firings": list(self.firings)[:n],
            "ensemble_width": W,
            "cycles": {k: int(self.cycles[i]) for i, k in enumerate(self.CYCLE_SLOTS[:4])} |
                      {self.CYCLE_SLOTS[4 + j]: int(self.cycles[4 + 1 + j]) for j in range(5)} |
                      {"flush": int(self.cycles[10]), "total": int(self.cycles[11]),
                       "n1_gather": int(self.cycles[12]), "compute": int(self.cycles[13]),
                       "compact": int(self.cycles[14]), "tiles": int(self.cycles[15])},
            "active_lane_fraction": [(it / (float(W) * e)) if e else 0.0 for it, e in zip(items, ens)],
            "launch": {"grid": self.grid, "block": self.block, "smem_per_block": self.smem_per_block,
                       "blocks_per_sm": self.blocks_per_sm, "chunk_parents": self.chunk_parents},
        }


class Request(ctypes.Structure):
    _fields_ = [("n_regions", ctypes.c_uint64), ("parents", ctypes.c_void_p), ("region_len", ctypes.c_void_p),
                ("elements", ctypes.c_void_p), ("n_elements", ctypes.c_uint64), ("ctx", ctypes.c_void_p),
                ("out_count", ctypes.c_void_p), ("out_sum", ctypes.c_void_p), ("out_min", ctypes.c_void_p),
                ("total_elements_hint", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "batches", "largest_batch",
                                               "in_flight", "queued", "arena_live", "arena_peak", "gathered",
                                               "per_array")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class RsError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lib = None


def lib(build_if_missing: bool = True):
    """Load librs.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        path = _build.PROF_LIB if os.environ.get("RS_PROFILE_BUILD") == "1" else _build.LIB
        if build_if_missing and path == _build.PROF_LIB:
            _build.build(profile=True)
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not found at {path}; the CUDA library is required")
        L = ctypes.CDLL(path)
        P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        sig = {
            "rs_default_opts": ([ctypes.POINTER(Opts)], ctypes.c_int),
            "rs_pipeline_create": ([ctypes.POINTER(StageDesc), U32, ctypes.POINTER(Opts), ctypes.POINTER(P)],
                                   ctypes.c_int),
            "rs_pipeline_destroy": ([P], ctypes.c_int),
            "rs_pipeline_set_opts": ([P, ctypes.POINTER(Opts)], ctypes.c_int),
            "rs_pipeline_get_opts": ([P, ctypes.POINTER(Opts)], ctypes.c_int),
            "rs_stream_submit": ([P, ctypes.POINTER(StreamDesc), ctypes.POINTER(U64)], ctypes.c_int),
            "rs_stream_state_size": ([P, ctypes.POINTER(StreamDesc), ctypes.POINTER(U64), ctypes.POINTER(U64)],
                                     ctypes.c_int),
            "rs_stream_submit_slice": ([P, ctypes.POINTER(StreamDesc), P, U64, U64, U64, ctypes.POINTER(U64)],
                                       ctypes.c_int),
            "rs_clear_streams": ([P], ctypes.c_int),
            "rs_workspace_size": ([P, ctypes.POINTER(U64)], ctypes.c_int),
            "rs_run": ([P, P, U64, P], ctypes.c_int),
            "rs_fetch_region_results": ([P, U64, ctypes.POINTER(RegionResults), P], ctypes.c_int),
            "rs_stream_upload": ([P, U64, ctypes.POINTER(HostInputs), P], ctypes.c_int),
            "rs_get_stats": ([P, P, P, ctypes.POINTER(Stats)], ctypes.c_int),
            "rs_graph_capture": ([P, P, U64, P], ctypes.c_int),
            "rs_graph_launch": ([P, P], ctypes.c_int),
            "rs_graph_release": ([P], ctypes.c_int),
            "rs_autotune": ([P, P, U64, P, U32, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_float)],
                            ctypes.c_int),
            "rs_timing_enable": ([P, U32], ctypes.c_int),
            "rs_timing_read": ([P, ctypes.POINTER(ctypes.c_float), U32, ctypes.POINTER(U32)], ctypes.c_int),
            "rs_run_noalloc": ([P, P], ctypes.c_int),
            "rs_server_create": ([ctypes.POINTER(StageDesc), U32, ctypes.POINTER(Opts), P, U64, U32, U32, P,
                                  ctypes.POINTER(P)], ctypes.c_int),
            "rs_server_set_slice_units": ([P, U32], ctypes.c_int),
            "rs_server_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(U64)], ctypes.c_int),
            "rs_server_progress": ([P], ctypes.c_int),
            "rs_server_poll": ([P, ctypes.POINTER(U64), U32, ctypes.POINTER(U32)], ctypes.c_int),
            "rs_server_get_stats": ([P, ctypes.POINTER(ServerStats)], ctypes.c_int),
            "rs_server_destroy": ([P], ctypes.c_int),
            "rs_calibrate_cascade": ([P, U64, U32, ctypes.POINTER(U32), ctypes.POINTER(U32), P, P], ctypes.c_int),
            "rs_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "rs_last_cuda_error": ([], ctypes.c_int),
            "rs_version": ([], U32),
            "rs_struct_sizes": ([ctypes.POINTER(U64), U32], U32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        c_sizes = (U64 * len(_MIRRORS))()
        n = L.rs_struct_sizes(c_sizes, len(_MIRRORS))
        mine = [ctypes.sizeof(globals()[m]) for m in _MIRRORS]
        if n != len(_MIRRORS) or list(c_sizes) != mine:
            raise RuntimeError(f"librs struct layout differs from the binding: C {list(c_sizes)[:n]} vs ctypes {mine}")
        _lib = L
    return _lib


def status_string(st: int) -> str:
    return lib().rs_status_string(int(st)).decode()


def check(st: int, what: str):
    if st != RS_OK:
        if st == RS_ERR_CUDA:
            raise RsError(st, f"{what} (cuda error {lib().rs_last_cuda_error()})")
        raise RsError(st, what)


def stage_desc(st) -> StageDesc:
    name, a = st[0], [int(x) & 0xFFFFFFFF for x in st[1:]]
    d = StageDesc()
    d.max_fanout = 1
    if name == "enum_hash":
        d.kind = RS_ENUM_HASH
    elif name == "enum_load":
        d.kind = RS_ENUM_LOAD
    elif name == "aggregate":
        d.kind = RS_AGGREGATE
    elif name == "emit":
        d.kind = RS_EMIT
    elif name == "filter_mod":
        d.kind, d.op = RS_FILTER, RS_OP_MOD_EQ
        d.params[0], d.params[1] = a[0], a[1]
    elif name == "filter_hash_ctx":
        d.kind, d.op = RS_FILTER, RS_OP_HASH_CTX_LT
        d.params[0], d.params[1] = a[0], a[1]
    elif name == "filter_weight_lt":
        d.kind, d.op = RS_FILTER, RS_OP_WEIGHT_LT
        d.params[0] = a[0]
    elif name == "map_mul":
        d.kind, d.op = RS_MAP, RS_OP_MUL_ADD
        d.params[0], d.params[1] = a[0], a[1]
    elif name == "expand":
        d.kind, d.op = RS_EXPAND, RS_OP_HASH_FANOUT
        d.max_fanout = a[0]
        d.params[0] = a[1]
    else:
        raise ValueError(f"unknown stage {name!r}")
    return d


FLAG_UNBALANCED_UNITS = 1      # RS_FLAG_UNBALANCED_UNITS
FLAG_PRIVATE_WORKSPACE = 2     # RS_FLAG_PRIVATE_WORKSPACE


def make_opts(strategy="tag", **kw) -> Opts:
    o = Opts()
    check(lib().rs_default_opts(ctypes.byref(o)), "rs_default_opts")
    o.queue_capacity = 0
    o.strategy = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _cur_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Pipeline:
    """A stage list bound to options; streams are submitted as torch CUDA tensors.

    inputs: a tree topology (Figure 1(b)) -- inputs[s] is the stage whose output stage s
    reads (inputs[0] is ignored); None is a linear pipeline.  boundary_modes: per-stage
    boundary modes (see `boundary_modes`)."""

    def __init__(self, stages, strategy="tag", inputs=None, **opts):
        self.stages = list(stages)
        self.inputs = list(inputs) if inputs is not None else None
        descs = [stage_desc(s) for s in self.stages]
        if self.inputs is not None:
            for i in range(1, len(descs)):
                descs[i].input = int(self.inputs[i])
        arr = (StageDesc * len(self.stages))(*descs)
        if "boundary_modes" in opts:
            opts["boundary_modes"] = boundary_modes(opts["boundary_modes"])
        # the workspace is this object's own tensor: runs may keep the stream table in it
        opts["flags"] = int(opts.get("flags", 0)) | FLAG_PRIVATE_WORKSPACE
        o = make_opts(strategy, **opts)
        h = ctypes.c_void_p()
        check(lib().rs_pipeline_create(arr, len(self.stages), ctypes.byref(o), ctypes.byref(h)),
              "rs_pipeline_create")
        self._h = h
        self._keep = []          # tensors referenced by submitted streams
        self._ws = None
        self.streams = []

    def close(self):
        if getattr(self, "_h", None):
            lib().rs_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def opts(self) -> dict:
        o = Opts()
        check(lib().rs_pipeline_get_opts(self._h, ctypes.byref(o)), "rs_pipeline_get_opts")
        return o.as_dict()

    def set_opts(self, strategy=None, **kw):
        o = Opts()
        check(lib().rs_pipeline_get_opts(self._h, ctypes.byref(o)), "rs_pipeline_get_opts")
        if strategy is not None:
            o.strategy = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        if "boundary_modes" in kw:
            kw["boundary_modes"] = boundary_modes(kw["boundary_modes"])
        if "flags" in kw:
            kw["flags"] = int(kw["flags"]) | FLAG_PRIVATE_WORKSPACE
        for k, v in kw.items():
            setattr(o, k, int(v))
        check(lib().rs_pipeline_set_opts(self._h, ctypes.byref(o)), "rs_pipeline_set_opts")

    def fanout_product(self) -> int:
        """Segment slots per element of an emit sink (product of the maximum fan-outs)."""
        F = 1
        for st in self.stages[1:-1]:
            if st[0] == "expand":
                F *= max(1, int(st[1]))
        return F

    def submit(self, dev: dict, outputs=("count", "sum", "min"), out=None, state=None, unit_begin=0,
               unit_count=None) -> dict:
        """Register a device stream (dict of torch CUDA tensors: parents, len, offsets,
        elements, ctx; any may be None).  Allocates its result tensors (or reuses `out`,
        the dict an earlier submit returned) and returns them in a dict with the stream
        id.  An emit pipeline's outputs are "count" and "values" (F x the stream's element
        count entries).  With unit_count set, the stream is submitted for a sliced run of
        its units [unit_begin, unit_begin + unit_count) with `state` (a uint8 CUDA tensor
        of at least state_size(dev)[0] bytes, kept by the caller across slices)."""
        import torch
        if out is not None:
            d = self._desc(dev, out)
            return self._register(dev, out, d, state, unit_begin, unit_count)
        R = int(dev["R"])
        dvc = torch.device("cuda")
        emit = self.stages[-1][0] == "emit"
        if emit:
            outputs = ("count", "values")
        out = {
            "count": torch.empty(R, dtype=torch.int32, device=dvc) if "count" in outputs else None,
            "sum": torch.empty(R, dtype=torch.int64, device=dvc) if "sum" in outputs else None,
            "min": torch.empty(R, dtype=torch.int32, device=dvc) if "min" in outputs else None,
        }
        if emit:
            n = max(1, self.fanout_product() * int(dev.get("total_elements", 0)))
            out["values"] = torch.empty(n, dtype=torch.int32, device=dvc)
        if sum(1 for st in self.stages[1:] if st[0] == "aggregate") > 1:
            # a tree's second leaf
            for k, dt in (("count", torch.int32), ("sum", torch.int64), ("min", torch.int32)):
                out[k + "2"] = torch.empty(R, dtype=dt, device=dvc) if out[k] is not None else None
        d = StreamDesc()
        d.n_regions = R
        d.parents = _ptr(dev.get("parents"))
        d.region_len = _ptr(dev.get("len"))
        d.region_offsets = _ptr(dev.get("offsets"))
        el = dev.get("elements")
        d.elements = _ptr(el)
        d.n_elements = 0 if el is None else int(el.numel())
        d.ctx = _ptr(dev.get("ctx"))
        d.out_count = _ptr(out["count"])
        d.out_sum = _ptr(out["sum"])
        d.out_min = _ptr(out["min"])
        d.total_elements_hint = int(dev.get("total_elements", 0))
        if out.get("values") is not None:
            d.out_values = _ptr(out["values"])
            d.out_values_len = int(out["values"].numel())
        d.out2_count = _ptr(out.get("count2"))
        d.out2_sum = _ptr(out.get("sum2"))
        d.out2_min = _ptr(out.get("min2"))
        return self._register(dev, out, d, state, unit_begin, unit_count)

    def _desc(self, dev: dict, out: dict):
        d = StreamDesc()
        d.n_regions = int(dev["R"])
        d.parents = _ptr(dev.get("parents"))
        d.region_len = _ptr(dev.get("len"))
        d.region_offsets = _ptr(dev.get("offsets"))
        el = dev.get("elements")
        d.elements = _ptr(el)
        d.n_elements = 0 if el is None else int(el.numel())
        d.ctx = _ptr(dev.get("ctx"))
        d.out_count = _ptr(out.get("count"))
        d.out_sum = _ptr(out.get("sum"))
        d.out_min = _ptr(out.get("min"))
        d.total_elements_hint = int(dev.get("total_elements", 0))
        if out.get("values") is not None:
            d.out_values = _ptr(out["values"])
            d.out_values_len = int(out["values"].numel())
        d.out2_count = _ptr(out.get("count2"))
        d.out2_sum = _ptr(out.get("sum2"))
        d.out2_min = _ptr(out.get("min2"))
        return d

    def _register(self, dev, out, d, state, unit_begin, unit_count):
        sid = ctypes.c_uint64()
        if unit_count is None:
            check(lib().rs_stream_submit(self._h, ctypes.byref(d), ctypes.byref(sid)), "rs_stream_submit")
        else:
            st_ptr = None if state is None else ctypes.c_void_p(state.data_ptr())
            st_len = 0 if state is None else int(state.numel())
            check(lib().rs_stream_submit_slice(self._h, ctypes.byref(d), st_ptr, st_len, int(unit_begin),
                                               int(unit_count), ctypes.byref(sid)), "rs_stream_submit_slice")
        self._keep.append((dev, out, state))
        out["id"] = int(sid.value)
        self.streams.append(out)
        return out

    def state_size(self, dev: dict) -> tuple:
        """(bytes of resident state, units) of a sliced run of the device stream `dev`."""
        d = self._desc(dev, {})
        b, u = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().rs_stream_state_size(self._h, ctypes.byref(d), ctypes.byref(b), ctypes.byref(u)),
              "rs_stream_state_size")
        return int(b.value), int(u.value)

    def clear(self):
        check(lib().rs_clear_streams(self._h), "rs_clear_streams")
        self._keep = []
        self.streams = []

    def workspace_bytes(self) -> int:
        n = ctypes.c_uint64()
        check(lib().rs_workspace_size(self._h, ctypes.byref(n)), "rs_workspace_size")
        return int(n.value)

    def workspace(self):
        import torch
        need = max(256, self.workspace_bytes())
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        # 256-byte aligned view
        off = (-self._ws.data_ptr()) % 256
        return self._ws[off:]

    def run(self):
        ws = self.workspace()
        check(lib().rs_run(self._h, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _cur_stream()), "rs_run")

    def run_noalloc(self):
        """rs_run without a workspace: scratch in the library's fixed device array."""
        check(lib().rs_run_noalloc(self._h, _cur_stream()), "rs_run_noalloc")

    def stats(self, raise_on_error=True) -> dict:
        ws = self.workspace()
        s = Stats()
        st = lib().rs_get_stats(self._h, ctypes.c_void_p(ws.data_ptr()), _cur_stream(), ctypes.byref(s))
        if raise_on_error:
            check(st, "rs_get_stats")
        d = s.as_dict(self.opts["ensemble_width"])
        d["status"] = st
        return d

    def fetch(self, sid: int, count=None, sum=None, min=None):
        r = RegionResults(_ptr(count), _ptr(sum), _ptr(min))
        check(lib().rs_fetch_region_results(self._h, sid, ctypes.byref(r), _cur_stream()),
              "rs_fetch_region_results")

    def upload(self, sid: int, host: dict):
        """Copy a stream's inputs from host tensors (keys parents, len, offsets, elements,
        ctx; page-locked for asynchronous copies) into its device arrays (rs_stream_upload)."""
        src = HostInputs(_ptr(host.get("parents")), _ptr(host.get("len")), _ptr(host.get("offsets")),
                         _ptr(host.get("elements")), _ptr(host.get("ctx")))
        check(lib().rs_stream_upload(self._h, sid, ctypes.byref(src), _cur_stream()), "rs_stream_upload")

    def graph_capture(self):
        ws = self.workspace()
        check(lib().rs_graph_capture(self._h, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _cur_stream()),
              "rs_graph_capture")

    def graph_launch(self):
        check(lib().rs_graph_launch(self._h, _cur_stream()), "rs_graph_launch")

    def graph_release(self):
        check(lib().rs_graph_release(self._h), "rs_graph_release")

    def timing_enable(self, capacity: int):
        check(lib().rs_timing_enable(self._h, int(capacity)), "rs_timing_enable")

    def timing_read(self, max_n: int = 65536) -> list:
        buf = (ctypes.c_float * max_n)()
        n = ctypes.c_uint32()
        check(lib().rs_timing_read(self._h, buf, max_n, ctypes.byref(n)), "rs_timing_read")
        return [float(buf[i]) for i in range(n.value)]

    def autotune(self, trials=3):
        ws = self.workspace()
        best = Opts()
        ms = ctypes.c_float()
        check(lib().rs_autotune(self._h, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _cur_stream(), trials,
                                ctypes.byref(best), ctypes.byref(ms)), "rs_autotune")
        return best.as_dict(), float(ms.value)


def calibrate_cascade(elements, ctx: int, salts, thetas, out=None):
    """rs_calibrate_cascade: the cascade's three context-hash filters over ONE region of
    `elements` (a CUDA uint32/int32 tensor), no region handling; a measurement aid.  Returns
    the device int64 tensor [count, sum] (filled asynchronously on the current stream)."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.int64, device=elements.device)
    s3 = (ctypes.c_uint32 * 3)(*[int(v) & 0xFFFFFFFF for v in salts])
    t3 = (ctypes.c_uint32 * 3)(*[int(v) & 0xFFFFFFFF for v in thetas])
    check(lib().rs_calibrate_cascade(_ptr(elements), int(elements.numel()), int(ctx) & 0xFFFFFFFF, s3, t3,
                                     _ptr(out), _cur_stream()), "rs_calibrate_cascade")
    return out


class Server:
    """Continuous-batching server (rs_server_*) over one stage list.

    The arena (device memory budget) is a torch uint8 tensor owned by this object.
    Requests are host streams: dicts of pinned int32/int64 CPU tensors (see
    `host_request`); their outputs are filled in place when poll() reports the id."""

    def __init__(self, stages, arena_bytes, strategy="tag", max_batch=0, max_inflight=0, stream=None,
                 slice_units=None, **opts):
        import torch
        self.stages = list(stages)
        arr = (StageDesc * len(self.stages))(*[stage_desc(s) for s in self.stages])
        o = make_opts(strategy, **opts)
        self.arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device="cuda")
        off = (-self.arena.data_ptr()) % 256
        self._arena_view = self.arena[off:]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        check(lib().rs_server_create(arr, len(self.stages), ctypes.byref(o),
                                     ctypes.c_void_p(self._arena_view.data_ptr()), int(arena_bytes),
                                     int(max_batch), int(max_inflight), ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(h)), "rs_server_create")
        self._h = h
        if slice_units is not None:
            check(lib().rs_server_set_slice_units(h, int(slice_units)), "rs_server_set_slice_units")
        self._live = {}
        self._ids = (ctypes.c_uint64 * 4096)()

    def submit(self, req: dict) -> int:
        r = Request()
        r.n_regions = int(req["R"])
        r.parents = _ptr(req.get("parents"))
        r.region_len = _ptr(req.get("len"))
        el = req.get("elements")
        r.elements = _ptr(el)
        r.n_elements = 0 if el is None else int(el.numel())
        r.ctx = _ptr(req.get("ctx"))
        r.out_count = _ptr(req.get("count"))
        r.out_sum = _ptr(req.get("sum"))
        r.out_min = _ptr(req.get("min"))
        r.total_elements_hint = int(req.get("total_elements", 0))
        rid = ctypes.c_uint64()
        check(lib().rs_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)), "rs_server_submit")
        self._live[int(rid.value)] = req      # keep the host buffers alive until done
        return int(rid.value)

    def progress(self):
        check(lib().rs_server_progress(self._h), "rs_server_progress")

    def poll(self) -> list:
        n = ctypes.c_uint32()
        check(lib().rs_server_poll(self._h, self._ids, 4096, ctypes.byref(n)), "rs_server_poll")
        done = [int(self._ids[i]) for i in range(n.value)]
        for i in done:
            self._live.pop(i, None)
        return done

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().rs_server_get_stats(self._h, ctypes.byref(st)), "rs_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().rs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_request(stream: dict, outputs=("count", "sum", "min")) -> dict:
    """Pinned host tensors for a server request: inputs from a host stream (numpy uint32)
    and empty output buffers."""
    import numpy as np
    import torch
    req = {"R": int(stream["R"])}
    for k in ("parents", "len", "elements", "ctx"):
        a = stream.get(k)
        req[k] = None if a is None else torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
    R = req["R"]
    req["count"] = torch.empty(R, dtype=torch.int32).pin_memory() if "count" in outputs else None
    req["sum"] = torch.empty(R, dtype=torch.int64).pin_memory() if "sum" in outputs else None
    req["min"] = torch.empty(R, dtype=torch.int32).pin_memory() if "min" in outputs else None
    if stream.get("len") is not None:
        req["total_elements"] = int(np.asarray(stream["len"], dtype=np.uint64).sum())
    return req


def to_device(stream: dict) -> dict:
    """Copy a host stream (numpy uint32 arrays) to CUDA tensors (int32 views of the bits)."""
    import numpy as np
    import torch
    dev = {"R": int(stream["R"])}
    for k in ("parents", "len", "offsets", "elements", "ctx"):
        a = stream.get(k)
        dev[k] = None if a is None else torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    if stream.get("len") is not None:
        dev["total_elements"] = int(np.asarray(stream["len"], dtype=np.uint64).sum())
    elif stream.get("offsets") is not None:
        o = stream["offsets"]
        dev["total_elements"] = int(o[-1]) - int(o[0]) if len(o) else 0
    return dev


def results_to_numpy(out: dict) -> dict:
    """Device result tensors -> numpy with the unsigned types of the ABI."""
    import numpy as np
    res = {}
    if out.get("count") is not None:
        res["count"] = out["count"].cpu().numpy().view(np.uint32)
    if out.get("sum") is not None:
        res["sum"] = out["sum"].cpu().numpy().view(np.uint64)
    if out.get("min") is not None:
        res["min"] = out["min"].cpu().numpy().view(np.uint32)
    if out.get("values") is not None:
        res["values"] = out["values"].cpu().numpy().view(np.uint32)
    for k, dt in (("count2", np.uint32), ("sum2", np.uint64), ("min2", np.uint32)):
        if out.get(k) is not None:
            res[k] = out[k].cpu().numpy().view(dt)
    return res


def run_stream(stages, stream: dict, strategy="tag", outputs=("count", "sum", "min"), inputs=None, **opts):
    """One-shot helper: upload a host stream, run the pipeline once, return numpy
    results and the run's statistics.  The output arrays start filled with a sentinel,
    so a region the run leaves unwritten shows up in the results."""
    import torch
    p = Pipeline(stages, strategy=strategy, inputs=inputs, **opts)
    dev = to_device(stream)
    out = p.submit(dev, outputs=outputs)
    for k in ("count", "sum", "min", "values", "count2", "sum2", "min2"):
        if out.get(k) is not None:
            out[k].fill_(0x5A5A5A5A)
    p.run()
    st = p.stats()
    torch.cuda.synchronize()
    res = results_to_numpy(out)
    p.close()
    return res, st
