"""Python front end of the sequential CPU oracle (oracle/rs_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module; the library's own code path never does.
It builds oracle/liboracle.so with gcc on first use and calls it through ctypes.

Pipelines are lists of plain tuples, e.g.
    [("enum_hash",), ("filter_mod", 2, 0), ("map_mul", 2654435761, 0), ("aggregate",)]
and streams are dicts with keys R, parents, len, offsets, elements, ctx (numpy
uint32 arrays or None), as drawn by the seeded workload generators.

Parity: pinned (see rs_oracle.c's header and tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {
    "enum_hash": 1,
    "enum_load": 2,
    "filter_mod": 10,
    "filter_hash_ctx": 11,
    "filter_weight_lt": 12,
    "map_mul": 20,
    "expand": 30,
    "aggregate": 40,
    "emit": 50,
}


class OraStage(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("fanout", ctypes.c_uint32),
                ("p0", ctypes.c_uint32), ("p1", ctypes.c_uint32),
                ("p2", ctypes.c_uint32), ("p3", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, -O2, pthreads) if it is missing or stale."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                                   "-o", tmp, _SRC, "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.ora_fmix32.argtypes = [ctypes.c_uint32]
        L.ora_fmix32.restype = ctypes.c_uint32
        L.ora_hash32.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.ora_hash32.restype = ctypes.c_uint32
        L.ora_run.argtypes = [ctypes.POINTER(OraStage), ctypes.c_int, ctypes.c_uint64,
                              P, P, P, P, P, P, P, P, ctypes.c_int]
        L.ora_run.restype = ctypes.c_int
        L.ora_run_sampled.argtypes = [ctypes.POINTER(OraStage), ctypes.c_int, ctypes.c_uint64,
                                      P, P, P, P, P, P, ctypes.c_uint64, P, P, P]
        L.ora_run_sampled.restype = ctypes.c_int
        L.ora_run_emit.argtypes = [ctypes.POINTER(OraStage), ctypes.c_int, ctypes.c_uint64,
                                   P, P, P, P, P, ctypes.c_uint32, P, P]
        L.ora_run_emit.restype = ctypes.c_int
        L.ora_run_tree.argtypes = [ctypes.POINTER(OraStage), P, ctypes.c_int, ctypes.c_uint64,
                                   P, P, P, P, P, P, P, P]
        L.ora_run_tree.restype = ctypes.c_int
        _lib = L
    return _lib


def fmix32(x: int) -> int:
    return int(lib().ora_fmix32(x & 0xFFFFFFFF))


def hash32(a: int, b: int) -> int:
    return int(lib().ora_hash32(a & 0xFFFFFFFF, b & 0xFFFFFFFF))


def _stages(pipeline):
    arr = (OraStage * len(pipeline))()
    for i, st in enumerate(pipeline):
        name, args = st[0], [int(a) & 0xFFFFFFFF for a in st[1:]]
        arr[i].op = OPS[name]
        if name == "expand":           # ("expand", k, salt)
            arr[i].fanout = args[0]
            arr[i].p0 = args[1]
        else:
            arr[i].fanout = 1
            for j, a in enumerate(args[:4]):
                setattr(arr[i], f"p{j}", a)
    return arr


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def run(pipeline, stream: dict, threads: int = 1) -> dict:
    """Per-region aggregates {count u32[R], sum u64[R], min u32[R]} of the stream."""
    R = int(stream["R"])
    count = np.empty(R, dtype=np.uint32)
    sm = np.empty(R, dtype=np.uint64)
    mn = np.empty(R, dtype=np.uint32)
    st = _stages(pipeline)
    rc = lib().ora_run(st, len(pipeline), R, _ptr(stream.get("parents")), _ptr(stream.get("len")),
                       _ptr(stream.get("offsets")), _ptr(stream.get("elements")), _ptr(stream.get("ctx")),
                       _ptr(count), _ptr(sm), _ptr(mn), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the pipeline or stream")
    return {"count": count, "sum": sm, "min": mn}


def run_sampled(pipeline, stream: dict, idx) -> dict:
    """Aggregates of the listed regions only (results in the order of idx)."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    m = idx.shape[0]
    count = np.empty(m, dtype=np.uint32)
    sm = np.empty(m, dtype=np.uint64)
    mn = np.empty(m, dtype=np.uint32)
    st = _stages(pipeline)
    rc = lib().ora_run_sampled(st, len(pipeline), int(stream["R"]), _ptr(stream.get("parents")),
                               _ptr(stream.get("len")), _ptr(stream.get("offsets")),
                               _ptr(stream.get("elements")), _ptr(stream.get("ctx")),
                               _ptr(idx), m, _ptr(count), _ptr(sm), _ptr(mn))
    if rc != 0:
        raise ValueError("oracle rejected the pipeline, stream or sample")
    return {"count": count, "sum": sm, "min": mn}


def fanout_product(pipeline) -> int:
    """F: the product of the element stages' maximum fan-outs (an expansion's k, 1
    otherwise); region r's segment of an emit sink's output holds F * L_r values."""
    F = 1
    for st in pipeline[1:-1]:
        if st[0] == "expand":
            F *= max(1, int(st[1]))
    return F


def _offsets(stream: dict) -> np.ndarray:
    if stream.get("offsets") is not None:
        o = stream["offsets"].astype(np.int64)
        return o - o[0]
    return np.concatenate(([0], np.cumsum(stream["len"].astype(np.int64))))


def run_emit(pipeline, stream: dict) -> dict:
    """Emit sink: {count u32[R], values u32[F * N], start i64[R + 1]}; region r's
    survivors are values[start[r] : start[r] + count[r]], in stream order
    (start[r] = F * (off_r - off_0))."""
    R = int(stream["R"])
    F = fanout_product(pipeline)
    off = _offsets(stream)
    N = int(off[-1])
    values = np.zeros(max(1, F * N), dtype=np.uint32)
    count = np.empty(R, dtype=np.uint32)
    st = _stages(pipeline)
    rc = lib().ora_run_emit(st, len(pipeline), R, _ptr(stream.get("parents")), _ptr(stream.get("len")),
                            _ptr(stream.get("offsets")), _ptr(stream.get("elements")), _ptr(stream.get("ctx")),
                            F, _ptr(values), _ptr(count))
    if rc != 0:
        raise ValueError("oracle rejected the pipeline or stream")
    return {"count": count, "values": values, "start": F * off}


def run_tree(pipeline, inputs, stream: dict) -> list:
    """Tree topology (Figure 1(b)): stage s reads the output of stage inputs[s]
    (inputs[0] is ignored; inputs[1] must be 0).  Returns one dict {count, sum, min}
    per aggregate leaf, in stage order."""
    R = int(stream["R"])
    n = len(pipeline)
    sinks = sum(1 for st in pipeline[1:] if st[0] == "aggregate")
    cnt = [np.empty(R, dtype=np.uint32) for _ in range(sinks)]
    sm = [np.empty(R, dtype=np.uint64) for _ in range(sinks)]
    mn = [np.empty(R, dtype=np.uint32) for _ in range(sinks)]
    up = (ctypes.c_int32 * n)(*([-1] + [int(i) for i in inputs[1:]]))
    pc = (ctypes.c_void_p * max(1, sinks))(*[a.ctypes.data for a in cnt])
    ps = (ctypes.c_void_p * max(1, sinks))(*[a.ctypes.data for a in sm])
    pm = (ctypes.c_void_p * max(1, sinks))(*[a.ctypes.data for a in mn])
    rc = lib().ora_run_tree(_stages(pipeline), up, n, R, _ptr(stream.get("parents")), _ptr(stream.get("len")),
                            _ptr(stream.get("offsets")), _ptr(stream.get("elements")), _ptr(stream.get("ctx")),
                            pc, ps, pm)
    if rc != sinks:
        raise ValueError("oracle rejected the tree or stream")
    return [{"count": c, "sum": s_, "min": m} for c, s_, m in zip(cnt, sm, mn)]
