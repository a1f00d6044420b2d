"""Build librs.so (the CUDA library behind include/rs.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import tempfile
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "librs.so")
PROF_LIB = os.path.join(HERE, "librs_prof.so")   # same code with the per-phase cycle counters
SOURCES = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
DEPS = (SOURCES + sorted(glob.glob(os.path.join(HERE, "csrc", "*.h"))) + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh")))
        + [os.path.join(ROOT, "include", "rs.h")])
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
LINK_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC"]
_lock = threading.Lock()


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in DEPS)


def _compile(cmd: list) -> subprocess.CompletedProcess:
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False, verbose: bool = False, profile: bool = False) -> str:
    """Compile every .cu under csrc/ into librs.so (or, with profile=True, into
    librs_prof.so with the cycle-breakdown counters) if missing or out of date.  The
    translation units compile in parallel, then link into one shared library."""
    lib = PROF_LIB if profile else LIB
    with _lock:
        if not force and not stale(lib):
            return lib
        tmp = lib + f".tmp{os.getpid()}"
        extra = ["-DRS_PROFILE=1"] if profile else []
        inc = ["-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc")]
        with tempfile.TemporaryDirectory(prefix="rs_build_") as d:
            objs = [os.path.join(d, os.path.basename(src)[:-3] + ".o") for src in SOURCES]
            cmds = [[NVCC, *FLAGS, *extra, *inc, "-c", "-o", o, src] for src, o in zip(SOURCES, objs)]
            with concurrent.futures.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
                outs = list(ex.map(_compile, cmds))
            outs.append(_compile([NVCC, *LINK_FLAGS, "-o", tmp, *objs]) if all(o.returncode == 0 for o in outs)
                        else None)
            failed = [o for o in outs if o is None or o.returncode != 0]
            if failed:
                msg = "".join(o.stdout + o.stderr for o in outs if o is not None and o.returncode != 0)
                raise RuntimeError("nvcc failed:\n" + msg)
        if verbose:
            print("".join(o.stderr for o in outs))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build(force=True, profile=True))
