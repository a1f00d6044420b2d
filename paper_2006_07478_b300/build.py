"""Build librs.so (the CUDA library behind include/rs.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import glob
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "librs.so")
PROF_LIB = os.path.join(HERE, "librs_prof.so")   # same code with the per-phase cycle counters
SOURCES = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
DEPS = SOURCES + sorted(glob.glob(os.path.join(HERE, "csrc", "*.h"))) + [os.path.join(ROOT, "include", "rs.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-v"]
_lock = threading.Lock()


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, verbose: bool = False, profile: bool = False) -> str:
    """Compile every .cu under csrc/ into librs.so (or, with profile=True, into
    librs_prof.so with the cycle-breakdown counters) if missing or out of date."""
    lib = PROF_LIB if profile else LIB
    with _lock:
        if not force and not stale(lib):
            return lib
        tmp = lib + f".tmp{os.getpid()}"
        extra = ["-DRS_PROFILE=1"] if profile else []
        cmd = [NVCC, *FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc"),
               "-o", tmp, *SOURCES]
        out = subprocess.run(cmd, capture_output=True, text=True)
        if out.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + out.stdout + out.stderr)
        if verbose:
            print(out.stderr)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build(force=True, profile=True))
