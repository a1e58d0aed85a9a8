"""Build libls.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2311_04362_gb300/libls.so``.  Objects go to ``_build/`` at the repo
root.  Nothing here needs a GPU: nvcc cross-compiles.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libls.so")
SOURCES = ["sketch.cu", "factor.cu", "iterate.cu", "batched.cu", "server.cu", "sparse.cu", "api.cu", "noalloc.cu", "fxpass.cu"]
# instruction-rate probe behind bench.py --rates (not part of libls.so)
RATES_LIB = os.path.join(HERE, "librates.so")
RATES_SOURCES = ["rates.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(src_files, out):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in src_files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libls.so and librates.so; returns the libls.so path."""
    _build_lib(SOURCES, LIB, force, verbose)
    _build_lib(RATES_SOURCES, RATES_LIB, force, verbose)
    return LIB


def _build_lib(sources, lib_path, force, verbose):
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "ls.h"))
    nvcc = _nvcc()
    jobs = []
    for s in sources:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OBJ, s.replace(".cu", ".o"))
        if force or _stale([src, *headers], obj):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
                if res.returncode != 0:
                    sys.stderr.write(res.stdout + res.stderr)
                    raise RuntimeError("nvcc failed: " + " ".join(cmd))
                if verbose and (res.stdout or res.stderr):
                    sys.stderr.write(res.stdout + res.stderr)
    objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in sources]
    if force or jobs or _stale(objs, lib_path):
        tmp = lib_path + f".tmp{os.getpid()}"
        res = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("link of " + os.path.basename(lib_path) + " failed")
        os.replace(tmp, lib_path)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
