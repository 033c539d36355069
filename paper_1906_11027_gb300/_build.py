"""In-tree build of the CUDA library ``_build/liblbm.so`` for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and the
objects are linked into one shared library.  Objects are rebuilt when their
source or any header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-lineinfo",
                     "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(obj: str, src: str, hdr_time: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < hdr_time


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (if needed) and return the path of liblbm.so."""
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    srcs = sources()
    hdr_time = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    nvcc = _nvcc()
    jobs_list = []
    for src in srcs:
        obj = os.path.join(OUT, "obj", os.path.basename(src)[:-3] + ".o")
        if _stale(obj, src, hdr_time):
            jobs_list.append((src, obj))

    def compile_one(item):
        src, obj = item
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc] + NVCC_FLAGS + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(tmp, obj)
        if verbose and r.stderr.strip():
            print(r.stderr)
        return obj

    if jobs_list:
        n = jobs or min(len(jobs_list), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            list(ex.map(compile_one, jobs_list))
    objs = [os.path.join(OUT, "obj", os.path.basename(s)[:-3] + ".o") for s in srcs]
    if jobs_list or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
