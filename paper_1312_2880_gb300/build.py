"""Build the CUDA library ``libhz.so`` in-tree with nvcc for sm_103a.

Each translation unit compiles in its own nvcc process (in parallel); the objects go to
``_build/`` beside this file and are linked with the static CUDA runtime. Only stale objects are
rebuilt. Run ``python -m paper_1312_2880_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libhz.so")
SOURCES = ("hz_vcycle.cu", "hz_fused.cu", "hz_stream.cu", "hz_kaczmarz.cu", "hz_tail.cu", "hz_krylov.cu",
           "hz_capi.cu", "hz_noalloc.cu", "hz_probe.cu", "hz_kgrid.cu", "hz_ray.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libhz.so")
    return exe


def _headers_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths.append(os.path.join(INCLUDE, "hz.h"))
    return max(os.path.getmtime(p) for p in paths)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> str:
    """Compile stale sources and link ``libhz.so``; returns the library path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_mtime()
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    jobs = []
    for s in srcs:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD_DIR, s.replace(".cu", ".o"))
        stale = force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr)
        extra = ["-Xptxas", "-v"] if ptxas_info else []
        jobs.append((src, obj, stale, [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]))

    def run(job):
        src, obj, stale, cmd = job
        if not stale:
            return src, ""
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
        return src, res.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for src, log in ex.map(run, jobs):
            if verbose and log:
                print(f"--- {os.path.basename(src)}\n{log}", file=sys.stderr)
    objs = [j[1] for j in jobs]
    if force or any(j[2] for j in jobs) or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
        os.path.getmtime(o) for o in objs
    ):
        tmp = LIB_PATH + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, ptxas_info="--ptxas" in sys.argv))
