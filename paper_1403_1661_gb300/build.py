"""Build the native library libswe_gb300.so in-tree (paper_1403_1661_gb300/_build/).

Host C++ with g++, kernels with nvcc for sm_103a only, compiled in parallel and
linked with the static CUDA runtime. Objects are rebuilt when a source or header
is newer than the object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(BUILD, "libswe_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The front end forms fused multiply-adds; the assembler is not allowed to fuse
# further multiplies and adds on its own, since it compiles a shared out-of-line
# function separately for each calling kernel and could round them differently:
# the stage and limiter bodies then compute the same bits in every kernel.
PTXAS = ["-Xptxas", "--fmad=false"]
CXX_SOURCES = ["refelem.cpp", "mesh.cpp", "solver.cpp"]
CU_SOURCES = ["kernels_n1.cu", "kernels_n2.cu", "kernels_n3.cu", "kernels_n4.cu", "kernels_n5.cu",
              "kernels_c2.cu", "kernels_c3.cu", "kernels_c4.cu", "kernels_c5.cu",
              "kernels_r2.cu", "kernels_r3.cu", "kernels_r4.cu", "kernels_r5.cu", "kernels_common.cu",
              "noalloc.cu", "tc05_projection.cu"]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _headers():
    out = [os.path.join(INCLUDE, "swe.h")]
    for f in os.listdir(CSRC):
        if f.endswith((".hpp", ".cuh", ".inc")):
            out.append(os.path.join(CSRC, f))
    return out


def _stale(obj: str, src: str, headers) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, *headers])


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}")
    return r.stdout


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile everything that is out of date and link the shared library; returns its path."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    headers = _headers()
    jobs = []
    objs = []
    for f in CXX_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if _stale(obj, src, headers):
            jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-Wno-unused-function",
                         f"-I{cuda}/include", f"-I{INCLUDE}", "-c", src, "-o", obj])
    for f in CU_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if _stale(obj, src, headers):
            cmd = [nvcc, "-std=c++17", "-O3", *ARCH, *PTXAS, "-lineinfo", "-Xcompiler", "-fPIC",
                   f"-I{INCLUDE}", "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            outs = list(ex.map(lambda c: _run(c, verbose), jobs))
        if ptxas_info:
            for o in outs:
                sys.stdout.write(o)
    if jobs or not os.path.exists(LIB):
        _run([nvcc, "-shared", *ARCH, "-cudart", "static", "-o", LIB, *objs], verbose)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
