"""In-tree build of libsdugks.so for sm_103a (nvcc + g++, no cmake).

The CUDA translation units are compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a``; the FP64 step unit additionally with
``--fmad=false`` so that its FP64 arithmetic rounds every product and sum.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libsdugks.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_UNITS = {
    "k_step_fp64.cu": ["--fmad=false"],
    "k_step_fp32.cu": [],
    "k_cart_fp64.cu": ["--fmad=false"],
    "k_cart.cu": [],
    "k_util.cu": [],
    "k_residual_noalloc.cu": [],
    "k_batch.cu": [],
    "k_dvm.cu": [],
}
CXX_UNITS = ["sdugks_host.cpp"]
HEADERS = ["sdugks_internal.h", "d2q9.cuh", "step_tiled.cuh", "step_cart.cuh"]


def _sources():
    return ([os.path.join(CSRC, u) for u in list(CU_UNITS) + CXX_UNITS + HEADERS]
            + [os.path.join(INCLUDE, "sdugks.h"), os.path.abspath(__file__)])


def _stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile the library if any source is newer than it; returns the .so path."""
    if not force and not _stale():
        return SO
    os.makedirs(BUILD, exist_ok=True)
    incs = ["-I", CSRC, "-I", INCLUDE]
    jobs, objs = [], []
    for unit, extra in CU_UNITS.items():
        obj = os.path.join(BUILD, unit + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *incs, *extra,
               "-c", os.path.join(CSRC, unit), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((unit, cmd))
        objs.append(obj)
    for unit in CXX_UNITS:
        obj = os.path.join(BUILD, unit + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function", *incs,
               "-I", os.path.join(CUDA_HOME, "include"), "-c", os.path.join(CSRC, unit), "-o", obj]
        jobs.append((unit, cmd))
        objs.append(obj)
    procs = [(u, c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for u, c in jobs]
    failed = []
    for u, c, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0 or ptxas_info:
            sys.stderr.write(f"--- {u}\n{out}")
        if p.returncode != 0:
            failed.append(u)
    if failed:
        raise RuntimeError(f"libsdugks build failed in {failed}")
    tmp = SO + f".tmp{os.getpid()}"
    link = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libsdugks link failed:\n" + r.stdout)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
