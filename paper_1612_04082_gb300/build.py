"""Build of the kifmm_elastic C-ABI library for sm_103a (in-tree, no cmake).

Each CUDA translation unit is compiled by nvcc in parallel, the FP64 host precompute by
g++ with OpenMP, and everything is linked into ``_lib/libkifmm_elastic.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libkifmm_elastic.so")
CU = ["api.cu", "direct.cu", "direct_hi.cu", "tree.cu", "fmm.cu", "bem.cu", "direct_noalloc.cu", "mlp.cu", "peak.cu"]
CPP = ["precompute.cpp", "periodic.cpp", "voxel.cpp", "shard.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 denormals flush to zero in the FMM kernels: their operands are nowhere near the
# denormal range, and the flush drops the denormal handling around the reciprocal square
# root of every pair evaluation.
EXTRA = {"fmm.cu": ["-ftz=true"]}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cu", ".cuh", ".cpp", ".h"))] + \
        [os.path.join(HERE, "..", "include", "kifmm_elastic.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(nvcc))
    procs, objs = [], []
    for f in CU:
        obj = os.path.join(OUT, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", *EXTRA.get(f, []), "-Xcompiler", "-fPIC", "-Xptxas",
               "-v" if verbose else "-O3", "-c", os.path.join(SRC, f), "-o", obj]
        procs.append((f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for f in CPP:
        obj = os.path.join(OUT, f + ".o")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", f"-I{cuda_home}/include", "-c",
               os.path.join(SRC, f), "-o", obj]
        procs.append((f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for f, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(f)
    if failed:
        raise RuntimeError(f"compilation failed: {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode:
        sys.stderr.write(r.stdout.decode(errors="replace"))
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
