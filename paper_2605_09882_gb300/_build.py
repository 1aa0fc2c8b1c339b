"""Builds libraytheia_gb300.so in-tree: nvcc for sm_103a, one object per
translation unit compiled in parallel, static CUDA runtime."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libraytheia_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fno-strict-aliasing"]
CUDA_SOURCES = ["rt_api.cu", "rt_octree.cu", "rt_forward.cu", "rt_adjoint.cu", "rt_gather.cu", "rt_chunked.cu", "rt_batched.cu", "rt_paths.cu", "rt_epilogue.cu", "rt_amr.cu", "rt_noalloc.cu", "rt_host_io.cu"]
CXX_SOURCES = ["rt_healpix.cpp"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    jobs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(obj_dir, src + ".o")
        flags = NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + os.environ.get("RT_NVCC_FLAGS", "").split()
        jobs.append([nvcc(), *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CXX_SOURCES:
        obj = os.path.join(obj_dir, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                     "-c", os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose or ptxas_info:
        for l in logs:
            if l.strip():
                print(l)
    objs = [os.path.join(obj_dir, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    tmp = LIB + f".{os.getpid()}.tmp"
    _run([nvcc(), *ARCH, "-shared", "-cudart=static", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
