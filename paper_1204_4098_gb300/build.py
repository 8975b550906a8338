"""Builds the in-tree CUDA shared library ``liblbm_gb300.so`` for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel) and
the objects are linked with ``nvcc -shared``.  Nothing is installed outside
the package directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm_gb300.so")
REPORT = os.path.join(BUILD, "ptxas_report.txt")  # -Xptxas -v output of the last build

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-Xptxas", "-v", "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]

SOURCES = [
    "lbm_step_f32.cu", "lbm_step_f64.cu", "lbm_step_bf16.cu", "lbm_step_f16.cu",
    "lbm_capi.cu", "lbm_eos_host.cpp", "lbm_noalloc.cu", "lbm_batch.cu", "lbm_mlp.cu",
    "lbm_selftest.cu", "lbm_host_mem.cpp",
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    extra = os.environ.get("LBM_NVCC_EXTRA", "").split()  # e.g. -DLBM_STRIP_MIN_BLOCKS=6
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build_library(verbose: bool = False) -> str:
    """Compile every CUDA/C++ source and link liblbm_gb300.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    with open(REPORT, "w") as f:  # registers / spills / shared memory per kernel
        f.write("".join(log for _, log in results))
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def ptxas_report() -> str:
    """Register / spill / shared-memory report of the last build (-Xptxas -v)."""
    os.makedirs(BUILD, exist_ok=True)
    return "".join(_compile(s)[1] for s in SOURCES if s.endswith(".cu"))


if __name__ == "__main__":
    print(build_library(verbose="-v" in sys.argv))
