"""Build of the CUDA library ``libspmps.so`` (sm_103a) into ``paper_1703_04789_gb300/_lib``.

Plain ``nvcc``: one object per translation unit, compiled in parallel, then one shared link.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libspmps.so")
SOURCES = ["host.cpp", "mpo_ab_initio.cpp", "kernels.cu", "engine.cu", "sweep.cu", "metric.cu", "noalloc.cu", "mlp.cu", "learned.cu", "tf32.cu", "state_io.cu", "properties.cu", "peaks.cu", "tc_gemm.cu", "ozaki.cu", "screen.cu", "excited.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src: str) -> str:
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(HERE, "..", "include"), "-x", "cu" if src.endswith(".cu") else "c++",
           "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False) -> str:
    """Compile every translation unit and link libspmps.so; returns the library path."""
    os.makedirs(OUT, exist_ok=True)
    newest_src = max(os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC))
    newest_src = max(newest_src, os.path.getmtime(os.path.join(HERE, "..", "include", "spmps.h")))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > newest_src:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    cmd = [_nvcc(), "-shared", *ARCH, "-o", LIB, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force=True))
