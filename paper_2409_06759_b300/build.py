"""Build libccb300.so in-tree for sm_103a (nvcc; no JIT, no torch extension)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libccb300.so")
BUILD = os.path.join(HERE, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]

SOURCES = ["kernels.cu", "accum.cu", "tc_gemm.cu", "no_alloc.cu", "plan.cpp", "cc_api.cpp"]


def _mtime(p: str) -> float:
    return os.path.getmtime(p) if os.path.exists(p) else -1.0


def build(verbose: bool = False, force: bool = False, ptxas_v: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "cc.h"))
    newest_header = max(_mtime(h) for h in headers)
    objs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if not force and _mtime(obj) >= max(_mtime(sp), newest_header):
            continue
        if src.endswith(".cpp"):
            cmd = [NVCC, *COMMON, "-x", "c++", "-c", sp, "-o", obj]
        else:
            cmd = [NVCC, *ARCH, *COMMON, "-c", sp, "-o", obj]
            if ptxas_v:
                cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
    if force or _mtime(OUT) < max(_mtime(o) for o in objs):
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", OUT, *objs]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
    return OUT


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_v="-v" in sys.argv)
