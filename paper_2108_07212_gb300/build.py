"""Build libperidem.so (sm_103a) in-tree with nvcc / g++.

Kernels of the FP64 path are compiled with ``-fmad=false`` so their FP64
expressions round exactly as written; the FP32-split and tensor-core kernels
keep FMA contraction.  The CUDA runtime is linked statically, so the library
loads on a machine without a GPU (meshing and bond building are host-only).
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
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libperidem.so")
INC = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, extra flags[, object name]): pd_persist.cu builds once per precision
# and thread count per node, so that the persistent kernels compile in parallel
_FP64_FLAGS = ["-fmad=false"]
# FP32-split force kernels: divisions and square roots to within 2 ulp (far
# inside the path's 1e-5 force tolerance) instead of the IEEE sequences
_FP32_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]
CU_SOURCES = [
    ("pd_common.cu", _FP64_FLAGS),
    ("pd_step64.cu", _FP64_FLAGS),
    ("pd_step32.cu", _FP32_FLAGS),
    ("pd_noalloc.cu", []),
    ("pd_mlp.cu", []),
    ("pd_surrogate.cu", []),
] + [("pd_persist.cu", (_FP32_FLAGS if fp32 else _FP64_FLAGS) + [f"-DPD_PERSIST_FP32={fp32}", f"-DPD_PERSIST_LANES={lanes}"],
      f"pd_persist{32 if fp32 else 64}_l{lanes}.o") for fp32 in (1, 0) for lanes in (1, 2, 4, 8)]
CPP_SOURCES = ["pd_host.cpp", "pd_basis.cpp"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_include(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def _sources():
    return sorted({os.path.join(CSRC, e[0]) for e in CU_SOURCES}) + [os.path.join(CSRC, s) for s in CPP_SOURCES] + [
        os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))] + [
        os.path.join(INC, "peridem.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cuinc = _cuda_include(nvcc)
    jobs = []
    for entry in CU_SOURCES:
        src, extra = entry[0], entry[1]
        obj = os.path.join(OUT, entry[2] if len(entry) > 2 else src + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
               *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    for src in CPP_SOURCES:
        obj = os.path.join(OUT, src + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INC, "-I", CSRC, "-I", cuinc,
               "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(max(os.cpu_count() or 1, 1), 16, len(jobs))) as ex:
        outs = list(ex.map(run, [c for c, _ in jobs]))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for _, o in jobs] + ["-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
