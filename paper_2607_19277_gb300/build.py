"""Build libagile.so in-tree for sm_103a (nvcc, one -gencode, translation units in parallel).

Usage: python -m paper_2607_19277_gb300.build   (or call build())
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libagile.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU_SOURCES = ["stage_hd.cu", "stage_mhd.cu", "stage_mhd_res.cu", "stage_srhd.cu", "stage_srhd_synge.cu", "stage_ffhd.cu", "aux_kernels.cu",
              "cooling.cu", "capi.cu"]
CPP_SOURCES = ["mesh.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
# Every FP32 kernel uses the fast single-precision divide and square root (max 2 ulp) and
# flushes denormals, so that a quantity formed in two kernels (the CFL speeds fused into the
# last stage and the standalone speed reduction) has the same bits; FP64 arithmetic is
# unaffected by these flags.
FAST_FP32 = ["--prec-div=false", "--prec-sqrt=false", "--ftz=true"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    # objects built with other flags are stale too
    stamp = os.path.join(OUT, "flags.txt")
    flags = " ".join(ARCH + NVCC_FLAGS + FAST_FP32)
    if not os.path.exists(stamp) or open(stamp).read() != flags:
        force = True
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "agile.h"))
    jobs = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            extra = FAST_FP32
            jobs.append([nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc] + NVCC_FLAGS + ["-x", "c++", "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, LIB)
        with open(stamp, "w") as f:
            f.write(flags)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
