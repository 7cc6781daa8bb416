"""Builds liblc.so in-tree (``paper_1804_09996_gb300/_lib/liblc.so``) for sm_103a.

The CUDA translation unit is compiled by nvcc, the host units by g++, in parallel, and
linked by nvcc with the static CUDA runtime.  Re-running is cheap: objects are rebuilt
only when a source or header is newer.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU = ["lc_search.cu", "lc_walk_f32.cu", "lc_walk_f16.cu", "lc_build_gpu.cu"]
CPP = ["lc_capi.cpp", "lc_build.cpp", "lc_serve.cpp", "lc_tune.cpp"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblc.so")
    return p


def _deps():
    hdrs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(INCLUDE, "lc.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    hdr_time = _deps()
    jobs = []
    objs = []
    for f in CU + CPP:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT_DIR, f.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time):
            continue
        if f.endswith(".cu"):
            cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                   "-c", src, "-o", obj]
        else:
            cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
            # no multiply-add contraction: the host build gives the same bits on x86 and Arm, and
            # the device codeword assignment reproduces it exactly
            cmd = ["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fPIC", "-pthread", "-Wall", "-I", cuda_inc,
                   "-c", src, "-o", obj]
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, pr in jobs:
        out, _ = pr.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if pr.returncode != 0:
            failed.append((cmd, out))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError(f"building liblc.so failed:\n{msg}")
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("linking liblc.so failed:\n" + " ".join(cmd) + "\n" + r.stdout)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
