"""Compile the CUDA library in-tree for sm_103a.

Produces ``paper_1305_3162_gb300/_lib/libslp_gb300.so`` from the sources in
``csrc/``: the kernels are compiled by nvcc (one -gencode, compute_103a /
sm_103a, -lineinfo), the host plan code by g++, translation units in
parallel.  Re-running is incremental on source timestamps.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libslp_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU_SOURCES = ["k_grid.cu", "k_fft.cu", "k_near.cu", "k_static.cu", "k_tri.cu", "k_fem.cu"]
CPP_SOURCES = ["slp_plan.cpp", "slp_batch.cpp", "slp_serve.cpp", "slp_fem.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _headers():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                out.append(os.path.join(d, f))
    return out


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = "nvcc"
    hdrs = _headers()
    jobs = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "1444",
                   "-I", INCLUDE, "-c", s, "-o", o]
            jobs.append(cmd)
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cpp", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wno-deprecated-declarations", "-I", os.path.join(cuda, "include"),
                   "-I", INCLUDE,
                   "-c", s, "-o", o]
            jobs.append(cmd)
    procs = [(cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for cmd in jobs]
    failed = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if pr.returncode != 0:
            failed.append(cmd[-1])
    if failed:
        raise RuntimeError(f"compilation failed: {failed}")
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart", "-lpthread"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
