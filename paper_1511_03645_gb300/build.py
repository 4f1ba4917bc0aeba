"""Build libadjamr.so (CUDA kernels for sm_103a + C++ host code) in-tree.

Translation units compile in parallel: the .cu files with nvcc
(-gencode arch=compute_103a,code=sm_103a, --fmad=false so every FP64
operation rounds as written), the .cpp files with g++ -ffp-contract=off.
Output: paper_1511_03645_gb300/_build/libadjamr.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libadjamr.so")

CU = ["kernels_step.cu", "kernels_amr.cu", "fp64_peak.cu", "noalloc.cu"]
CPP = ["hierarchy.cpp", "batch.cpp", "serve.cpp"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libadjamr")


def _cuda_home(nvcc):
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [os.path.join(CSRC, "internal.h"), os.path.join(INC, "adjamr.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cuda = _cuda_home(nvcc)
    jobs = []
    objs = []
    for f in CU:
        o = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "-I", INC, "-I", CSRC, "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_v:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((f, cmd))
        objs.append(o)
    for f in CPP:
        o = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall",
               "-I", INC, "-I", CSRC, "-I", os.path.join(cuda, "include"), "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append((f, cmd))
        objs.append(o)
    procs = [(f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for f, cmd in jobs]
    failed = []
    for f, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or (verbose and out):
            sys.stderr.write(f"--- {f}\n{out}\n")
        if p.returncode != 0:
            failed.append(f)
    if failed:
        raise RuntimeError("libadjamr build failed: " + ", ".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libadjamr link failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas" in sys.argv))
