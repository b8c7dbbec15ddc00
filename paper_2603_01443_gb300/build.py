"""Build the C-ABI library ``libcutsim.so`` in-tree (sm_103a only).

Every CUDA translation unit is compiled with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and the host
C++ units with the system C++ compiler, all in parallel, then linked into
``paper_2603_01443_gb300/libcutsim.so`` against the shared CUDA runtime (the
one PyTorch also loads).  Run ``python -m paper_2603_01443_gb300.build``.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcutsim.so")

CU_SOURCES = ["runtime.cu", "sv_kernels.cu", "merge_kernels.cu", "merge_tc.cu", "merge_ozaki.cu",
              "reduce_kernels.cu",
              "batch.cu", "mlp.cu",
              "gather_static.cu"]
CPP_SOURCES = ["program.cpp", "plan.cpp", "kak.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cxx() -> str:
    for cand in (os.environ.get("CXX"), shutil.which("g++"), shutil.which("c++")):
        if cand:
            return cand
    raise RuntimeError("no host C++ compiler found")


def commands(ptxas_verbose: bool = False):
    nvcc = _nvcc()
    cxx = _cxx()
    inc = ["-I", INCLUDE, "-I", CSRC]
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for src in CPP_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [cxx, "-O2", "-std=c++17", "-fPIC", "-Wall", *inc, "-I", cuda_inc, "-c",
               os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", LIB] + [o for _, o in jobs]
    return jobs, link


def build(verbose: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    jobs, link = commands(ptxas_verbose)
    procs = []
    for cmd, obj in jobs:
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((cmd, text))
        elif text.strip() and (verbose or ptxas_verbose):
            print(text)
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("compilation failed:\n" + msg)
    if verbose:
        print(" ".join(link), flush=True)
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv))
