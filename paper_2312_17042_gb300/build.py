"""Build the CUDA library libcteno.so in-tree for sm_103a (GB300).

Every translation unit is compiled in parallel: the CUDA sources with nvcc
(-gencode arch=compute_103a,code=sm_103a), the host C++ sources with g++ (-ffp-contract=off so
that x86-64 and aarch64 builds round identically, OpenMP for the stencil search). The objects
are linked into paper_2312_17042_gb300/libcteno.so with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcteno.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU = ["setup.cu", "flux.cu", "recon_2d.cu", "recon_3d.cu", "recon_2d_high.cu", "alu_peak.cu", "noalloc.cu"]
CPP = ["api.cpp", "mesh.cpp", "tables.cpp"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "include")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))] + [
        os.path.join(INCLUDE, "cteno.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in CU:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I" + INCLUDE, "-c", os.path.join(CSRC, f), "-o", obj]
        if ptxas_info:
            cmd.insert(2, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for f in CPP:
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fopenmp",
               "-I" + INCLUDE, "-I" + _cuda_include(), "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for (cmd, _), out in zip(jobs, outs):
            print(" ".join(cmd))
            if out.strip():
                print(out)
    tmp = LIB + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp] + [o for _, o in jobs] + ["-lgomp", "-cudart=static"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
