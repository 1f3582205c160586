"""Builds the native library ``_build/libscion.so`` for sm_103a.

Host code (the BVH builder and packer) is compiled with g++ (C++17, OpenMP,
no floating-point contraction); the C ABI and the traversal kernels with nvcc
(``-gencode arch=compute_103a,code=sm_103a``, ``--fmad=false`` so that only
explicit fmaf calls fuse). The kernel families are separate translation units
built in parallel.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libscion.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "--fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false",
              "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
             "-Wall", "-I", INCLUDE]

FAMILIES = [(f"own_p{p}", ["-DSCION_OWN=1", f"-DSCION_PREC={p}"]) for p in (0, 3, 4, 6)] + [
    (f"w{w}_p{p}", [f"-DSCION_W={w}", f"-DSCION_PREC={p}"]) for w in (2, 4, 8) for p in (0, 1, 2, 5)]


def _sources():
    out = []
    for name in os.listdir(CSRC):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            out.append(os.path.join(CSRC, name))
    out += [os.path.join(INCLUDE, n) for n in os.listdir(INCLUDE)]
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libscion.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    for fam, defs in FAMILIES:
        obj = os.path.join(BUILD, f"trace_{fam}.o")
        jobs.append([NVCC, *ARCH, *NVCC_FLAGS, *extra, *defs, "-c",
                     os.path.join(CSRC, "trace_inst.cu"), "-o", obj])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, "-Xcompiler", "-fopenmp", "-c",
                 os.path.join(CSRC, "api.cu"), "-o", os.path.join(BUILD, "api.o")])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, "backward.cu"), "-o",
                 os.path.join(BUILD, "backward.o")])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, "lbvh.cu"), "-o",
                 os.path.join(BUILD, "lbvh.o")])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, "gpack.cu"), "-o",
                 os.path.join(BUILD, "gpack.o")])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, "refit.cu"), "-o",
                 os.path.join(BUILD, "refit.o")])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, "batched.cu"), "-o",
                 os.path.join(BUILD, "batched.o")])
    jobs.append([NVCC, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, "membw.cu"), "-o",
                 os.path.join(BUILD, "membw.o")])
    jobs.append(["g++", *CXX_FLAGS, "-c", os.path.join(CSRC, "builder.cpp"), "-o",
                 os.path.join(BUILD, "builder.o")])
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose or ptxas_info:
        for lg in logs:
            if lg.strip():
                print(lg, file=sys.stderr)
    objs = [j[-1] for j in jobs]
    tmp = LIB + f".{os.getpid()}.tmp"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
