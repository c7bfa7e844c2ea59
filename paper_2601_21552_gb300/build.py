"""Build libscuba.so in-tree for sm_103a (GB300).

Host C++ translation units are compiled with g++, CUDA ones with nvcc
(-gencode arch=compute_103a,code=sm_103a), all in parallel, then linked into
paper_2601_21552_gb300/_build/libscuba.so. No cmake.

The same sources are also linked, with the CUDA units compiled under
-DSCUBA_CHECKED, into _build/libscuba_checked.so: the checked build, whose
kernels test their indexes into the instance's buffers and report a failed
check through the call's status (SCUBA_ERR_INTERNAL and a message naming the
site) instead of touching memory out of bounds. The binding loads it when
SCUBA_LIBRARY=checked is set.
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libscuba.so")
LIB_CHECKED = os.path.join(OUT, "libscuba_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

HOST_SRCS = ["encoder.cpp", "verify.cpp", "host_api.cpp"]
CUDA_SRCS = ["solver.cu", "mlp.cu"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return [os.path.join(CSRC, s) for s in HOST_SRCS + CUDA_SRCS]


def _deps():
    extra = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return _sources() + extra + [os.path.join(ROOT, "include", "scuba.h")]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and all(os.path.exists(x) and os.path.getmtime(x) >= newest
                         for x in (LIB, LIB_CHECKED)):
        return LIB
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(_nvcc()))), "include")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", cuda_inc]
    defs = []
    for var in ("SCUBA_LEARNED_MINBLOCKS", "SCUBA_CDCL_MINBLOCKS"):
        if os.environ.get(var):
            defs.append(f"-D{var}=" + str(int(os.environ[var])))
    jobs = []
    objs = []
    for s in HOST_SRCS:
        o = os.path.join(OUT, s + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-c", os.path.join(CSRC, s),
                     "-o", o] + inc)
    objs_checked = list(objs)
    for s in CUDA_SRCS:
        for checked in (False, True):
            o = os.path.join(OUT, s + (".checked.o" if checked else ".o"))
            (objs_checked if checked else objs).append(o)
            jobs.append([_nvcc(), "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                         "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, s), "-o", o]
                        + ARCH + inc + defs + (["-DSCUBA_CHECKED"] if checked else []))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    for lib, o in ((LIB_CHECKED, objs_checked), (LIB, objs)):
        tmp = lib + f".{os.getpid()}.tmp"
        run([_nvcc(), "-shared", "-o", tmp] + o + ARCH + ["-lcudart", "-lpthread"])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
