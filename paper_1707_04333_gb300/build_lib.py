"""Build libfetdpic.so in-tree: sm_103a CUDA kernels + C++ host setup.

    python -m paper_1707_04333_gb300.build_lib

Translation units compile in parallel; the FP64 kernel file is built with
-fmad=false (no FMA contraction) and all host code with -ffp-contract=off, so
the plain-FP64 path rounds exactly as its formulas are written.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfetdpic.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = {
    "kernels_fp64.cu": ["-fmad=false"],
    "kernels_fp32.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "kernels_common.cu": [],
    "kernels_check.cu": [],
    "fetdpic_api.cu": [],
}
CPP_SOURCES = ["mesh_setup.cpp"]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _sources():
    return [os.path.join(SRC, f) for f in list(CU_SOURCES) + CPP_SOURCES] + \
        [os.path.join(SRC, "fetdpic_internal.h"), os.path.join(SRC, "field_device.cuh"),
         os.path.join(INCLUDE, "fetdpic.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    home = _cuda_home(nvcc)
    common = ["-O3", "-std=c++17", "-lineinfo", "-I", INCLUDE, "-I", SRC,
              "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math"]
    jobs = []
    for f, extra in CU_SOURCES.items():
        obj = os.path.join(OUT_DIR, f + ".o")
        jobs.append((obj, [nvcc, *ARCH, *common, *extra, "-c", os.path.join(SRC, f), "-o", obj]))
    for f in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        jobs.append((obj, ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                           "-pthread", "-I", INCLUDE, "-I", SRC, "-I", os.path.join(home, "include"),
                           "-c", os.path.join(SRC, f), "-o", obj]))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(run, [c for _, c in jobs]))
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = os.path.join(home, "lib64")
    run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *[o for o, _ in jobs],
         "-Xlinker", f"-rpath,{libdir}", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
