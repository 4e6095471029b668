"""Builds libapril.so in-tree: the host builder (g++) and the sm_103a CUDA
kernels (nvcc), compiled in parallel and linked into one shared library."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libapril.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXX_SOURCES = ["build_sets.cpp"]
CU_SOURCES = ["filter.cu", "server.cu", "select.cu", "build_device.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, s) for s in CXX_SOURCES + CU_SOURCES] + \
        [os.path.join(CSRC, "april_internal.h"), os.path.join(HERE, "..", "include", "april.h")] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(s) <= t for s in _sources() if os.path.exists(s))


def build(force: bool = False, verbose: bool = False, out: str | None = None, defines=()) -> str:
    """Compile libapril.so (or `out`), with optional -D definitions."""
    target = out or OUT
    if not force and out is None and up_to_date():
        return OUT
    build_dir = BUILD if out is None else out + "_build"
    os.makedirs(build_dir, exist_ok=True)
    dflags = [f"-D{d}" for d in defines]
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in CXX_SOURCES:
        o = os.path.join(build_dir, s + ".o")
        objs.append(o)
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-Wall", *dflags, "-c",
                     os.path.join(CSRC, s), "-o", o])
    for s in CU_SOURCES:
        o = os.path.join(build_dir, s + ".o")
        objs.append(o)
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *dflags,
                     "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3",
                     "-c", os.path.join(CSRC, s), "-o", o])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    failed = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(j))
    if failed:
        raise RuntimeError("compilation failed: " + "; ".join(failed))
    tmp = target + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
