"""Compile the CUDA library for sm_103a into ``libgpcheby.so`` beside this file.

Each translation unit in ``csrc/`` is compiled by nvcc in parallel into
``_build/``; the objects are linked into one shared library with the shared
CUDA runtime (the same libcudart PyTorch loads).  ``python -m
paper_2412_10789_gb300.build`` rebuilds; ``GP_PTXAS_VERBOSE=1`` prints
register and shared-memory usage.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.environ.get("GP_BUILD_SRC") or os.path.join(HERE, "csrc")
# GP_BUILD_TAG / GP_BUILD_DEFINES build a variant library (libgpcheby_<tag>.so)
# with extra -D options, e.g. GP_BUILD_DEFINES="GP_STEP_THREADS=768".
_TAG = os.environ.get("GP_BUILD_TAG", "")
BUILD = os.path.join(HERE, "_build" + (f"_{_TAG}" if _TAG else ""))
LIB = os.path.join(HERE, f"libgpcheby_{_TAG}.so" if _TAG else "libgpcheby.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    # objects and the library are only reused on the machine type that built them
    import platform
    stamp = os.path.join(BUILD, "MACHINE")
    machine = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != machine:
        force = True
        with open(stamp, "w") as f:
            f.write(machine + "\n")
    srcs = _sources()
    hdrs = _headers()
    ptxas_v = os.environ.get("GP_PTXAS_VERBOSE") == "1"
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "--expt-relaxed-constexpr",
              "-I", os.path.join(HERE, "..", "include")] + ARCH
    if ptxas_v:
        common += ["-Xptxas", "-v"]
    for d in os.environ.get("GP_BUILD_DEFINES", "").split():
        common.append("-D" + d)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + hdrs):
            lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
            cmd = [nvcc] + common + lang + ["-c", src, "-o", obj + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
            if (verbose or ptxas_v) and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            os.replace(obj + ".tmp", obj)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-cudart", "shared"] + ARCH + objs + ["-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
