"""Build step of the CUDA library: nvcc for sm_103a, in tree.

Compiles every ``csrc/*.cu`` translation unit in parallel and links them into
``_lib/libfse.so`` (static CUDA runtime), and the same units again with
``-DFSE_BOUNDS_CHECK`` into ``_lib/libfse_checked.so`` (the kernels check
their shared-memory, output and block-list indices and report violations
through ``fse_sync``).  Only ``-gencode arch=compute_103a,code=sm_103a`` is
emitted: the library targets GB300 alone.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libfse.so")
LIB_CHECKED = os.path.join(LIBDIR, "libfse_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfse.so")


def _deps() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def needs_build() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_CHECKED)):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return any(os.path.getmtime(p) > t for p in _deps())


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libfse.so and libfse_checked.so if any source is
    newer than either; returns the path of libfse.so."""
    if not force and not needs_build():
        return LIB
    nvcc = _nvcc()
    os.makedirs(LIBDIR, exist_ok=True)
    variants = [(LIB, "obj", []), (LIB_CHECKED, "obj_checked", ["-DFSE_BOUNDS_CHECK"])]
    for _lib, sub, _flags in variants:
        os.makedirs(os.path.join(LIBDIR, sub), exist_ok=True)
    units = sorted(glob.glob(os.path.join(CSRC, "*.cu")))

    def compile_one(job):
        src, sub, flags = job
        obj = os.path.join(LIBDIR, sub, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    jobs = [(u, sub, flags) for _lib, sub, flags in variants for u in units]
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, _sub, _flags) in enumerate(variants):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + \
            objs[k * len(units):(k + 1) * len(units)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
