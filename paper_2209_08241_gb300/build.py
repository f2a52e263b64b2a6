"""In-tree build of the CUDA library ``libnrm.so`` for sm_103a.

Compiles the translation units under ``csrc/`` in parallel with nvcc (one
``-gencode arch=compute_103a,code=sm_103a``), links them into a shared library
with the CUDA runtime linked statically (so it loads on machines without a
GPU, where its calls return NRM_ERR_NO_DEVICE), and writes it to
``_build/libnrm.so``. No torch types cross this library's interface.

With ``debug=True`` (``--debug``) it builds the checking variant
``_build/libnrm_debug.so`` instead (``-DNRM_DEBUG_CHECKS``: every shared-memory
access and every geometry-dependent global access of the kernels is
range-checked; a failed check skips the access, prints the site and records
NRM_ERR_BOUNDS in the status word). The binding loads it when the environment
variable NRM_LIB_VARIANT is ``debug``.

Usage: ``python -m paper_2209_08241_gb300.build [--force] [--verbose] [--debug]``.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libnrm.so")
DEBUG_BUILD = os.path.join(BUILD, "debug")
DEBUG_LIB = os.path.join(BUILD, "libnrm_debug.so")

SOURCES = ["nrm_forward.cu", "nrm_forward_points.cu", "nrm_forward_param.cu", "nrm_backward.cu", "nrm_api.cpp", "nrm_noalloc.cu", "nrm_eval.cu", "nrm_planefit.cu", "nrm_multiscale.cu", "nrm_selftest.cu"]
HEADERS = ["nrm_internal.h", "nrm_device.cuh", "nrm_forward_kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnrm.so")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "nrm.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(debug: bool = False) -> bool:
    lib = DEBUG_LIB if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(nvcc: str, src: str, obj: str, verbose: bool, debug: bool = False) -> None:
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
           f"-I{INCLUDE}", f"-I{CSRC}", "-c", os.path.join(CSRC, src), "-o", obj]
    if debug:
        cmd.insert(1, "-DNRM_DEBUG_CHECKS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds ``_build/libnrm.so`` (or, with ``debug``, the checking variant
    ``_build/libnrm_debug.so``) if any input is newer; returns its path."""
    lib = DEBUG_LIB if debug else LIB
    if not force and up_to_date(debug):
        return lib
    nvcc = _nvcc()
    objdir = DEBUG_BUILD if debug else BUILD
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        futs = [ex.submit(_compile, nvcc, s, o, verbose, debug) for s, o in zip(SOURCES, objs)]
        for f in futs:
            f.result()
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
