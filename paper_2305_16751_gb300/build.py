"""Builds the CUDA library (sm_103a) in-tree with nvcc.

The library is ``libdomagg.so`` beside this file.  Translation units are
compiled in parallel, then linked; nothing is installed anywhere.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libdomagg.so")
# the checked build: the same sources with DOMAGG_CHECKED (every kernel tests
# its computed indices and reports DOMAGG_ERR_BOUNDS instead of touching
# memory outside a buffer); for tests and debugging
LIB_CHECKED = os.path.join(HERE, "libdomagg_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["domagg.cu", "sort.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "domagg.h"))
    return files


def _stale() -> bool:
    for lib in (LIB, LIB_CHECKED):
        if not os.path.exists(lib):
            return True
        t = os.path.getmtime(lib)
        if any(os.path.getmtime(f) > t for f in _deps()):
            return True
    return False


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    # tuning constants (e.g. "-DDOMAGG_SEG_THREADS=128"), for sweeps
    extra += [f for f in os.environ.get("DOMAGG_NVCC_DEFINES", "").split() if f.startswith("-D")]

    def compile_one(job) -> str:
        src, checked = job
        obj = os.path.join(BUILD_DIR, src.replace(".cu", "_checked.o" if checked else ".o"))
        flags = ["-DDOMAGG_CHECKED"] if checked else []
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose_ptxas and not checked:
            print(r.stderr)
        return obj

    jobs = [(src, checked) for checked in (False, True) for src in SOURCES]
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for lib, these in ((LIB, objs[:len(SOURCES)]), (LIB_CHECKED, objs[len(SOURCES):])):
        tmp = f"{lib}.{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *these]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
