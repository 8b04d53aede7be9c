"""Build libemg.so in-tree with nvcc for sm_103a (translation units compiled in parallel)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libemg.so")
# host build of the per-cell adjoint functions, for CPU checks against the oracle (tests only)
HOSTCHECK = os.path.join(PKG, "libemg_hostcheck.so")
SOURCES = ["emg.cu", "launch2d.cu", "launch3d.cu", "noalloc.cu", "adjoint.cu", "kaczmarz.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "--diag-suppress=177"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "emg.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


def build_hostcheck(force: bool = False) -> str:
    """libemg_hostcheck.so: csrc/hostcheck.cu compiled for the host only (the adjoint's per-cell
    functions looped on the CPU), which the CPU tests compare with the FP64 oracle."""
    src = os.path.join(CSRC, "hostcheck.cu")
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [src]
    if not force and os.path.exists(HOSTCHECK) and all(os.path.getmtime(d) <= os.path.getmtime(HOSTCHECK) for d in deps):
        return HOSTCHECK
    tmp = HOSTCHECK + ".tmp"
    cmd = [nvcc()] + ARCH + ["-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                             src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for hostcheck.cu:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, HOSTCHECK)
    return HOSTCHECK


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
    print(build_hostcheck(force="--force" in sys.argv))
