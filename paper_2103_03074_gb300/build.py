"""Build libtn.so in place: CUDA sources with nvcc for sm_103a, host C++ with
g++, linked against the shared CUDA runtime.  Object files go to _build/.
Each product is rebuilt unless a digest of its inputs (source and header
bytes, command line, machine) matches the one stored beside it, so objects
or a library made from other sources, flags or on another machine are never
reused."""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libtn.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels.cu", "tc_gemm.cu", "noalloc.cu", "costmodel.cu", "postselect.cu"]
CPP_SOURCES = ["plan.cpp", "network.cpp", "order.cpp", "api_host.cpp", "headtail.cpp"]


def _headers():
    return sorted([os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")] +
                  [os.path.join(INCLUDE, "tn.h")])


def _digest(paths, cmd):
    """Content digest of the inputs of one build product: the files' bytes,
    the command line and the machine (an object built elsewhere never
    matches)."""
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update("\0".join(cmd).encode())
    for p in paths:
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _up_to_date(out, digest):
    stamp = out + ".digest"
    if not os.path.exists(out) or not os.path.exists(stamp):
        return False
    with open(stamp) as f:
        return f.read().strip() == digest


def _stamp(out, digest):
    with open(out + ".digest", "w") as f:
        f.write(digest + "\n")


def _compile(src: str, verbose_ptxas: bool) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    if src.endswith(".cu"):
        cmd = [NVCC] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", path, "-o", obj] + inc
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", path, "-o", obj,
               "-I" + os.path.join(CUDA_HOME, "include")] + inc
    digest = _digest([path] + _headers(), cmd)
    if _up_to_date(obj, digest) and not verbose_ptxas:
        return obj
    if verbose_ptxas and src.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    _stamp(obj, digest)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            if f.endswith(".o"):
                os.remove(os.path.join(BUILD, f))
    srcs = CU_SOURCES + CPP_SOURCES
    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs + ["-lpthread"]
    digest = _digest(objs, cmd)
    if not _up_to_date(LIB, digest):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        _stamp(LIB, digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
