"""Build libwl.so (the CUDA sm_103a library behind include/wl.h) in-tree.

    python -m paper_2407_16032_b300.build [--force] [--verbose]

Each translation unit of csrc/ compiles to an object in _build/ (in parallel),
then nvcc links the shared library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwl.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", os.path.join(ROOT, "include")]


def units():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(ROOT, "include", "wl.h")])


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in sources())


def _compile(src: str, verbose: bool):
    obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC, *FLAGS, *(["-Xptxas=-v"] if verbose else []), "-c", "-o", obj + ".tmp", src]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    srcs = units()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), srcs))
    failed = [(s, r) for s, _, r in results if r.returncode != 0]
    for s, r in failed:
        sys.stderr.write(f"--- {os.path.basename(s)}\n" + r.stdout + r.stderr)
    if failed:
        raise RuntimeError("nvcc failed building libwl.so")
    objs = []
    for s, obj, r in results:
        if verbose:
            sys.stderr.write(f"--- {os.path.basename(s)}\n" + r.stderr)
        os.replace(obj + ".tmp", obj)
        objs.append(obj)
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", LIB + ".tmp", *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libwl.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
