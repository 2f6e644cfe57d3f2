"""Builds liblbch.so in-tree with nvcc for sm_103a (GB300): one object per translation
unit, compiled in parallel, then linked."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblbch.so")
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, "lbch_api.cu"), os.path.join(CSRC, "lbnop.cu")]
DEPENDS = SOURCES + [os.path.join(CSRC, n) for n in
                     ("lbch_step.cuh", "lbch_aux.cuh", "lbch_lattice.cuh", "lbch_f2.cuh", "lbch_batch.cuh", "lbch3.cuh", "lbnop_tc.cuh")] + [
    os.path.join(ROOT, "include", n) for n in ("lbch.h", "lbch3.h", "lbnop.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPENDS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the library if it is missing or older than its sources; returns its path."""
    if not force and not stale():
        return LIB
    tag = f".tmp{os.getpid()}"
    objs = [os.path.splitext(src)[0] + tag + ".o" for src in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)

    try:
        with ThreadPoolExecutor(len(SOURCES)) as ex:
            list(ex.map(compile_one, zip(SOURCES, objs)))
        tmp = LIB + tag
        subprocess.run([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", *objs, "-o", tmp],
                       check=True)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
