"""Build the CUDA library in-tree: paper_1805_10904_gb300/lib/libgb300louvain.so.

Each translation unit is compiled for sm_103a in parallel, then linked with nvcc.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libgb300louvain.so")
SOURCES = ["k_move.cu", "k_move_batch.cu", "k_move_first.cu", "k_coarsen.cu", "k_level.cu",
           "engine.cu", "noalloc.cu", "k_edges.cu"]
HEADERS = ["lv_common.cuh", "lv_scan.cuh", "lv_kernels.h", "k_move_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fno-strict-aliasing"]


def _nvcc() -> str:
    for c in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.isabs(c) and os.path.exists(c):
            return c
    return "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(HERE, "..", "include", "louvain.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(LIBDIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, s):
            cmd = [nvcc] + NVCC_FLAGS + ["-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((o, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                              stderr=subprocess.STDOUT)))
    failed = []
    for o, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((o, out.decode(errors="replace")))
        else:
            os.replace(o + ".tmp", o)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"{o}:\n{t}" for o, t in failed))
    if force or procs or not os.path.exists(LIB) or any(
            os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
