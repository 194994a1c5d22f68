"""Multi-threaded CPU synchronous Louvain (OpenMP) -- a CPU baseline.

The paper compares its GPU code with an 8-thread CPU parallel Louvain (Sec. 6).  This
package is this project's own parallel CPU form of the same synchronous method that the
CUDA library runs (same readings, exact integer arithmetic), timed beside the GPU and the
single-threaded oracle; its results equal the oracle's for every thread count.  It is a
baseline, not a fallback: the CUDA library never calls it.  It shares no code with the
CUDA library or with the oracle; ``louvain_omp.c`` holds the arithmetic, this module only
compiles it and marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "louvain_omp.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liblouvain_omp.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile louvain_omp.c into cpu_omp/lib/liblouvain_omp.so (gcc -O2 -fopenmp)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.lomp_run.restype = P
        lib.lomp_run.argtypes = [i64, P, P, P, i64, i64, i32, i32, i32, i32, i32, P]
        lib.lomp_free.argtypes = [P]
        lib.lomp_free.restype = None
        for name, rt in (("lomp_num_levels", i32), ("lomp_tw", i64), ("lomp_edge_visits", i64),
                         ("lomp_sweeps", i64), ("lomp_hit_cap", i32), ("lomp_trace_len", i64)):
            getattr(lib, name).restype = rt
            getattr(lib, name).argtypes = [P]
        lib.lomp_max_threads.restype = i32
        lib.lomp_max_threads.argtypes = []
        lib.lomp_level.restype = None
        lib.lomp_level.argtypes = [P, i32, P, P, P, P, P, P, P]
        lib.lomp_trace.restype = None
        lib.lomp_trace.argtypes = [P, P, P, P, P]
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().lomp_max_threads())


def _i128(hi, lo) -> int:
    return (int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)


@dataclass
class Level:
    labels: np.ndarray
    ncomm: int
    qn: int
    qn_init: int
    iters: int
    n: int
    nnz: int


@dataclass
class Result:
    tw: int
    levels: List[Level]
    trace: List[tuple] = field(default_factory=list)
    edge_visits: int = 0
    sweeps: int = 0
    hit_iter_cap: bool = False


def louvain(rp, col, w=None, threads: int = 0, theta=(1, 1_000_000), max_iters: int = 1000,
            max_levels: int = 64, vertex_following: bool = True,
            vf_all_levels: bool = False) -> Result:
    """Full multi-level synchronous Louvain with `threads` OpenMP threads (0: default).
    Rows must list each column once, in increasing order."""
    lib = _load()
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
    n = len(rp) - 1
    st = ctypes.c_int32(0)
    h = lib.lomp_run(n, rp.ctypes.data, col.ctypes.data, None if w is None else w.ctypes.data,
                     int(theta[0]), int(theta[1]), int(max_iters), int(max_levels),
                     int(bool(vertex_following)), int(bool(vf_all_levels)), int(threads),
                     ctypes.addressof(st))
    if not h:
        raise RuntimeError(f"lomp_run failed with status {st.value}")
    try:
        levels = []
        for l in range(lib.lomp_num_levels(h)):
            lab = np.empty(n, np.int32)
            nc, it, nl, ml = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
            qn, qi = np.zeros(2, np.int64), np.zeros(2, np.int64)
            lib.lomp_level(h, l, lab.ctypes.data, ctypes.addressof(nc), qn.ctypes.data,
                           qi.ctypes.data, ctypes.addressof(it), ctypes.addressof(nl),
                           ctypes.addressof(ml))
            levels.append(Level(lab, nc.value, _i128(*qn), _i128(*qi), it.value, nl.value,
                                ml.value))
        T = lib.lomp_trace_len(h)
        tl, ti = np.empty(T, np.int32), np.empty(T, np.int32)
        tm, tq = np.empty(T, np.int64), np.empty(2 * T, np.int64)
        if T:
            lib.lomp_trace(h, tl.ctypes.data, ti.ctypes.data, tm.ctypes.data, tq.ctypes.data)
        trace = [(int(tl[t]), int(ti[t]), int(tm[t]), _i128(tq[2 * t], tq[2 * t + 1]))
                 for t in range(T)]
        return Result(lib.lomp_tw(h), levels, trace, lib.lomp_edge_visits(h),
                      lib.lomp_sweeps(h), bool(lib.lomp_hit_cap(h)))
    finally:
        lib.lomp_free(h)
