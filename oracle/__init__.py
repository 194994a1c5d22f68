"""CPU oracle of synchronous parallel Louvain (arXiv 1805.10904) -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library:
the arithmetic lives in ``louvain_oracle.c`` (plain sequential C, int64 sums and
int128 products), and this module only compiles it and marshals arrays.

Parity status of each exported function (what pins it to the paper, in tests/):
  modularity      -- pinned: networkx modularity, disjoint-clique closed form,
                     singleton closed form, brute-force matrix form.
  gain            -- pinned: equals half the Eq. 3 difference before/after the move.
  sweep           -- pinned: hand-worked cases of Sec. 3.1 rules, brute-force
                     local-optimality check of the final state.
  vertex_following-- pinned: hand-worked star / isolated pair / path cases.
  renumber        -- pinned: order-preserving compaction checked against numpy.unique.
  coarsen         -- pinned: dense P^T A P (numpy matmul) on small graphs.
  louvain         -- pinned: Q <= brute-force optimum (n <= 12), planted cliques
                     recovered, Theorem 1 and TW / Q preservation across levels; the
                     outer stop of Algorithm 2 against exact fractions.
  color           -- pinned: proper colouring equal to the sequential greedy colouring
                     in decreasing priority order.
  louvain(coloring=True) -- pinned: with one vertex per colour class it is sequential
                     local moving (textbook Blondel gain with removal first); hand-worked
                     two-colour case; Q <= brute force; planted cliques; Theorem 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "louvain_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liblouvain_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/lib/liblouvain_oracle.so (gcc, -O2, no -march)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fno-strict-aliasing", "-fPIC", "-shared",
               "-Wall", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    lib.oracle_run.restype = P
    lib.oracle_run.argtypes = [i64, P, P, P, i64, i64, i32, i32, i32, i32, P]
    lib.oracle_run_ex.restype = P
    lib.oracle_run_ex.argtypes = [i64, P, P, P, i64, i64, i32, i32, i32, i32, i32, i32, i32, P]
    lib.oracle_color.restype = i32
    lib.oracle_color.argtypes = [i64, P, P, P]
    lib.oracle_res_num_levels.restype = i32
    lib.oracle_res_num_levels.argtypes = [P]
    lib.oracle_res_tw.restype = i64
    lib.oracle_res_tw.argtypes = [P]
    lib.oracle_res_edge_visits.restype = i64
    lib.oracle_res_edge_visits.argtypes = [P]
    lib.oracle_res_sweeps.restype = i64
    lib.oracle_res_sweeps.argtypes = [P]
    lib.oracle_res_hit_iter_cap.restype = i32
    lib.oracle_res_hit_iter_cap.argtypes = [P]
    lib.oracle_res_level.restype = None
    lib.oracle_res_level.argtypes = [P, i32, P, P, P, P, P, P, P, P]
    lib.oracle_res_trace_len.restype = i64
    lib.oracle_res_trace_len.argtypes = [P]
    lib.oracle_res_trace.restype = None
    lib.oracle_res_trace.argtypes = [P, P, P, P, P]
    lib.oracle_res_free.restype = None
    lib.oracle_res_free.argtypes = [P]
    lib.oracle_modularity.restype = i64
    lib.oracle_modularity.argtypes = [i64, P, P, P, P, P]
    lib.oracle_gain.restype = None
    lib.oracle_gain.argtypes = [i64, P, P, P, P, i64, i32, P]
    lib.oracle_sweep.restype = i64
    lib.oracle_sweep.argtypes = [i64, P, P, P, P, P]
    lib.oracle_vertex_following.restype = None
    lib.oracle_vertex_following.argtypes = [i64, P, P, P]
    lib.oracle_renumber.restype = i64
    lib.oracle_renumber.argtypes = [i64, P, P]
    lib.oracle_below_threshold.restype = i32
    lib.oracle_below_threshold.argtypes = [P, P, i64, i64, i64]
    lib.oracle_coarsen.restype = P
    lib.oracle_coarsen.argtypes = [i64, P, P, P, P]
    lib.oracle_graph_n.restype = i64
    lib.oracle_graph_n.argtypes = [P]
    lib.oracle_graph_nnz.restype = i64
    lib.oracle_graph_nnz.argtypes = [P]
    lib.oracle_graph_copy.restype = None
    lib.oracle_graph_copy.argtypes = [P, P, P, P]
    lib.oracle_graph_free.restype = None
    lib.oracle_graph_free.argtypes = [P]
    _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _i128(limbs) -> int:
    hi, lo = int(limbs[0]), int(limbs[1])
    return (hi << 64) | (lo & 0xFFFFFFFFFFFFFFFF)


def _limbs(v: int) -> np.ndarray:
    return np.array([v >> 64, ((v & 0xFFFFFFFFFFFFFFFF) ^ (1 << 63)) - (1 << 63)], dtype=np.int64)


def _csr(rp, col, w=None, wdtype=np.int64):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=wdtype)
    return rp, col, w


class OracleError(RuntimeError):
    pass


@dataclass
class OracleLevel:
    labels: np.ndarray   # int32[n0], community of each original vertex after this level
    ncomm: int
    qn: int              # exact (2W)^2 * Q
    qn_init: int         # Qn of the level's state before its first sweep
    q: float             # (double)Qn / (double)TW^2
    iters: int
    n: int               # vertices of the graph this level ran on
    nnz: int             # stored entries of that graph


@dataclass
class OracleResult:
    tw: int
    levels: List[OracleLevel]
    trace: List[tuple] = field(default_factory=list)  # (level, iter, moved, qn)
    edge_visits: int = 0
    sweeps: int = 0
    hit_iter_cap: bool = False


def louvain(rp, col, w=None, theta=(1, 1_000_000), max_iters=1000, max_levels=64,
            vertex_following=True, vf_all_levels=False, threshold_mode=0,
            post_merge=False, coloring=False) -> OracleResult:
    """Full multi-level synchronous Louvain (Algorithm 2 around Algorithm 1).
    threshold_mode 0: absolute phase test; 1: the relative test printed in Algorithm 1.
    post_merge: the post-phase merge of single-neighbour-community vertices (Sec. 5.1.2).
    coloring: sweeps take the colour classes of a distance-1 colouring one after the other
    (Lu et al.'s colouring heuristic, reading R17)."""
    lib = _load()
    rp, col, w = _csr(rp, col, w, np.int32)
    n = len(rp) - 1
    st = ctypes.c_int32(0)
    h = lib.oracle_run_ex(n, _ptr(rp), _ptr(col), _ptr(w), int(theta[0]), int(theta[1]),
                          int(max_iters), int(max_levels), int(bool(vertex_following)),
                          int(bool(vf_all_levels)), int(threshold_mode), int(bool(post_merge)),
                          int(bool(coloring)), ctypes.addressof(st))
    if not h:
        raise OracleError(f"oracle_run failed with status {st.value}")
    try:
        L = lib.oracle_res_num_levels(h)
        levels = []
        for l in range(L):
            lab = np.empty(n, dtype=np.int32)
            nc = ctypes.c_int64()
            qn = np.zeros(2, np.int64)
            qi = np.zeros(2, np.int64)
            it = ctypes.c_int32()
            nl = ctypes.c_int64()
            ml = ctypes.c_int64()
            q = ctypes.c_double()
            lib.oracle_res_level(h, l, _ptr(lab), ctypes.addressof(nc), _ptr(qn), _ptr(qi),
                                 ctypes.addressof(it), ctypes.addressof(nl), ctypes.addressof(ml),
                                 ctypes.addressof(q))
            levels.append(OracleLevel(lab, nc.value, _i128(qn), _i128(qi), q.value, it.value,
                                      nl.value, ml.value))
        T = lib.oracle_res_trace_len(h)
        tl = np.empty(T, np.int32)
        ti = np.empty(T, np.int32)
        tm = np.empty(T, np.int64)
        tq = np.empty(2 * T, np.int64)
        if T:
            lib.oracle_res_trace(h, _ptr(tl), _ptr(ti), _ptr(tm), _ptr(tq))
        trace = [(int(tl[t]), int(ti[t]), int(tm[t]), _i128(tq[2 * t:2 * t + 2])) for t in range(T)]
        return OracleResult(lib.oracle_res_tw(h), levels, trace, lib.oracle_res_edge_visits(h),
                            lib.oracle_res_sweeps(h), bool(lib.oracle_res_hit_iter_cap(h)))
    finally:
        lib.oracle_res_free(h)


def color(rp, col):
    """Distance-1 colouring of reading R17: (colour of every vertex, number of colours)."""
    lib = _load()
    rp, col, _ = _csr(rp, col)
    out = np.empty(len(rp) - 1, np.int32)
    k = lib.oracle_color(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(out))
    if k < 0:
        raise OracleError("bad input")
    return out, int(k)


def modularity(rp, col, w, C):
    """Eq. 3 times TW^2 for labels C: returns (Qn, TW) as exact Python ints."""
    lib = _load()
    rp, col, w = _csr(rp, col, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    out = np.zeros(2, np.int64)
    tw = lib.oracle_modularity(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(w), _ptr(C), _ptr(out))
    if tw < 0:
        raise OracleError("bad input")
    return _i128(out), tw


def gain(rp, col, w, C, i, b) -> int:
    """(2W)^2/2 times the Eq. 4 gain of moving vertex i into community b: G_b - G_stay."""
    lib = _load()
    rp, col, w = _csr(rp, col, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    out = np.zeros(2, np.int64)
    lib.oracle_gain(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(w), _ptr(C), int(i), int(b), _ptr(out))
    return _i128(out)


def sweep(rp, col, w, C):
    """One synchronous local-moving sweep from state C: returns (C_next, moved)."""
    lib = _load()
    rp, col, w = _csr(rp, col, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    Cn = np.empty_like(C)
    moved = lib.oracle_sweep(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(w), _ptr(C), _ptr(Cn))
    if moved < 0:
        raise OracleError("bad input")
    return Cn, int(moved)


def vertex_following(rp, col):
    lib = _load()
    rp, col, _ = _csr(rp, col)
    C = np.empty(len(rp) - 1, np.int32)
    lib.oracle_vertex_following(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(C))
    return C


def renumber(C):
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.int32)
    new_id = np.empty_like(C)
    k = lib.oracle_renumber(len(C), _ptr(C), _ptr(new_id))
    return new_id, int(k)


def below_threshold(qn_new: int, qn_old: int, tw: int, num: int, den: int) -> bool:
    lib = _load()
    a, b = _limbs(qn_new), _limbs(qn_old)
    return bool(lib.oracle_below_threshold(_ptr(a), _ptr(b), int(tw), int(num), int(den)))


def coarsen(rp, col, w, C):
    """Induced graph of partition C (Sec. 5.1.2): returns (rp', col', w') with sorted rows."""
    lib = _load()
    rp, col, w = _csr(rp, col, w)
    C = np.ascontiguousarray(C, dtype=np.int32)
    h = lib.oracle_coarsen(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(w), _ptr(C))
    if not h:
        raise OracleError("bad input")
    try:
        n = lib.oracle_graph_n(h)
        m = lib.oracle_graph_nnz(h)
        rp2 = np.empty(n + 1, np.int64)
        col2 = np.empty(max(m, 1), np.int32)
        w2 = np.empty(max(m, 1), np.int64)
        lib.oracle_graph_copy(h, _ptr(rp2), _ptr(col2), _ptr(w2))
        return rp2, col2[:m].copy(), w2[:m].copy()
    finally:
        lib.oracle_graph_free(h)
