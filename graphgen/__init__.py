"""Seeded synthetic graph generators (input data only).

Serves both the CPU oracle and the CUDA library with identical inputs and holds
none of the community-detection arithmetic.  Large models (R-MAT, planted
partition, Chung-Lu) are compiled C (``graphgen.c``, counter-based SplitMix64
draws, OpenMP when available); the small structured graphs used by the tests are
built here with numpy.

Every graph is returned as ``Graph(rp, col, w)``: symmetric CSR, int64 row
offsets, int32 column ids, int32 weights >= 1.  Rows are sorted by column and
hold no duplicates.  Loops appear only where a builder adds them on purpose.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into graphgen/lib/libgraphgen.so (OpenMP if gcc supports it)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:4] + ["-fopenmp"] + base[4:], capture_output=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, i64, i32, u64, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                 ctypes.c_uint64, ctypes.c_double)
        lib.gg_rmat.restype = P
        lib.gg_rmat.argtypes = [i32, i32, f64, f64, f64, i32, i32, u64]
        lib.gg_sbm.restype = P
        lib.gg_sbm.argtypes = [i64, i64, f64, f64, i32, i32, u64, i64]
        lib.gg_chung_lu.restype = P
        lib.gg_chung_lu.argtypes = [i64, f64, f64, i32, i32, u64]
        lib.gg_from_pairs.restype = P
        lib.gg_from_pairs.argtypes = [i64, i64, P, P, i32, i32, u64]
        lib.gg_graph_n.restype = i64
        lib.gg_graph_n.argtypes = [P]
        lib.gg_graph_nnz.restype = i64
        lib.gg_graph_nnz.argtypes = [P]
        lib.gg_graph_copy.restype = None
        lib.gg_graph_copy.argtypes = [P, P, P, P]
        lib.gg_graph_free.restype = None
        lib.gg_graph_free.argtypes = [P]
        lib.gg_mix64.restype = u64
        lib.gg_mix64.argtypes = [u64]
        lib.gg_cb64.restype = u64
        lib.gg_cb64.argtypes = [u64, u64]
        lib.gg_stream_key.restype = u64
        lib.gg_stream_key.argtypes = [u64, u64]
        lib.gg_openmp_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Graph:
    rp: np.ndarray   # int64[n + 1]
    col: np.ndarray  # int32[nnz]
    w: np.ndarray    # int32[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return len(self.rp) - 1

    @property
    def nnz(self) -> int:
        return int(self.rp[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rp)


def _take(h, name) -> Graph:
    lib = _load()
    if not h:
        raise ValueError(f"generator {name} rejected its arguments or ran out of memory")
    try:
        n = lib.gg_graph_n(h)
        m = lib.gg_graph_nnz(h)
        rp = np.empty(n + 1, np.int64)
        col = np.empty(max(m, 1), np.int32)
        w = np.empty(max(m, 1), np.int32)
        lib.gg_graph_copy(h, rp.ctypes.data, col.ctypes.data, w.ctypes.data)
        return Graph(rp, col[:m], w[:m], name)
    finally:
        lib.gg_graph_free(h)


def mix64(z: int) -> int:
    return int(_load().gg_mix64(z & 0xFFFFFFFFFFFFFFFF))


def graph_seed(base: int, k: int) -> int:
    """Seed of graph k in a seeded family: SplitMix64 counter draw (base, k)."""
    lib = _load()
    return int(lib.gg_cb64(lib.gg_stream_key(base, 0), k))


def openmp_threads() -> int:
    return int(_load().gg_openmp_threads())


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         wmin: int = 1, wmax: int = 16, seed: int = 22) -> Graph:
    h = _load().gg_rmat(scale, edge_factor, a, b, c, wmin, wmax, seed)
    return _take(h, f"rmat{scale}")


def sbm(n: int, block_size: int, p_in: float, p_out: float, wmin: int = 1, wmax: int = 4,
        seed: int = 1, exact_limit: int = 32768) -> Graph:
    h = _load().gg_sbm(n, block_size, p_in, p_out, wmin, wmax, seed, exact_limit)
    return _take(h, f"sbm{n}")


def chung_lu(n: int, gamma: float = 2.1, avg_deg: float = 10.0, wmin: int = 1, wmax: int = 8,
             seed: int = 3) -> Graph:
    h = _load().gg_chung_lu(n, gamma, avg_deg, wmin, wmax, seed)
    return _take(h, f"chunglu{n}")


def batch_mix_params(num_graphs: int, seed: int = 512, n_min: int = 1000,
                     n_max: int = 200_000):
    """Parameters of the mixed batch workload: graph k has a log-uniform size in
    [n_min, n_max]; even k are planted partitions (block size log-uniform in [32, 512],
    average degree uniform in [8, 40], 80% of it inside the block), odd k Chung-Lu
    power-law graphs (exponent 2.1, average degree 10); weights uniform in [1, 8].
    Every draw comes from the counter-based stream of graph_seed(seed, k)."""
    out = []
    for k in range(num_graphs):
        gs = graph_seed(seed, k)
        rng = np.random.Generator(np.random.PCG64(gs))
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        if k % 2 == 0:
            b = int(round(np.exp(rng.uniform(np.log(32), np.log(512)))))
            b = max(2, min(b, n))
            d = float(rng.uniform(8.0, 40.0))
            p_in = min(1.0, 0.8 * d / max(b - 1, 1))
            p_out = 0.2 * d / max(n - b, 1)
            out.append(("sbm", n, b, p_in, p_out, gs))
        else:
            out.append(("chung_lu", n, 2.1, 10.0, gs))
    return out


def batch_mix_graph(params) -> Graph:
    if params[0] == "sbm":
        _, n, b, p_in, p_out, gs = params
        return sbm(n, b, p_in, p_out, 1, 8, gs)
    _, n, gamma, avg, gs = params
    return chung_lu(n, gamma, avg, 1, 8, gs)


def batch_mix(num_graphs: int, seed: int = 512, n_min: int = 1000,
              n_max: int = 200_000):
    """The graphs of batch_mix_params (see there)."""
    return [batch_mix_graph(p) for p in batch_mix_params(num_graphs, seed, n_min, n_max)]


def from_pairs(n: int, pairs: Iterable[Tuple[int, int]], wmin: int = 1, wmax: int = 1,
               seed: int = 0) -> Graph:
    p = np.asarray(list(pairs), dtype=np.int32).reshape(-1, 2)
    pu = np.ascontiguousarray(p[:, 0])
    pv = np.ascontiguousarray(p[:, 1])
    h = _load().gg_from_pairs(n, len(pu), pu.ctypes.data, pv.ctypes.data, wmin, wmax, seed)
    return _take(h, "pairs")


# --------------------------------------------------------------------------
# Small structured graphs (numpy), optionally with explicit weights and loops.
# --------------------------------------------------------------------------

def from_edges(n: int, edges: Sequence[Tuple[int, int, int]], name: str = "") -> Graph:
    """Symmetric CSR from explicit undirected (u, v, w) triples; (u, u, w) is a loop
    stored once.  Duplicate pairs are rejected."""
    rows = [dict() for _ in range(n)]
    for u, v, wt in edges:
        if not (0 <= u < n and 0 <= v < n):
            raise ValueError("vertex out of range")
        if v in rows[u]:
            raise ValueError("duplicate edge")
        rows[u][v] = wt
        if u != v:
            rows[v][u] = wt
    rp = np.zeros(n + 1, np.int64)
    cols, ws = [], []
    for i in range(n):
        ks = sorted(rows[i])
        cols.extend(ks)
        ws.extend(rows[i][k] for k in ks)
        rp[i + 1] = rp[i] + len(ks)
    return Graph(rp, np.asarray(cols, np.int32), np.asarray(ws, np.int32), name)


def erdos_renyi(n: int, p: float, seed: int, wmax: int = 1, loops: float = 0.0) -> Graph:
    rng = np.random.default_rng(seed)
    edges = []
    for i in range(n):
        if loops > 0 and rng.random() < loops:
            edges.append((i, i, int(rng.integers(1, wmax + 1))))
        for j in range(i + 1, n):
            if rng.random() < p:
                edges.append((i, j, int(rng.integers(1, wmax + 1))))
    return from_edges(n, edges, f"er{n}")


def cliques_ring(k: int, m: int, w_in: int = 1, w_bridge: int = 1) -> Graph:
    """k cliques of m vertices, clique c's last vertex joined to clique c+1's first."""
    n = k * m
    edges = []
    for c in range(k):
        base = c * m
        for i in range(m):
            for j in range(i + 1, m):
                edges.append((base + i, base + j, w_in))
        if k > 1 and (k > 2 or c == 0):
            edges.append((base + m - 1, ((c + 1) % k) * m, w_bridge))
    return from_edges(n, edges, f"cliques{k}x{m}")


def disjoint_cliques(k: int, m: int, w: int = 1) -> Graph:
    edges = []
    for c in range(k):
        for i in range(m):
            for j in range(i + 1, m):
                edges.append((c * m + i, c * m + j, w))
    return from_edges(k * m, edges, f"disjoint{k}x{m}")


def star(leaves: int, w: int = 1) -> Graph:
    return from_edges(leaves + 1, [(0, i, w) for i in range(1, leaves + 1)], f"star{leaves}")


def path(n: int, w: int = 1) -> Graph:
    return from_edges(n, [(i, i + 1, w) for i in range(n - 1)], f"path{n}")


def random_small(seed: int, n_max: int = 40, wmax: int = 9) -> Graph:
    """A random small graph of a random family (for fuzzing parity)."""
    rng = np.random.default_rng(seed)
    kind = int(rng.integers(0, 6))
    n = int(rng.integers(1, n_max + 1))
    if kind == 0:
        return erdos_renyi(n, float(rng.uniform(0.02, 0.5)), seed, wmax, loops=0.1)
    if kind == 1:
        bs = int(rng.integers(2, 9))
        return sbm(max(n, 2), bs, float(rng.uniform(0.3, 1.0)), float(rng.uniform(0.0, 0.1)),
                   1, wmax, seed)
    if kind == 2:
        return star(max(1, n - 1), int(rng.integers(1, wmax + 1)))
    if kind == 3:
        return path(n, int(rng.integers(1, wmax + 1)))
    if kind == 4:
        k = int(rng.integers(1, 5))
        m = int(rng.integers(2, 7))
        return cliques_ring(k, m, int(rng.integers(1, wmax + 1)), 1)
    # several disconnected random parts plus isolated vertices
    parts = []
    off = 0
    edges = []
    for _ in range(int(rng.integers(1, 4))):
        m = int(rng.integers(1, 10))
        g = erdos_renyi(m, 0.4, int(rng.integers(1 << 30)), wmax, loops=0.2)
        for i in range(m):
            for t in range(g.rp[i], g.rp[i + 1]):
                j = int(g.col[t])
                if j >= i:
                    edges.append((off + i, off + j, int(g.w[t])))
        off += m
        parts.append(m)
    off += int(rng.integers(0, 4))
    return from_edges(off, edges, "parts")


def check_csr(g: Graph) -> None:
    """Structural checks of the generator contract (raise AssertionError)."""
    n = g.n
    assert g.rp[0] == 0 and np.all(np.diff(g.rp) >= 0)
    assert g.col.dtype == np.int32 and g.w.dtype == np.int32
    assert len(g.col) == g.nnz == len(g.w)
    if g.nnz == 0:
        return
    assert g.col.min() >= 0 and g.col.max() < n
    assert g.w.min() >= 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rp))
    key = rows * n + g.col.astype(np.int64)
    assert np.all(np.diff(key) > 0), "rows must be sorted and duplicate-free"
    tkey = g.col.astype(np.int64) * n + rows
    order = np.argsort(tkey)
    assert np.array_equal(tkey[order], key), "adjacency must be symmetric"
    assert np.array_equal(g.w[order], g.w), "weights must be symmetric"
