"""Thin ctypes binding of the C ABI in include/louvain.h (argument marshalling only).

Every step of community detection runs in the CUDA library; this module passes
pointers, sizes and the current torch stream, and lets the library allocate device
memory through PyTorch's caching allocator.  If the library has not been built the
import of the binding succeeds but every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgb300louvain.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_NOT_SYMMETRIC = 2
ERR_DUPLICATE_EDGE = 3
ERR_BAD_WEIGHT = 4
ERR_INDEX_RANGE = 5
ERR_OOM = 6
ERR_CUDA = 7
ERR_TIMEOUT = 8
ERR_INTERNAL = 9
PENDING = 10
ERR_REJECTED = 11
ERR_TOO_LARGE = 12
PTR_HOST = 0
PTR_DEVICE = 1

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("theta_num", ctypes.c_int64),
        ("theta_den", ctypes.c_int64),
        ("max_iters", ctypes.c_int32),
        ("max_levels", ctypes.c_int32),
        ("vertex_following", ctypes.c_int32),
        ("vf_all_levels", ctypes.c_int32),
        ("checks", ctypes.c_int32),
        ("force_int128", ctypes.c_int32),
        ("wide_sums", ctypes.c_int32),
        ("bin_small", ctypes.c_int32),
        ("bin_mid1", ctypes.c_int32),
        ("bin_mid2", ctypes.c_int32),
        ("bin_cta1", ctypes.c_int32),
        ("bin_cta2", ctypes.c_int32),
        ("bin_cta3", ctypes.c_int32),
        ("chunk_entries", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("cuda_graphs", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("threshold_mode", ctypes.c_int32),
        ("post_merge", ctypes.c_int32),
        ("keep_coarse", ctypes.c_int32),
        ("sweep_streams", ctypes.c_int32),
        ("part_keys", ctypes.c_int32),
        ("coloring", ctypes.c_int32),
        ("host_labels", ctypes.c_int32),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class LouvainError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"louvain error {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load the CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing at {LIB_PATH}: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.louvain_abi_version.restype = ctypes.c_int
    lib.louvain_config_init.argtypes = [ctypes.POINTER(Config)]
    lib.louvain_create.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(P)]
    lib.louvain_destroy.argtypes = [P]
    lib.louvain_destroy.restype = None
    lib.louvain_last_error.argtypes = [P]
    lib.louvain_last_error.restype = ctypes.c_char_p
    lib.louvain_run.argtypes = [P, i64, P, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
    lib.louvain_run_batch.argtypes = [P, i32, P, P, P, P, P, ctypes.c_int, P, P]
    lib.louvain_serve_open.argtypes = [P, ctypes.c_uint64, ctypes.c_int]
    lib.louvain_submit.argtypes = [P, i64, P, P, P, ctypes.c_int, P]
    lib.louvain_poll.argtypes = [P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(P)]
    lib.louvain_serve_status.argtypes = [P, P]
    lib.louvain_serve_close.argtypes = [P]
    lib.louvain_result_num_levels.argtypes = [P]
    lib.louvain_result_num_vertices.argtypes = [P]
    lib.louvain_result_num_vertices.restype = i64
    lib.louvain_result_labels.argtypes = [P, ctypes.c_int, ctypes.POINTER(P), P]
    lib.louvain_result_labels_device.argtypes = [P, ctypes.c_int, ctypes.POINTER(P)]
    lib.louvain_result_labels_into.argtypes = [P, ctypes.c_int, P]
    lib.louvain_result_modularity.argtypes = [P, ctypes.c_int, P, P, P, P]
    lib.louvain_result_level_info.argtypes = [P, ctypes.c_int, P, P, P, P, P]
    lib.louvain_result_trace.argtypes = [P, P, P, P, P, P]
    lib.louvain_result_counters.argtypes = [P, P, P]
    lib.louvain_num_bins.restype = ctypes.c_int
    lib.louvain_result_exec_info.argtypes = [P, P]
    lib.louvain_autotune.argtypes = [P, i64, P, P, P, ctypes.c_int, P, P, P, P]
    lib.louvain_csr_from_edges.argtypes = [P, i64, i64, P, P, P, ctypes.c_int, P, P, P, P, P]
    lib.louvain_result_coarse_graph.argtypes = [P, ctypes.c_int, P, P, P]
    lib.louvain_result_coarse_copy.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_int]
    lib.louvain_resume.argtypes = [P, i32, P, i64, P, P, P, i32, ctypes.c_int, P,
                                   ctypes.POINTER(P)]
    lib.louvain_result_bin_stats.argtypes = [P, ctypes.c_int, P, P, P, P, P]
    lib.louvain_result_coarsen_stats.argtypes = [P, P, P, P]
    lib.louvain_result_free.argtypes = [P]
    lib.louvain_result_free.restype = None
    _lib = lib
    return lib


def _i128(hi, lo) -> int:
    return (int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)


def _ptr_of(a):
    """(pointer, kind, keepalive) of a torch tensor or numpy array."""
    if a is None:
        return None, None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                a = a.contiguous()
            return a.data_ptr(), (PTR_DEVICE if a.is_cuda else PTR_HOST), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a)
    return a.ctypes.data, PTR_HOST, a


@dataclass
class Level:
    ncomm: int
    q: float
    qn: int
    qn_init: int
    iters: int
    n: int
    nnz: int
    hit_iter_cap: bool


class Result:
    """Owns a louvain_result*; labels are copied to the host on first access."""

    def __init__(self, lib, ptr, owner=None):
        self._lib = lib
        self._p = ptr
        # the handle owns the allocator callbacks that free this result's device memory
        self._owner = owner

    def close(self):
        if self._p:
            self._lib.louvain_result_free(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self) -> int:
        return self._lib.louvain_result_num_levels(self._p)

    @property
    def n(self) -> int:
        return self._lib.louvain_result_num_vertices(self._p)

    def labels(self, level: int, copy: bool = True) -> np.ndarray:
        """Labels of the input vertices after `level`.  copy=True: a new array.  copy=False:
        a read-only view of the result's own host copy (made during the run when the handle
        has host_labels=True, else on this first access); the view keeps the result alive
        and is valid until close()."""
        if not copy:
            p = ctypes.c_void_p()
            rc = self._lib.louvain_result_labels(self._p, level, ctypes.byref(p), None)
            if rc != OK:
                raise LouvainError(rc, "louvain_result_labels")
            if self.n == 0:
                return np.empty(0, np.int32)
            buf = (ctypes.c_int32 * self.n).from_address(p.value)
            buf._owner = self  # the result outlives the view
            view = np.frombuffer(buf, dtype=np.int32)
            view.flags.writeable = False
            return view
        out = np.empty(self.n, np.int32)
        rc = self._lib.louvain_result_labels_into(self._p, level,
                                                  out.ctypes.data if self.n else None)
        if rc != OK:
            raise LouvainError(rc, "louvain_result_labels_into")
        return out

    def labels_device_ptr(self, level: int) -> int:
        p = ctypes.c_void_p()
        rc = self._lib.louvain_result_labels_device(self._p, level, ctypes.byref(p))
        if rc != OK:
            raise LouvainError(rc, "louvain_result_labels_device")
        return p.value or 0

    def level(self, level: int) -> Level:
        q = ctypes.c_double()
        qn = np.zeros(2, np.int64)
        qi = np.zeros(2, np.int64)
        tw = ctypes.c_int64()
        rc = self._lib.louvain_result_modularity(self._p, level, ctypes.addressof(q),
                                                 qn.ctypes.data, qi.ctypes.data,
                                                 ctypes.addressof(tw))
        if rc != OK:
            raise LouvainError(rc, "louvain_result_modularity")
        it = ctypes.c_int32()
        nl = ctypes.c_int64()
        ml = ctypes.c_int64()
        nc = ctypes.c_int64()
        cap = ctypes.c_int32()
        self._lib.louvain_result_level_info(self._p, level, ctypes.addressof(it),
                                            ctypes.addressof(nl), ctypes.addressof(ml),
                                            ctypes.addressof(nc), ctypes.addressof(cap))
        return Level(nc.value, q.value, _i128(*qn), _i128(*qi), it.value, nl.value, ml.value,
                     bool(cap.value))

    def levels(self) -> List[Level]:
        return [self.level(l) for l in range(self.num_levels)]

    @property
    def tw(self) -> int:
        tw = ctypes.c_int64()
        if self.num_levels == 0:
            return 0
        self._lib.louvain_result_modularity(self._p, 0, None, None, None, ctypes.addressof(tw))
        return tw.value

    def trace(self):
        ln = ctypes.c_int64()
        self._lib.louvain_result_trace(self._p, ctypes.addressof(ln), None, None, None, None)
        T = ln.value
        lv = np.zeros(T, np.int32)
        it = np.zeros(T, np.int32)
        mv = np.zeros(T, np.int64)
        qn = np.zeros(2 * T, np.int64)
        if T:
            self._lib.louvain_result_trace(self._p, None, lv.ctypes.data, it.ctypes.data,
                                           mv.ctypes.data, qn.ctypes.data)
        return [(int(lv[t]), int(it[t]), int(mv[t]), _i128(qn[2 * t], qn[2 * t + 1]))
                for t in range(T)]

    def bin_stats(self):
        """Per bin slot: dict(time_ms, launches, alg_bytes, rows, entries).  Slots
        0 .. num_bins - 1 cover every sweep but the first of each phase, slot num_bins + b
        bin b in the first sweep of each phase (entries scored without tables)."""
        out = []
        for b in range(2 * self._lib.louvain_num_bins()):
            t = ctypes.c_double()
            v = [ctypes.c_int64() for _ in range(4)]
            self._lib.louvain_result_bin_stats(self._p, b, ctypes.addressof(t),
                                               *[ctypes.addressof(x) for x in v])
            out.append({"time_ms": t.value, "launches": v[0].value, "alg_bytes": v[1].value,
                        "rows": v[2].value, "entries": v[3].value})
        return out

    def coarse_graph(self, level: int):
        """(row_ptr, col_idx, weights) numpy arrays of the graph induced after recorded level
        `level` (keep_coarse runs), or None when the run stopped there."""
        n, nnz, wb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        rc = self._lib.louvain_result_coarse_graph(self._p, level, ctypes.addressof(n),
                                                   ctypes.addressof(nnz), ctypes.addressof(wb))
        if rc != OK:
            return None
        rp = np.empty(n.value + 1, np.int64)
        col = np.empty(max(nnz.value, 1), np.int32)
        w = np.empty(max(nnz.value, 1), np.int32 if wb.value == 4 else np.int64)
        rc = self._lib.louvain_result_coarse_copy(self._p, level, rp.ctypes.data, col.ctypes.data,
                                                  w.ctypes.data, PTR_HOST)
        if rc != OK:
            raise LouvainError(rc, "louvain_result_coarse_copy")
        return rp, col[:nnz.value], w[:nnz.value]

    def coarsen_stats(self):
        """(coarse graphs built, their algorithmic bytes, induction device ms (profile
        runs only)) -- louvain_result_coarsen_stats."""
        k, b, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        rc = self._lib.louvain_result_coarsen_stats(self._p, ctypes.addressof(k),
                                                    ctypes.addressof(b), ctypes.addressof(t))
        if rc != OK:
            raise LouvainError(rc, "louvain_result_coarsen_stats")
        return k.value, b.value, t.value

    def exec_info(self):
        """(sweeps in CUDA graphs, host-loop sweeps, level steps, graph captures, autotuning
        trials of this call, 1 if the tuned bins came from the cache)."""
        v = np.zeros(6, np.int64)
        self._lib.louvain_result_exec_info(self._p, v.ctypes.data)
        return tuple(int(x) for x in v)

    def counters(self):
        c = np.zeros(8, np.int64)
        t = np.zeros(8, np.float64)
        self._lib.louvain_result_counters(self._p, c.ctypes.data, t.ctypes.data)
        return c, t


class Louvain:
    """A library handle bound to one CUDA device.

    torch_alloc=True routes the library's device allocations through PyTorch's
    caching allocator (so PyTorch owns device memory); otherwise the library uses
    stream-ordered cudaMallocAsync.
    """

    def __init__(self, device: int = 0, theta=(1, 1_000_000), max_iters: int = 1000,
                 max_levels: int = 64, vertex_following: bool = True,
                 vf_all_levels: bool = False, checks: int = 1, force_int128: bool = False,
                 wide_sums: bool = False, bins=None, chunk_entries: int = 0,
                 profile: bool = False, torch_alloc: bool = True, cuda_graphs: bool = True,
                 autotune: bool = False, threshold_mode: int = 0, post_merge: bool = False,
                 alloc_hook=None, keep_coarse: bool = False, sweep_streams: int = 4,
                 part_keys: int = 0, coloring: bool = False, host_labels: bool = False):
        lib = load()
        self._lib = lib
        cfg = Config()
        lib.louvain_config_init(ctypes.byref(cfg))
        cfg.theta_num, cfg.theta_den = int(theta[0]), int(theta[1])
        cfg.max_iters = max_iters
        cfg.max_levels = max_levels
        cfg.vertex_following = int(vertex_following)
        cfg.vf_all_levels = int(vf_all_levels)
        cfg.checks = checks
        cfg.force_int128 = int(force_int128)
        cfg.wide_sums = int(wide_sums)
        if bins is not None:  # (small, mid1, mid2, cta1, cta2, cta3)
            (cfg.bin_small, cfg.bin_mid1, cfg.bin_mid2, cfg.bin_cta1, cfg.bin_cta2,
             cfg.bin_cta3) = [int(x) for x in bins]
        if chunk_entries:
            cfg.chunk_entries = chunk_entries
        cfg.profile = int(profile)
        cfg.cuda_graphs = int(cuda_graphs)
        cfg.autotune = int(autotune)
        cfg.threshold_mode = int(threshold_mode)
        cfg.post_merge = int(post_merge)
        cfg.keep_coarse = int(keep_coarse)
        cfg.sweep_streams = int(sweep_streams)
        if part_keys:
            cfg.part_keys = int(part_keys)
        cfg.coloring = int(coloring)
        cfg.host_labels = int(host_labels)
        self.device = device
        # alloc_hook(bytes) -> bool may refuse an allocation (failure-injection tests)
        self.alloc_hook = alloc_hook
        if torch_alloc:
            import torch

            def _alloc(size, ctx, stream):
                hook = self.alloc_hook
                if hook is not None and not hook(int(size)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), device,
                                                              int(stream or 0))
                except Exception:
                    return None

            def _free(ptr, ctx, stream):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            cfg.alloc, cfg.free = self._cb
        self._cfg = cfg
        h = ctypes.c_void_p()
        rc = lib.louvain_create(ctypes.byref(cfg), device, ctypes.byref(h))
        if rc != OK:
            raise LouvainError(rc, "louvain_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.louvain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return (self._lib.louvain_last_error(self._h) or b"").decode()

    def run(self, row_ptr, col_idx, weights=None, stream: Optional[int] = None) -> Result:
        """Multi-level Louvain on a symmetric CSR (torch CUDA tensors: read in place;
        torch CPU tensors or numpy arrays: copied inside the call)."""
        rp, k1, keep1 = _ptr_of(row_ptr)
        col, k2, keep2 = _ptr_of(col_idx)
        w, k3, keep3 = _ptr_of(weights)
        kinds = {k for k in (k1, k2, k3) if k is not None}
        if len(kinds) != 1:
            raise ValueError("row_ptr, col_idx and weights must all be on the host or all on the device")
        n = int(keep1.shape[0]) - 1
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(self.device).cuda_stream
            except Exception:
                stream = 0
        out = ctypes.c_void_p()
        rc = self._lib.louvain_run(self._h, n, rp, col, w, kinds.pop(), ctypes.c_void_p(stream),
                                   ctypes.byref(out))
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return Result(self._lib, out, self)

    def autotune(self, row_ptr, col_idx, weights=None, stream: Optional[int] = None):
        """louvain_autotune: (bins 6-tuple, chunk_entries, best trial ms, trials)."""
        rp, k1, keep1 = _ptr_of(row_ptr)
        col, k2, keep2 = _ptr_of(col_idx)
        w, k3, keep3 = _ptr_of(weights)
        kinds = {k for k in (k1, k2, k3) if k is not None}
        if len(kinds) != 1:
            raise ValueError("row_ptr, col_idx and weights must all be on the host or all on the device")
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(self.device).cuda_stream
            except Exception:
                stream = 0
        b = np.zeros(7, np.int32)
        ms = ctypes.c_double()
        tr = ctypes.c_int32()
        rc = self._lib.louvain_autotune(self._h, int(keep1.shape[0]) - 1, rp, col, w,
                                        kinds.pop(), ctypes.c_void_p(stream), b.ctypes.data,
                                        ctypes.addressof(ms), ctypes.addressof(tr))
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return tuple(int(x) for x in b[:6]), int(b[6]), ms.value, tr.value

    def resume(self, start_level: int, qn_prev: int, row_ptr, col_idx, weights,
               stream: Optional[int] = None) -> Result:
        """louvain_resume from a saved level (weights int32 or int64 host arrays)."""
        rp = np.ascontiguousarray(np.asarray(row_ptr, np.int64))
        col = np.ascontiguousarray(np.asarray(col_idx, np.int32))
        w = np.ascontiguousarray(weights)
        wb = 8 if w.dtype == np.int64 else 4
        w = w.astype(np.int64 if wb == 8 else np.int32, copy=False)
        q = np.array([qn_prev >> 64, qn_prev & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64).view(np.int64)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(self.device).cuda_stream
            except Exception:
                stream = 0
        out = ctypes.c_void_p()
        rc = self._lib.louvain_resume(self._h, int(start_level), q.ctypes.data, len(rp) - 1,
                                      rp.ctypes.data, col.ctypes.data, w.ctypes.data, wb,
                                      PTR_HOST, ctypes.c_void_p(stream), ctypes.byref(out))
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return Result(self._lib, out, self)

    def csr_from_edges(self, n: int, src, dst, weights=None, stream: Optional[int] = None):
        """louvain_csr_from_edges: (row_ptr, col_idx, weights) as torch CUDA tensors of the
        symmetric CSR of an undirected edge list (numpy / torch arrays, host or device)."""
        import torch
        s_, k1, keep1 = _ptr_of(src)
        d_, k2, keep2 = _ptr_of(dst)
        w_, k3, keep3 = _ptr_of(weights)
        kinds = {k for k in (k1, k2, k3) if k is not None}
        if len(kinds) != 1:
            raise ValueError("src, dst and weights must all be on the host or all on the device")
        m = int(keep1.shape[0])
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        dev = torch.device("cuda", self.device)
        rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
        col = torch.empty(max(2 * m, 1), dtype=torch.int32, device=dev)
        w = torch.empty(max(2 * m, 1), dtype=torch.int32, device=dev)
        nnz = ctypes.c_int64()
        rc = self._lib.louvain_csr_from_edges(self._h, n, m, s_, d_, w_, kinds.pop(),
                                              ctypes.c_void_p(stream), rp.data_ptr(),
                                              col.data_ptr(), w.data_ptr(),
                                              ctypes.addressof(nnz))
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return rp, col[:nnz.value], w[:nnz.value]

    def run_batch(self, graph_vptr, row_ptr, col_idx, weights=None, graph_eptr=None,
                  stream: Optional[int] = None) -> List[Result]:
        """louvain_run_batch: one result per graph of a stacked block-diagonal CSR (graph g
        owns vertices graph_vptr[g] .. graph_vptr[g+1]-1; column ids are global).
        graph_vptr / graph_eptr are host arrays; the CSR arrays as in run()."""
        gv = np.ascontiguousarray(np.asarray(graph_vptr, dtype=np.int64))
        ge = None if graph_eptr is None else np.ascontiguousarray(
            np.asarray(graph_eptr, dtype=np.int64))
        G = int(gv.shape[0]) - 1
        if G < 1:
            raise ValueError("graph_vptr needs at least two entries")
        rp, k1, keep1 = _ptr_of(row_ptr)
        col, k2, keep2 = _ptr_of(col_idx)
        w, k3, keep3 = _ptr_of(weights)
        kinds = {k for k in (k1, k2, k3) if k is not None}
        if len(kinds) != 1:
            raise ValueError("row_ptr, col_idx and weights must all be on the host or all on the device")
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(self.device).cuda_stream
            except Exception:
                stream = 0
        outs = (ctypes.c_void_p * G)()
        rc = self._lib.louvain_run_batch(self._h, G, gv.ctypes.data,
                                         None if ge is None else ge.ctypes.data, rp, col, w,
                                         kinds.pop(), ctypes.c_void_p(stream), outs)
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return [Result(self._lib, ctypes.c_void_p(outs[g]), self) for g in range(G)]


    # ------------------------------------------------------------ serving
    def serve_open(self, hbm_budget_bytes: int, max_slots: int) -> None:
        """Start the request loop (louvain_serve_open)."""
        rc = self._lib.louvain_serve_open(self._h, int(hbm_budget_bytes), int(max_slots))
        if rc != OK:
            raise LouvainError(rc, self.last_error())

    def submit(self, row_ptr, col_idx, weights=None) -> int:
        """Queue one graph (host arrays, copied before the call returns); returns its ticket."""
        rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int64))
        col = np.ascontiguousarray(np.asarray(col_idx, dtype=np.int32))
        w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.int32))
        t = ctypes.c_uint64()
        rc = self._lib.louvain_submit(self._h, int(rp.shape[0]) - 1, rp.ctypes.data,
                                      col.ctypes.data, None if w is None else w.ctypes.data,
                                      PTR_HOST, ctypes.addressof(t))
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0) -> Optional[Result]:
        """The ticket's result, or None while it is pending; raises the graph's error."""
        out = ctypes.c_void_p()
        rc = self._lib.louvain_poll(self._h, int(ticket), int(wait_ms), ctypes.byref(out))
        if rc == PENDING:
            return None
        if rc != OK:
            raise LouvainError(rc, self.last_error())
        return Result(self._lib, out, self)

    def serve_status(self):
        """(bytes admitted, slots in use, queued, finished and not polled)."""
        st = np.zeros(4, np.int64)
        rc = self._lib.louvain_serve_status(self._h, st.ctypes.data)
        if rc != OK:
            raise LouvainError(rc, "serving is not open")
        return tuple(int(x) for x in st)

    def serve_close(self) -> None:
        rc = self._lib.louvain_serve_close(self._h)
        if rc != OK:
            raise LouvainError(rc, "serving is not open")


def stack_graphs(graphs):
    """Stack graphs given as (row_ptr, col_idx, weights) numpy arrays into the block-diagonal
    CSR of louvain_run_batch: returns (graph_vptr, graph_eptr, row_ptr, col_idx, weights).
    Column ids are shifted to global ids; weights None means all 1."""
    vptr = [0]
    eptr = [0]
    rps, cols, ws = [], [], []
    for rp, col, w in graphs:
        rp = np.asarray(rp, np.int64)
        col = np.asarray(col, np.int32)
        n = rp.shape[0] - 1
        nnz = int(rp[-1])
        rps.append(rp[1:] + eptr[-1])
        cols.append(col[:nnz] + np.int32(vptr[-1]))
        ws.append(np.ones(nnz, np.int32) if w is None else np.asarray(w, np.int32)[:nnz])
        vptr.append(vptr[-1] + n)
        eptr.append(eptr[-1] + nnz)
    row_ptr = np.concatenate([np.zeros(1, np.int64)] + rps).astype(np.int64)
    col_idx = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    weights = np.concatenate(ws).astype(np.int32) if ws else np.zeros(0, np.int32)
    return (np.asarray(vptr, np.int64), np.asarray(eptr, np.int64), row_ptr, col_idx, weights)
