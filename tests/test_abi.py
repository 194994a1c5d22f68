"""The C-ABI library loads and exports every symbol that include/*.h declares.

Runs without a GPU: it builds the library (nvcc cross-compiles for sm_103a), loads it,
and calls only host-side entry points.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(louvain_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1805_10904_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["louvain_create", "louvain_run", "louvain_destroy", "louvain_result_labels",
                     "louvain_result_modularity", "louvain_last_error", "louvain_config_init"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_config_defaults(lib):
    from paper_1805_10904_gb300.louvain import Config
    cfg = Config()
    assert lib.louvain_config_init(ctypes.byref(cfg)) == 0
    assert cfg.struct_size == ctypes.sizeof(Config)
    assert (cfg.theta_num, cfg.theta_den) == (1, 1_000_000)
    assert cfg.max_iters == 1000 and cfg.vertex_following == 1 and cfg.checks == 1
    assert cfg.cuda_graphs == 1 and cfg.sweep_streams == 4 and cfg.autotune == 0
    assert cfg.threshold_mode == 0 and cfg.post_merge == 0 and cfg.keep_coarse == 0
    assert cfg.part_keys == 2048
    assert lib.louvain_config_init(None) == 1


def test_invalid_config_rejected_before_any_device_call(lib):
    from paper_1805_10904_gb300.louvain import Config
    cfg = Config()
    lib.louvain_config_init(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    bad = Config.from_buffer_copy(cfg)
    bad.theta_den = 0
    assert lib.louvain_create(ctypes.byref(bad), 0, ctypes.byref(h)) == 1
    bad = Config.from_buffer_copy(cfg)
    bad.chunk_entries = 1000
    assert lib.louvain_create(ctypes.byref(bad), 0, ctypes.byref(h)) == 1
    bad = Config.from_buffer_copy(cfg)
    bad.bin_small = 9
    assert lib.louvain_create(ctypes.byref(bad), 0, ctypes.byref(h)) == 1
    for field, value in (("sweep_streams", 5), ("threshold_mode", 2), ("post_merge", 3),
                         ("keep_coarse", -1), ("part_keys", 63), ("part_keys", -5),
                         ("coloring", 2), ("host_labels", 2), ("host_labels", -1)):
        bad = Config.from_buffer_copy(cfg)
        setattr(bad, field, value)
        assert lib.louvain_create(ctypes.byref(bad), 0, ctypes.byref(h)) == 1
    assert not h.value


def test_null_handle_calls_are_safe(lib):
    lib.louvain_last_error.restype = ctypes.c_char_p
    assert lib.louvain_last_error(None) == b""
    lib.louvain_destroy(None)
    lib.louvain_result_free(None)
    assert lib.louvain_result_num_levels(None) == 0
    assert lib.louvain_result_coarsen_stats(None, None, None, None) == 1
    assert lib.louvain_run(None, 0, None, None, None, 0, None, None) == 1
    assert lib.louvain_run_batch(None, 1, None, None, None, None, None, 0, None, None) == 1
    assert lib.louvain_serve_open(None, ctypes.c_uint64(1), 1) == 1
    assert lib.louvain_submit(None, 0, None, None, None, 0, None) == 1
    assert lib.louvain_poll(None, ctypes.c_uint64(1), 0, None) == 1
    assert lib.louvain_serve_status(None, None) == 1
    assert lib.louvain_serve_close(None) == 1
    assert lib.louvain_csr_from_edges(None, 0, 0, None, None, None, 0, None, None, None, None,
                                      None) == 1
    assert lib.louvain_result_labels_into(None, 0, None) == 1
    assert lib.louvain_result_bin_stats(None, 0, None, None, None, None, None) == 1


def test_stack_graphs_builds_block_diagonal_csr():
    import numpy as np
    import graphgen as gg
    from paper_1805_10904_gb300 import stack_graphs
    graphs = [gg.path(4, 2), gg.from_edges(0, []), gg.star(3), gg.from_edges(2, [(1, 1, 5)])]
    vptr, eptr, rp, col, w = stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    assert list(vptr) == [0, 4, 4, 8, 10]
    assert list(eptr) == [0, 6, 6, 12, 13]
    assert rp.dtype == np.int64 and col.dtype == np.int32 and w.dtype == np.int32
    whole = gg.Graph(rp, col, w, "stacked")
    gg.check_csr(whole)
    for k, g in enumerate(graphs):
        v0, v1 = vptr[k], vptr[k + 1]
        sub = rp[v0:v1 + 1] - rp[v0]
        assert np.array_equal(sub, g.rp)
        assert np.array_equal(col[rp[v0]:rp[v1]] - v0, g.col)
        assert np.array_equal(w[rp[v0]:rp[v1]], g.w)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1805_10904_gb300.louvain as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        L.load()
