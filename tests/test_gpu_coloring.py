"""Parity of the colouring variant (config.coloring, reading R17: Lu et al.'s colouring
heuristic) with the oracle's colouring mode, through the C ABI.

The colouring, the class order and every class's decisions are exact, so labels, Qn, the
sweep trace and the counters must be identical, in every bin configuration (each kernel
path filtered to one colour class) and with the other variants.  Batches and serving
reject the option.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

from test_gpu_parity import assert_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def lv():
    import paper_1805_10904_gb300 as m
    m.load()
    return m


ORACLE_KEYS = ("theta", "max_iters", "max_levels", "vertex_following", "vf_all_levels",
               "threshold_mode", "post_merge")


def run_both(torch, lv, g, **kw):
    ref = oracle.louvain(g.rp, g.col, g.w, coloring=True,
                         **{k: kw[k] for k in ORACLE_KEYS if k in kw})
    res = lv.Louvain(0, coloring=True, **kw).run(*to_dev(torch, g))
    return res, ref


@pytest.mark.parametrize("seed", range(30))
def test_coloring_fuzz(torch, lv, seed):
    g = gg.random_small(seed, n_max=80)
    res, ref = run_both(torch, lv, g, vertex_following=bool(seed % 3))
    assert_parity(res, ref)


BIN_CONFIGS = [
    {},
    {"bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32},
    {"bins": (0, 0, 0, 0, 0, 1), "chunk_entries": 32},
    {"bins": (0, 0, 0, 0, 0, 12288)},
    {"force_int128": True, "wide_sums": True, "bins": (2, 4, 8, 16, 32, 64),
     "chunk_entries": 64},
    {"profile": True, "sweep_streams": 0},
]


@pytest.mark.parametrize("cfg", BIN_CONFIGS)
@pytest.mark.parametrize("kind", ["planted", "rmat", "chung_lu"])
def test_coloring_bins(torch, lv, cfg, kind):
    if kind == "planted":
        g = gg.sbm(4096, 128, 0.10, 0.002, 1, 4, seed=1)
    elif kind == "rmat":
        g = gg.rmat(13, 16, seed=13)
    else:
        g = gg.chung_lu(6000, 2.1, 10.0, 1, 8, seed=5)
    res, ref = run_both(torch, lv, g, **cfg)
    assert_parity(res, ref)


@pytest.mark.parametrize("kw", [{"threshold_mode": 1, "theta": (1, 1000)},
                                {"vf_all_levels": True}, {"post_merge": True},
                                {"max_iters": 2}, {"max_levels": 2}, {"theta": (1, 30)}])
def test_coloring_with_other_options(torch, lv, kw):
    g = gg.rmat(12, 16, seed=21)
    res, ref = run_both(torch, lv, g, **kw)
    assert_parity(res, ref)


def test_coloring_host_pointers(torch, lv):
    g = gg.sbm(2000, 50, 0.3, 0.01, 1, 6, seed=8)
    ref = oracle.louvain(g.rp, g.col, g.w, coloring=True)
    res = lv.Louvain(0, coloring=True).run(g.rp, g.col, g.w)
    assert_parity(res, ref)


def test_coloring_four_cycle(torch, lv):
    g = gg.from_edges(4, [(0, 1, 1), (1, 2, 1), (2, 3, 1), (3, 0, 1)])
    res = lv.Louvain(0, coloring=True, vertex_following=False).run(*to_dev(torch, g))
    assert res.num_levels == 1
    assert res.labels(0).tolist() == [0, 1, 1, 0] and res.level(0).qn == 0
    assert res.trace() == [(0, 1, 2, 0), (0, 2, 0, 0), (1, 1, 0, 0)]


def test_coloring_rejected_by_batch_and_serving(torch, lv):
    graphs = [gg.sbm(300, 30, 0.25, 0.01, 1, 4, seed=2), gg.rmat(9, 8, seed=3)]
    vptr, eptr, rp, col, w = lv.stack_graphs([(x.rp, x.col, x.w) for x in graphs])
    h = lv.Louvain(0, coloring=True)
    with pytest.raises(lv.LouvainError) as e:
        h.run_batch(vptr, rp, col, w, graph_eptr=eptr)
    from paper_1805_10904_gb300.louvain import ERR_INVALID_ARG
    assert e.value.code == ERR_INVALID_ARG
    with pytest.raises(lv.LouvainError):
        h.serve_open(1 << 30, 4)
    # the handle still runs single graphs
    res = h.run(*to_dev(torch, graphs[0]))
    assert_parity(res, oracle.louvain(graphs[0].rp, graphs[0].col, graphs[0].w, coloring=True))
