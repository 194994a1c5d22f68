"""config.host_labels: every recorded level's labels are copied to pinned host memory while
the later levels run.  The labels (copied out or viewed in place), Qn and the trace must be
those of a run without the option, and of the oracle; views stay valid while the result is
alive, also after its handle is gone; batches and served graphs get the same labels.
"""
import gc

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


GRAPHS = [gg.rmat(14, 16, seed=41), gg.sbm(4096, 128, 0.10, 0.002, 1, 4, seed=3),
          gg.chung_lu(6000, 2.1, 10.0, 1, 8, seed=7)]


@pytest.mark.parametrize("k", range(len(GRAPHS)))
def test_host_labels_equal_device_labels_and_oracle(torch, lv, k):
    g = GRAPHS[k]
    ref = oracle.louvain(g.rp, g.col, g.w)
    plain = lv.Louvain(0).run(*to_dev(torch, g))
    h = lv.Louvain(0, host_labels=True)
    for rep in range(3):  # later runs reuse the pinned blocks of the earlier ones
        res = h.run(*to_dev(torch, g))
        assert_parity(res, ref)
        for l in range(res.num_levels):
            view = res.labels(l, copy=False)
            assert not view.flags.writeable
            assert np.array_equal(view, plain.labels(l))
            assert np.array_equal(view, ref.levels[l].labels)
        res.close()


def test_host_pointer_inputs_and_views_outlive_the_handle(torch, lv):
    g = GRAPHS[0]
    ref = oracle.louvain(g.rp, g.col, g.w)
    h = lv.Louvain(0, host_labels=True, torch_alloc=False)
    views = [h.run(g.rp, g.col, g.w).labels(l, copy=False) for l in range(len(ref.levels))]
    h.close()
    del h
    gc.collect()
    for l, v in enumerate(views):  # each view holds its (temporary) result
        assert np.array_equal(v, ref.levels[l].labels)


def test_host_labels_in_a_batch(torch, lv):
    graphs = [gg.sbm(300, 30, 0.25, 0.01, 1, 4, seed=2), gg.rmat(9, 8, seed=3), GRAPHS[2]]
    vptr, eptr, rp, col, w = lv.stack_graphs([(x.rp, x.col, x.w) for x in graphs])
    results = lv.Louvain(0, host_labels=True).run_batch(vptr, rp, col, w, graph_eptr=eptr)
    for g, res in zip(graphs, results):
        ref = oracle.louvain(g.rp, g.col, g.w)
        assert res.num_levels == len(ref.levels)
        for l in range(res.num_levels):
            assert np.array_equal(res.labels(l, copy=False), ref.levels[l].labels)
            assert np.array_equal(res.labels(l), ref.levels[l].labels)


def test_host_labels_when_served(torch, lv):
    h = lv.Louvain(0, host_labels=True, torch_alloc=False)
    h.serve_open(1 << 30, 4)
    try:
        tickets = [(g, h.submit(g.rp, g.col, g.w)) for g in GRAPHS]
        for g, t in tickets:
            res = h.poll(t, wait_ms=-1)
            ref = oracle.louvain(g.rp, g.col, g.w)
            for l in range(res.num_levels):
                assert np.array_equal(res.labels(l, copy=False), ref.levels[l].labels)
    finally:
        h.serve_close()

