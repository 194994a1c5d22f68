"""Properties of the full multi-level run on R-MAT scale 22 (edge factor 16, seed 22) that
hold at any size, checked without the oracle: every level's labels are a compaction
0..k-1, levels only merge, and the Qn the GPU reports equals Eq. 3 recomputed from the
labels with numpy integer arithmetic.  (Label-for-label parity with the oracle at this
size is in test_gpu_golden.py.)"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def graph():
    return gg.rmat(22, 16, 0.57, 0.19, 0.19, 1, 16, seed=22)


@pytest.fixture(scope="module")
def dev_graph(graph):
    import torch
    d = torch.device("cuda:0")
    return [torch.from_numpy(x).to(d) for x in (graph.rp, graph.col, graph.w)]


def _qn_numpy(g, labels):
    """Eq. 3 times (2W)^2 from the labels, with numpy integer sums (independent of both
    the oracle and the library)."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rp))
    w = g.w.astype(np.int64)
    internal = int(w[labels[rows] == labels[g.col]].sum())
    dvert = np.zeros(g.n, np.int64)
    np.add.at(dvert, rows, w)
    dcomm = np.zeros(int(labels.max()) + 1, np.int64)
    np.add.at(dcomm, labels, dvert)
    tw = int(dvert.sum())
    sq = sum(int(x) * int(x) for x in dcomm)
    return tw * internal - sq, tw


def test_full_run_properties(graph, dev_graph):
    import paper_1805_10904_gb300 as lv
    res = lv.Louvain(0, profile=True, autotune=True).run(*dev_graph)
    assert res.num_levels >= 2
    prev = None
    for l in range(res.num_levels):
        lab = res.labels(l)
        lev = res.level(l)
        k = lev.ncomm
        assert lab.min() == 0 and lab.max() == k - 1 and len(np.unique(lab)) == k
        if prev is not None:
            # a community of level l-1 maps into exactly one community of level l
            pairs = np.unique(prev.astype(np.int64) * (k + 1) + lab)
            assert len(pairs) == len(np.unique(prev))
        qn, tw = _qn_numpy(graph, lab)
        assert tw == res.tw and qn == lev.qn
        prev = lab
