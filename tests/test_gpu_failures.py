"""Failures made on the host (no GPU fault): an allocator that refuses the k-th device
allocation must give LOUVAIN_ERR_OOM and leave the handle usable, for plain runs, batches
and serving; results after the failure must still equal the oracle's."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_1805_10904_gb300 as m
    m.load()
    return m


def refuse_at(k):
    count = [0]

    def hook(nbytes):
        count[0] += 1
        return count[0] != k

    return hook, count


def same_as_oracle(res, g):
    ref = oracle.louvain(g.rp, g.col, g.w)
    assert res.num_levels == len(ref.levels)
    for l, rl in enumerate(ref.levels):
        assert np.array_equal(res.labels(l), rl.labels) and res.level(l).qn == rl.qn


@pytest.mark.parametrize("k", [1, 3, 10, 25, 60, 120])
def test_failed_allocation_in_a_run(lv, k):
    import torch
    g = gg.rmat(12, 16, seed=12)
    d = [torch.from_numpy(a).cuda() for a in (g.rp, g.col, g.w)]
    hook, count = refuse_at(k)
    h = lv.Louvain(0, alloc_hook=hook)
    try:
        res = h.run(*d)
    except lv.LouvainError as e:
        assert e.code == lv.louvain.ERR_OOM
    else:  # the run needed fewer than k allocations
        assert count[0] < k
        same_as_oracle(res, g)
    h.alloc_hook = None
    same_as_oracle(h.run(*d), g)


@pytest.mark.parametrize("k", [2, 15, 40])
def test_failed_allocation_in_a_batch(lv, k):
    import torch
    graphs = [gg.sbm(400 + 40 * i, 40, 0.2, 0.01, 1, 4, seed=i) for i in range(5)]
    vptr, eptr, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    d = [torch.from_numpy(a).cuda() for a in (rp, col, w)]
    hook, count = refuse_at(k)
    h = lv.Louvain(0, alloc_hook=hook)
    try:
        h.run_batch(vptr, *d)
    except lv.LouvainError as e:
        assert e.code == lv.louvain.ERR_OOM
    else:
        assert count[0] < k
    h.alloc_hook = None
    for g, res in zip(graphs, h.run_batch(vptr, *d)):
        same_as_oracle(res, g)


def test_failed_allocation_while_serving(lv):
    """An allocation refused inside the serving engine fails the graphs it holds with OOM;
    graphs submitted afterwards are served correctly."""
    graphs = [gg.sbm(300 + 30 * i, 30, 0.25, 0.01, 1, 4, seed=i) for i in range(4)]
    state = {"refuse": False}
    h = lv.Louvain(0, alloc_hook=lambda nbytes: not state["refuse"])
    h.serve_open(1 << 30, 4)
    ok = h.submit(graphs[0].rp, graphs[0].col, graphs[0].w)
    same_as_oracle(h.poll(ok, -1), graphs[0])
    state["refuse"] = True
    t = h.submit(graphs[1].rp, graphs[1].col, graphs[1].w)
    with pytest.raises(lv.LouvainError) as e:
        h.poll(t, -1)
    assert e.value.code == lv.louvain.ERR_OOM
    state["refuse"] = False
    for g in graphs[2:]:
        same_as_oracle(h.poll(h.submit(g.rp, g.col, g.w), -1), g)
    h.serve_close()
