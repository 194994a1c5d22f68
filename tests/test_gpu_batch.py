"""louvain_run_batch: every graph of a batch must get exactly the result of its own plain run.

The batch stacks graphs into one block-diagonal CSR; each graph keeps its own 2W, its own
phase controller (Algorithm 1 stopping rule) and its own outer test (Algorithm 2), so its
labels, Qn, iteration counts, trace and edge visits must equal both the oracle's and
louvain_run's on that graph alone, whatever the other graphs do.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

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


def dev(torch, *arrays):
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


def same_result(a, b):
    """Two library results (batch member vs plain run) are identical."""
    assert a.n == b.n and a.num_levels == b.num_levels
    for l in range(a.num_levels):
        assert np.array_equal(a.labels(l), b.labels(l)), f"labels differ at level {l}"
        assert a.level(l) == b.level(l)
    assert a.trace() == b.trace()
    assert a.counters()[0][0] == b.counters()[0][0]


def matches_oracle(res, ref):
    assert res.num_levels == len(ref.levels)
    for l, rl in enumerate(ref.levels):
        lev = res.level(l)
        assert np.array_equal(res.labels(l), rl.labels), f"labels differ at level {l}"
        assert lev.ncomm == rl.ncomm and lev.qn == rl.qn and lev.qn_init == rl.qn_init
        assert lev.iters == rl.iters and lev.n == rl.n and lev.nnz == rl.nnz
        assert lev.q == rl.q or abs(lev.q - rl.q) <= 1e-12 * abs(rl.q)
    assert res.trace() == ref.trace
    assert res.counters()[0][0] == ref.edge_visits


def mixed_graphs(seed):
    """Graphs of very different sizes and shapes, including the degenerate ones."""
    gs = [
        gg.sbm(600, 40, 0.3, 0.01, 1, 4, seed=seed),
        gg.from_edges(0, []),                                  # empty graph
        gg.chung_lu(900, 2.1, 10.0, 1, 8, seed=seed + 1),
        gg.from_edges(5, []),                                  # vertices, no edges
        gg.star(30),
        gg.rmat(9, 8, seed=seed + 2),
        gg.path(17, 3),
        gg.cliques_ring(6, 5),
        gg.from_edges(1, [(0, 0, 4)]),                         # one vertex with a loop
        gg.random_small(seed + 3, n_max=60),
        gg.sbm(2000, 100, 0.1, 0.002, 1, 8, seed=seed + 4),
        gg.disjoint_cliques(4, 3),
    ]
    return gs


BATCH_CONFIGS = [
    {},
    {"bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32},
    {"bins": (0, 0, 0, 0, 0, 2)},
    {"force_int128": True, "wide_sums": True, "bins": (0, 0, 0, 0, 0, 1), "chunk_entries": 32},
    {"theta": (1, 100), "max_levels": 2},
    {"max_iters": 2, "vertex_following": False},
    {"vf_all_levels": True, "theta": (0, 1)},
    {"cuda_graphs": False},
    {"threshold_mode": 1, "theta": (1, 1000)},
    {"post_merge": True, "max_iters": 2},
]


@pytest.mark.parametrize("ci", range(len(BATCH_CONFIGS)))
def test_batch_equals_plain_and_oracle(torch, lv, ci):
    kw = BATCH_CONFIGS[ci]
    graphs = mixed_graphs(100 + ci)
    h = lv.Louvain(0, **kw)
    vptr, eptr, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    batch = h.run_batch(vptr, *dev(torch, rp, col, w), graph_eptr=eptr)
    assert len(batch) == len(graphs)
    okw = {k: kw[k] for k in ("theta", "max_iters", "max_levels", "vertex_following",
                              "vf_all_levels", "threshold_mode", "post_merge") if k in kw}
    for g, res in zip(graphs, batch):
        plain = h.run(*dev(torch, g.rp, g.col, g.w))
        same_result(res, plain)
        matches_oracle(res, oracle.louvain(g.rp, g.col, g.w, **okw))


def test_batch_of_one_is_plain_run(torch, lv):
    g = gg.rmat(12, 16, seed=7)
    h = lv.Louvain(0)
    vptr, eptr, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w)])
    (res,) = h.run_batch(vptr, *dev(torch, rp, col, w))
    same_result(res, h.run(*dev(torch, g.rp, g.col, g.w)))


def test_batch_host_pointers_and_free_order(torch, lv):
    graphs = [gg.sbm(300 + 50 * k, 30, 0.3, 0.01, 1, 4, seed=k) for k in range(6)]
    h = lv.Louvain(0)
    vptr, _, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    batch = h.run_batch(vptr, rp, col, w)          # host arrays: copied inside the call
    refs = [oracle.louvain(g.rp, g.col, g.w) for g in graphs]
    # free results out of order; the others' shared label arrays must stay valid
    for k in (3, 0, 5):
        batch[k].close()
    for k in (1, 2, 4):
        matches_oracle(batch[k], refs[k])


def test_batch_unweighted(torch, lv):
    graphs = [gg.erdos_renyi(200 + 37 * k, 0.05, seed=k) for k in range(5)]
    h = lv.Louvain(0)
    vptr, _, rp, col, _ = lv.stack_graphs([(g.rp, g.col, None) for g in graphs])
    batch = h.run_batch(vptr, *dev(torch, rp, col), None)
    for g, res in zip(graphs, batch):
        ones = np.ones(g.nnz, np.int32)
        matches_oracle(res, oracle.louvain(g.rp, g.col, ones))


def test_batch_mix_sample(torch, lv):
    """A sample of the mixed workload (planted partitions and Chung-Lu power-law graphs of
    log-uniform sizes), smaller graphs so the oracle finishes quickly."""
    graphs = gg.batch_mix(24, seed=77, n_min=1000, n_max=12000)
    h = lv.Louvain(0)
    vptr, eptr, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    batch = h.run_batch(vptr, *dev(torch, rp, col, w), graph_eptr=eptr)
    for g, res in zip(graphs, batch):
        matches_oracle(res, oracle.louvain(g.rp, g.col, g.w))


def test_batch_rejects_bad_input(torch, lv):
    a = gg.path(4)
    b = gg.path(3)
    h = lv.Louvain(0)
    vptr, eptr, rp, col, w = lv.stack_graphs([(a.rp, a.col, a.w), (b.rp, b.col, b.w)])
    # an edge that crosses from graph 0 into graph 1
    bad = col.copy()
    bad[0] = 5
    with pytest.raises(lv.LouvainError) as e:
        h.run_batch(vptr, *dev(torch, rp, bad, w))
    assert e.value.code == lv.louvain.ERR_INDEX_RANGE
    # graph offsets that decrease, or that do not cover the CSR's entries
    with pytest.raises(lv.LouvainError) as e:
        h.run_batch(np.array([0, 5, 4, 7]), *dev(torch, rp, col, w))
    assert e.value.code == lv.louvain.ERR_INDEX_RANGE
    with pytest.raises(lv.LouvainError) as e:
        h.run_batch(vptr, *dev(torch, rp, col, w), graph_eptr=eptr + 1)
    assert e.value.code == lv.louvain.ERR_INDEX_RANGE
    # the handle stays usable
    res = h.run_batch(vptr, *dev(torch, rp, col, w))
    matches_oracle(res[1], oracle.louvain(b.rp, b.col, b.w))


def test_batch_mixing_wide_and_narrow_graphs(torch, lv):
    """One graph with 2W above 2^32 switches the whole step to int128 gains, 64-bit table
    sums and int64 coarse weights; the other graphs' results must not change."""
    big_w = gg.sbm(500, 25, 0.3, 0.01, 1, 4, seed=9)
    w = big_w.w.astype(np.int64) * (1 << 22)  # weights up to 2^24, 2W above 2^32
    assert int(w.sum()) > 2 ** 32 and int(w.max()) < 2 ** 31
    heavy = gg.Graph(big_w.rp, big_w.col, w.astype(np.int32), "heavy")
    graphs = [gg.sbm(700, 35, 0.25, 0.01, 1, 4, seed=1), heavy, gg.rmat(10, 8, seed=4),
              gg.cliques_ring(8, 6)]
    h = lv.Louvain(0)
    vptr, eptr, rp, col, ww = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    batch = h.run_batch(vptr, *dev(torch, rp, col, ww), graph_eptr=eptr)
    for g, res in zip(graphs, batch):
        same_result(res, h.run(*dev(torch, g.rp, g.col, g.w)))
        matches_oracle(res, oracle.louvain(g.rp, g.col, g.w))
