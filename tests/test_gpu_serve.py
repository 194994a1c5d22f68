"""Serving (louvain_serve_open / submit / poll): graphs that arrive over time join the graphs
already running at level boundaries; each graph's result must be identical to its plain
louvain_run and to the oracle, whatever else was in flight, and admission must respect the
slot count and the device-memory budget.
"""
import threading
import time

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


def same_result(a, b):
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
        assert lev.qn == rl.qn and lev.iters == rl.iters and lev.ncomm == rl.ncomm
    assert res.trace() == ref.trace
    assert res.counters()[0][0] == ref.edge_visits


def request_mix(seed):
    gs = []
    for k in range(14):
        kind = k % 4
        if kind == 0:
            gs.append(gg.rmat(8 + (k % 5), 16, seed=seed + k))
        elif kind == 1:
            gs.append(gg.sbm(300 + 97 * k, 32 + 8 * (k % 5), 0.2, 0.004, 1, 16, seed=seed + k))
        elif kind == 2:
            gs.append(gg.chung_lu(500 + 61 * k, 2.1, 10.0, 1, 8, seed=seed + k))
        else:
            gs.append(gg.random_small(seed + k, n_max=70))
    gs.insert(5, gg.from_edges(0, []))      # empty graph
    gs.insert(9, gg.from_edges(3, []))      # no edges
    return gs


@pytest.mark.parametrize("slots", [1, 3, 64])
def test_served_results_equal_plain_runs(torch, lv, slots):
    graphs = request_mix(40 + slots)
    plain_h = lv.Louvain(0)
    plain = [plain_h.run(g.rp, g.col, g.w) for g in graphs]
    h = lv.Louvain(0, torch_alloc=False)
    h.serve_open(8 << 30, slots)
    tickets = []
    for k, g in enumerate(graphs):
        tickets.append(h.submit(g.rp, g.col, g.w))
        if k % 3 == 0:
            time.sleep(0.002)  # arrivals spread over the running steps
    results = [h.poll(t, -1) for t in tickets]
    h.serve_close()
    for g, r, p in zip(graphs, results, plain):
        same_result(r, p)
    for k in (0, 1, 2):
        matches_oracle(results[k], oracle.louvain(graphs[k].rp, graphs[k].col, graphs[k].w))


def test_serving_from_a_second_thread_with_polling(torch, lv):
    graphs = [gg.sbm(400 + 50 * k, 40, 0.25, 0.005, 1, 16, seed=k) for k in range(10)]
    h = lv.Louvain(0, torch_alloc=False)
    h.serve_open(4 << 30, 4)
    tickets = [None] * len(graphs)

    def producer():
        for k, g in enumerate(graphs):
            tickets[k] = h.submit(g.rp, g.col, g.w)
            time.sleep(0.003)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    results = {}
    deadline = time.time() + 120
    while len(results) < len(graphs) and time.time() < deadline:
        for k, t in enumerate(tickets):
            if k not in results:
                r = h.poll(t, 0)
                if r is not None:
                    results[k] = r
        time.sleep(0.001)
    h.serve_close()
    assert len(results) == len(graphs)
    for k, g in enumerate(graphs):
        matches_oracle(results[k], oracle.louvain(g.rp, g.col, g.w))


def test_budget_rejects_oversized_and_bad_graphs_fail_alone(torch, lv):
    small = [gg.sbm(200 + 10 * k, 20, 0.3, 0.01, 1, 4, seed=k) for k in range(4)]
    big = gg.rmat(12, 16, seed=3)
    bad = gg.path(6)
    bad_col = bad.col.copy()
    bad_col[2] = 99  # outside [0, n)
    h = lv.Louvain(0, torch_alloc=False)
    budget = 4 << 20  # holds all the small graphs, but not the R-MAT graph alone
    h.serve_open(budget, 8)
    t_small = [h.submit(g.rp, g.col, g.w) for g in small[:2]]
    t_big = h.submit(big.rp, big.col, big.w)
    t_bad = h.submit(bad.rp, bad_col, bad.w)
    t_small += [h.submit(g.rp, g.col, g.w) for g in small[2:]]
    peak = 0
    for _ in range(50):
        peak = max(peak, h.serve_status()[0])
        time.sleep(0.001)
    with pytest.raises(lv.LouvainError) as e:
        h.poll(t_big, -1)
    assert e.value.code == lv.louvain.ERR_REJECTED
    with pytest.raises(lv.LouvainError) as e:
        h.poll(t_bad, -1)
    assert e.value.code == lv.louvain.ERR_INDEX_RANGE
    for t, g in zip(t_small, small):
        matches_oracle(h.poll(t, -1), oracle.louvain(g.rp, g.col, g.w))
    assert peak <= budget
    # a consumed ticket is unknown afterwards
    with pytest.raises(lv.LouvainError) as e:
        h.poll(t_small[0], 0)
    assert e.value.code == lv.louvain.ERR_INVALID_ARG
    h.serve_close()


def test_serving_handle_refuses_plain_runs_and_closes_with_unpolled_results(torch, lv):
    g = gg.sbm(500, 50, 0.2, 0.01, 1, 4, seed=2)
    h = lv.Louvain(0, torch_alloc=False)
    h.serve_open(1 << 30, 2)
    with pytest.raises(lv.LouvainError) as e:
        h.run(g.rp, g.col, g.w)
    assert e.value.code == lv.louvain.ERR_INVALID_ARG
    for _ in range(3):
        h.submit(g.rp, g.col, g.w)  # never polled
    h.serve_close()
    # the handle runs plain graphs again once serving is closed
    matches_oracle(h.run(g.rp, g.col, g.w), oracle.louvain(g.rp, g.col, g.w))
