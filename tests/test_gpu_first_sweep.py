"""The first sweep of every phase scores row entries directly, without tables.

A phase starts from singletons (plus vertex following), so on rows that list each column at
most once the candidates of a vertex other than its own community are distinct and each
comes from one entry.  The library takes that path whenever it holds (induced graphs always,
input graphs whose rows have strictly increasing columns) and the table kernels otherwise.
Every case here must give the oracle's result exactly, and the bin statistics must show
which path each phase's first sweep took.
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


def assert_parity(res, ref):
    assert res.num_levels == len(ref.levels)
    for l, rl in enumerate(ref.levels):
        lev = res.level(l)
        assert np.array_equal(res.labels(l), rl.labels), f"labels differ at level {l}"
        assert lev.ncomm == rl.ncomm and lev.qn == rl.qn and lev.qn_init == rl.qn_init
        assert lev.iters == rl.iters and lev.n == rl.n and lev.nnz == rl.nnz
    assert res.trace() == ref.trace
    assert res.counters()[0][0] == ref.edge_visits


def phases(res):
    """Phases run (recorded levels and the last one that merged nothing)."""
    return sum(1 for rec in res.trace() if rec[1] == 1)


def shuffled_rows(g, seed):
    """The same graph with the entries of every row in a random order."""
    rng = np.random.default_rng(seed)
    col, w = g.col.copy(), g.w.copy()
    for i in range(g.n):
        b, e = int(g.rp[i]), int(g.rp[i + 1])
        if e - b > 1:
            p = rng.permutation(e - b) + b
            col[b:e], w[b:e] = g.col[p], g.w[p]
    return gg.Graph(g.rp.copy(), col, w, g.name + "-shuffled")


def split_entries(g, seed, frac=0.3):
    """Edges of weight >= 2 stored as two entries (w1 + w2 = w) in both directions; rows
    stay sorted, with the column repeated."""
    rng = np.random.default_rng(seed)
    split = {}
    for i in range(g.n):
        for k in range(int(g.rp[i]), int(g.rp[i + 1])):
            j = int(g.col[k])
            if i < j and g.w[k] >= 2 and rng.random() < frac:
                split[(i, j)] = int(rng.integers(1, int(g.w[k])))
    rp, col, w = [0], [], []
    for i in range(g.n):
        for k in range(int(g.rp[i]), int(g.rp[i + 1])):
            j, x = int(g.col[k]), int(g.w[k])
            a = split.get((min(i, j), max(i, j)))
            if a is None or i == j:
                col.append(j)
                w.append(x)
            else:
                col += [j, j]
                w += [a, x - a]
        rp.append(len(col))
    return gg.Graph(np.array(rp, np.int64), np.array(col, np.int32), np.array(w, np.int32),
                    g.name + "-split")


def vf_heavy(seed):
    """Hubs with many degree-one leaves, isolated pairs, a leaf on a leaf chain, loops."""
    rng = np.random.default_rng(seed)
    edges = {}

    def add(u, v, x):
        edges.setdefault((min(u, v), max(u, v)), x)

    n = 0
    hubs = []
    for _ in range(12):
        hub = n
        hubs.append(hub)
        leaves = int(rng.integers(3, 40))
        for t in range(leaves):
            add(hub, hub + 1 + t, int(rng.integers(1, 5)))
        n += leaves + 1
    for a in range(len(hubs)):  # hubs joined in a ring
        add(hubs[a], hubs[(a + 1) % len(hubs)], 2)
    for _ in range(6):  # isolated pairs, the last with a loop
        add(n, n + 1, 3)
        n += 2
    add(n - 1, n - 1, 2)
    add(n, n + 1, 1)  # a chain ending in a hub
    add(n + 1, n + 2, 1)
    add(n + 2, 0, 4)
    n += 3
    return gg.from_edges(n, [(u, v, x) for (u, v), x in edges.items()])


CASES = [
    lambda: gg.sbm(4096, 64, 0.2, 0.004, 1, 4, seed=31),
    lambda: gg.rmat(13, 16, seed=32),
    lambda: gg.chung_lu(9000, 2.1, 10.0, 1, 8, seed=33),
    lambda: vf_heavy(34),
    lambda: gg.random_small(35, n_max=80),
]
CONFIGS = [
    {},
    {"bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32},   # cluster bins and chunked rows
    {"bins": (0, 0, 0, 0, 0, 2), "force_int128": True},  # rows in 1024-thread CTAs
    {"vf_all_levels": True, "cuda_graphs": False},
    {"vertex_following": False, "wide_sums": True},
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("ci", range(len(CONFIGS)))
def test_first_sweep_every_phase(torch, lv, case, ci):
    g = CASES[case]()
    kw = CONFIGS[ci]
    okw = {k: kw[k] for k in ("vertex_following", "vf_all_levels") if k in kw}
    h = lv.Louvain(0, profile=True, **kw)
    res = h.run(*dev(torch, g.rp, g.col, g.w))
    assert_parity(res, oracle.louvain(g.rp, g.col, g.w, **okw))
    nb = len(res.bin_stats()) // 2
    assert res.bin_stats()[nb]["launches"] == phases(res)   # every phase began table-free
    assert res.bin_stats()[0]["launches"] == res.counters()[0][1] - phases(res)


@pytest.mark.parametrize("case", [0, 1, 2])
@pytest.mark.parametrize("chunk", [32, 256])
def test_every_row_chunked(torch, lv, case, chunk):
    """Bin bounds (0, 0, 0, 0, 0, 1) send every row longer than 16 (the largest cluster
    bin's bound) to the chunked bin (all-zero bounds mean the defaults); in the first sweep
    a row spanning several chunks is combined from per-chunk partial argmaxes."""
    g = CASES[case]()
    h = lv.Louvain(0, profile=True, bins=(0, 0, 0, 0, 0, 1), chunk_entries=chunk)
    res = h.run(*dev(torch, g.rp, g.col, g.w))
    assert_parity(res, oracle.louvain(g.rp, g.col, g.w))
    nb = len(res.bin_stats()) // 2
    # every phase whose graph still has a row longer than 16 launched the chunk kernels
    assert 1 <= res.bin_stats()[2 * nb - 1]["launches"] <= phases(res)
    assert 1 <= res.bin_stats()[nb - 1]["launches"] <= res.counters()[0][1] - phases(res)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_unsorted_rows_take_tables_at_the_first_level(torch, lv, case):
    g = shuffled_rows(CASES[case](), seed=case)
    h = lv.Louvain(0, profile=True)
    res = h.run(*dev(torch, g.rp, g.col, g.w))
    assert_parity(res, oracle.louvain(g.rp, g.col, g.w))
    nb = len(res.bin_stats()) // 2
    if any(np.any(np.diff(g.col[g.rp[i]:g.rp[i + 1]]) <= 0) for i in range(g.n)):
        assert res.bin_stats()[nb]["launches"] == phases(res) - 1  # induced levels only


@pytest.mark.parametrize("case", [0, 1, 3])
def test_repeated_columns(torch, lv, case):
    g = split_entries(CASES[case](), seed=40 + case)
    h = lv.Louvain(0, profile=True)
    res = h.run(*dev(torch, g.rp, g.col, g.w))
    assert_parity(res, oracle.louvain(g.rp, g.col, g.w))
    nb = len(res.bin_stats()) // 2
    assert res.bin_stats()[nb]["launches"] == phases(res) - 1


def test_batch_with_one_unsorted_graph(torch, lv):
    graphs = [CASES[0](), shuffled_rows(gg.rmat(10, 8, seed=3), 1), CASES[3](),
              gg.cliques_ring(6, 5)]
    h = lv.Louvain(0)
    vptr, eptr, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    batch = h.run_batch(vptr, *dev(torch, rp, col, w), graph_eptr=eptr)
    for g, res in zip(graphs, batch):
        assert_parity(res, oracle.louvain(g.rp, g.col, g.w))


@pytest.mark.parametrize("part_keys", [64, 1 << 30])
@pytest.mark.parametrize("scale", [16, 17])
def test_chunked_rows_partitioned_merge(torch, lv, scale, part_keys):
    """Table sweeps merge a chunked row's keys partition by partition.  part_keys = 64 gives
    many small partitions; 2^30 gives one partition per row, so the hub rows' partitions
    outgrow the shared table and spill into the row's global table."""
    g = gg.rmat(scale, 16, seed=5)
    h = lv.Louvain(0, profile=True, bins=(0, 0, 0, 0, 0, 1), chunk_entries=256,
                   part_keys=part_keys)
    res = h.run(*dev(torch, g.rp, g.col, g.w))
    assert_parity(res, oracle.louvain(g.rp, g.col, g.w))
