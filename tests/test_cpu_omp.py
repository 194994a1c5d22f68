"""The multi-threaded CPU baseline (cpu_omp, OpenMP) against the oracle: every level's
labels, Qn, Qn at the level's start, sweep count and graph sizes, the sweep trace
(Algorithm 1) and the edge-visit count are identical, for 1, 2, 3 and 8 threads, on the
generator families of the benchmark workloads and on the small structured graphs of the
oracle's pins (cliques, stars, paths, graphs with loops and isolated vertices)."""
import numpy as np
import pytest

import cpu_omp
import graphgen as gg
import oracle


def same(a, b):
    assert a.tw == b.tw
    assert len(a.levels) == len(b.levels)
    for x, y in zip(a.levels, b.levels):
        assert np.array_equal(x.labels, y.labels)
        assert (x.ncomm, x.qn, x.qn_init, x.iters, x.n, x.nnz) == \
               (y.ncomm, y.qn, y.qn_init, y.iters, y.n, y.nnz)
    assert a.trace == b.trace
    assert a.edge_visits == b.edge_visits and a.sweeps == b.sweeps
    assert a.hit_iter_cap == b.hit_iter_cap


GRAPHS = {
    "sbm4096": lambda: gg.sbm(4096, 128, 0.10, 0.002, 1, 4, seed=1),
    "rmat14": lambda: gg.rmat(14, 16, seed=14),
    "chung_lu": lambda: gg.chung_lu(5000, 2.1, 10.0, 1, 8, seed=4),
    "cliques_ring": lambda: gg.cliques_ring(6, 6, 4, 1),
    "star": lambda: gg.star(9, 3),
    "path": lambda: gg.path(17, 2),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_omp_equals_oracle(name, threads):
    g = GRAPHS[name]()
    same(cpu_omp.louvain(g.rp, g.col, g.w, threads=threads), oracle.louvain(g.rp, g.col, g.w))


@pytest.mark.parametrize("seed", range(24))
def test_omp_equals_oracle_fuzz(seed):
    g = gg.random_small(seed, n_max=60)
    for kw in ({}, {"vf_all_levels": True}, {"vertex_following": False},
               {"theta": (1, 30)}, {"max_iters": 2}, {"max_levels": 2}):
        same(cpu_omp.louvain(g.rp, g.col, g.w, threads=3, **kw),
             oracle.louvain(g.rp, g.col, g.w, **kw))


def test_omp_unweighted_and_empty():
    g = gg.rmat(10, 8, seed=2)
    same(cpu_omp.louvain(g.rp, g.col, None, threads=4), oracle.louvain(g.rp, g.col, None))
    empty = cpu_omp.louvain(np.zeros(1, np.int64), np.zeros(0, np.int32), None, threads=2)
    assert empty.levels == [] and empty.trace == []


def test_omp_rejects_repeated_columns():
    rp = np.array([0, 2, 3, 4], np.int64)
    col = np.array([1, 1, 0, 0], np.int32)
    with pytest.raises(RuntimeError):
        cpu_omp.louvain(rp, col, None, threads=2)
