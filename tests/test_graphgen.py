"""Seeded input generators: determinism, CSR contract, distribution statistics."""
import numpy as np
import pytest

import graphgen as gg


def test_sbm_planted_partition_shape():
    """4,096 vertices in 32 blocks of 128, p_in = 0.10, p_out = 0.002, weights in [1, 4]."""
    g = gg.sbm(4096, 128, 0.10, 0.002, 1, 4, seed=1)
    gg.check_csr(g)
    assert g.n == 4096
    # expected degree 127 * 0.10 + 3968 * 0.002 = 20.64
    assert abs(g.nnz / g.n - 20.64) < 0.5
    assert g.w.min() == 1 and g.w.max() == 4
    rows = np.repeat(np.arange(g.n), g.degrees())
    intra = (rows // 128 == g.col // 128).mean()
    assert abs(intra - 12.7 / 20.64) < 0.02


def test_determinism_and_seed_sensitivity():
    a = gg.rmat(12, seed=7)
    b = gg.rmat(12, seed=7)
    c = gg.rmat(12, seed=8)
    assert np.array_equal(a.rp, b.rp) and np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w)
    assert not (len(a.col) == len(c.col) and np.array_equal(a.col, c.col))


def test_rmat_contract_and_skew():
    g = gg.rmat(14, 16, seed=22)
    gg.check_csr(g)
    assert g.n == 1 << 14
    deg = g.degrees()
    # loops dropped and duplicates merged: at most 2 * 16 * n stored entries
    assert g.nnz <= 2 * 16 * g.n
    assert deg.max() > 50 * deg.mean()
    assert (deg == 0).sum() > 0
    assert g.w.min() >= 1 and g.w.max() <= 16


def test_chung_lu_power_law():
    g = gg.chung_lu(50_000, 2.1, 10.0, 1, 8, seed=3)
    gg.check_csr(g)
    deg = g.degrees()
    assert 6.0 < deg.mean() < 10.5
    assert deg.max() > 20 * deg.mean()


def test_from_pairs_merges_duplicates_and_drops_loops():
    g = gg.from_pairs(4, [(0, 1), (1, 0), (2, 2), (2, 3)], 1, 5, seed=3)
    gg.check_csr(g)
    assert g.nnz == 4
    assert g.col.tolist() == [1, 0, 3, 2]


def test_small_builders_contract():
    for s in range(30):
        gg.check_csr(gg.random_small(s))
    gg.check_csr(gg.cliques_ring(6, 6, 4, 1))
    with pytest.raises(ValueError):
        gg.from_edges(3, [(0, 1, 1), (1, 0, 1)])


def test_graph_seed_family():
    seeds = [gg.graph_seed(3, k) for k in range(100)]
    assert len(set(seeds)) == 100
    assert seeds == [gg.graph_seed(3, k) for k in range(100)]
