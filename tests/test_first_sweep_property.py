"""The precondition of the table-free first sweep, checked on the CPU with the oracle.

At the start of a phase every vertex is a singleton, except that vertex following (level 0,
or every level when asked) puts a degree-one vertex into its only neighbour's community.  On
a symmetric graph whose rows list each column once, the communities of row i's entries other
than C(i) are then pairwise distinct, so each candidate's e_{i->c} is a single entry's weight.
The GPU's first sweep relies on this; here it is checked for input graphs and for graphs the
oracle induces at later levels, and a repeated column is shown to break it.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle


def distinct_candidates(rp, col, C):
    """True when no row has two non-loop entries in the same community other than its own."""
    for i in range(len(rp) - 1):
        seen = set()
        for k in range(int(rp[i]), int(rp[i + 1])):
            j = int(col[k])
            if j == i or C[j] == C[i]:
                continue
            if C[j] in seen:
                return False
            seen.add(C[j])
    return True


def followers_carry_own_label(rp, col, C):
    """Every entry whose label differs from its column's id carries the row's own label."""
    for i in range(len(rp) - 1):
        for k in range(int(rp[i]), int(rp[i + 1])):
            j = int(col[k])
            if j != i and C[j] != j and C[j] != C[i]:
                return False
    return True


GRAPHS = [
    lambda s: gg.random_small(s, n_max=60),
    lambda s: gg.erdos_renyi(80, 0.04, seed=s, wmax=5, loops=0.2),
    lambda s: gg.rmat(9, 4, seed=s),
    lambda s: gg.chung_lu(400, 2.1, 3.0, 1, 4, seed=s),
    lambda s: gg.star(25),
    lambda s: gg.path(30, 2),
    lambda s: gg.from_edges(6, [(0, 1, 2), (2, 3, 1), (3, 3, 4), (4, 5, 1)]),  # isolated pairs
]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("seed", range(4))
def test_phase_start_candidates_are_distinct(gi, seed):
    g = GRAPHS[gi](500 + seed)
    singletons = np.arange(g.n, dtype=np.int32)
    assert distinct_candidates(g.rp, g.col, singletons)
    C = oracle.vertex_following(g.rp, g.col)
    assert followers_carry_own_label(g.rp, g.col, C)
    assert distinct_candidates(g.rp, g.col, C)


@pytest.mark.parametrize("seed", range(6))
def test_induced_graphs_keep_the_property(seed):
    """Every level's graph (singletons, and vertex following as with vf_all_levels)."""
    g = gg.rmat(10, 8, seed=600 + seed)
    rp, col, w = g.rp, g.col, g.w.astype(np.int64)
    for _ in range(4):
        n = len(rp) - 1
        if n == 0:
            break
        assert distinct_candidates(rp, col, np.arange(n, dtype=np.int32))
        C = oracle.vertex_following(rp, col)
        assert distinct_candidates(rp, col, C)
        # one level of moves from singletons, then the induced graph of that partition
        Cn, moved = oracle.sweep(rp, col, w, np.arange(n, dtype=np.int32))
        if moved == 0:
            break
        new_id, _ = oracle.renumber(Cn)
        rp, col, w = oracle.coarsen(rp, col, w, new_id[Cn])
        for a in range(len(rp) - 1):  # induced rows list every column once
            assert np.all(np.diff(col[rp[a]:rp[a + 1]]) > 0)


def test_repeated_column_breaks_the_property():
    """Vertices 0 and 1 joined by two entries of weight 2 each (a split weight 4), vertex 2 a
    leaf of 0.  Vertex 0's community appears twice among row 1's candidates, and scoring the
    entries one by one changes the decision: with 2W = 10, deg(0) = 5 and delta_1 = 4 a single
    entry gives 10*2 - 4*5 = 0 (no move), the merged weight 10*4 - 4*5 = 20 (move).  The
    library therefore takes the table kernels for rows whose columns do not strictly
    increase."""
    rp = np.array([0, 3, 5, 6], np.int64)
    col = np.array([1, 1, 2, 0, 0, 0], np.int32)
    w = np.array([2, 2, 1, 2, 2, 1], np.int64)
    singletons = np.arange(3, dtype=np.int32)
    assert not distinct_candidates(rp, col, singletons)
    tw, deg0, delta1 = int(w.sum()), 5, 4
    assert tw * 2 - delta1 * deg0 == 0 and tw * 4 - delta1 * deg0 == 20
    Cn, _ = oracle.sweep(rp, col, w, singletons)
    assert Cn[1] == 0
