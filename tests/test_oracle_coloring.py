"""Pins of the oracle's colouring variant (reading R17: Lu et al.'s colouring heuristic,
which Sec. 7 names among the "other heuristics" of the parallel Louvain it builds on).

- The colouring: its priorities are SplitMix64's output function (checked against the
  generator's published first output for seed 0), the colouring is proper, and the
  Jones-Plassmann rounds give exactly the sequential greedy colouring in decreasing
  priority order (each vertex the smallest colour its higher-priority neighbours left).
- The colour-class schedule: on a complete graph every vertex has a colour of its own, so
  a coloured sweep is sequential local moving in colour order -- restated here as the
  textbook removal-then-insert form (remove v from its community, score each neighbouring
  community, insert into the best), with Sec. 3.1's tie and singlet rules.
- A case worked by hand (the 4-cycle, where synchronous sweeps swap neighbours forever in
  pairs and colouring does not), and whole-run properties: Q never above the brute-force
  optimum, planted cliques recovered, Theorem 1, Q preserved across levels.
"""
from collections import defaultdict
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle

from test_oracle_pins import _all_partitions_qn, dense

M64 = (1 << 64) - 1


def splitmix64_output(v: int) -> int:
    """SplitMix64's output function on state v + golden gamma (Steele, Lea, Flood 2014)."""
    z = (v + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_priority_is_splitmix64():
    # the first output of SplitMix64 seeded with 0 is 0xE220A8397B1DCDAF
    assert splitmix64_output(0) == 0xE220A8397B1DCDAF


def greedy_in_priority_order(g):
    order = sorted(range(g.n), key=lambda v: -splitmix64_output(v))
    color = [-1] * g.n
    for v in order:
        taken = {color[u] for u in g.col[g.rp[v]:g.rp[v + 1]] if u != v and color[u] >= 0}
        c = 0
        while c in taken:
            c += 1
        color[v] = c
    return np.asarray(color, np.int32)


GRAPHS = [gg.random_small(s, n_max=60) for s in range(30)] + [
    gg.rmat(10, 8, seed=3), gg.sbm(500, 25, 0.3, 0.01, 1, 4, seed=2), gg.star(12),
    gg.cliques_ring(5, 5), gg.path(9)]


@pytest.mark.parametrize("k", range(len(GRAPHS)))
def test_coloring_is_proper_greedy_in_priority_order(k):
    g = GRAPHS[k]
    color, ncol = oracle.color(g.rp, g.col)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    off_diag = rows != g.col
    assert not np.any(color[rows[off_diag]] == color[g.col[off_diag]])  # proper
    assert np.array_equal(color, greedy_in_priority_order(g))
    assert ncol == (int(color.max()) + 1 if g.n else 0)


def sequential_level0(g, theta=(1, 1_000_000), max_iters=1000):
    """Sequential local moving in decreasing priority order, textbook form: v leaves its
    community a, every neighbouring community c scores 2W * k_{v,c} - delta_v * deg(c)
    (loop left out of k_{v,c}; deg without v), v joins the best-scoring c (ties to the
    smallest label) if it beats returning to a, unless v was a singleton and c is a
    singleton with a larger label.  Stops when nothing moved or the Eq. 3 gain of a sweep
    is below theta.  Returns (labels, [(moved, Qn)] per sweep)."""
    A = dense(g)
    n = g.n
    delta = A.sum(axis=1).astype(object)
    tw = int(sum(delta))
    order = sorted(range(n), key=lambda v: -splitmix64_output(v))
    C = list(range(n))
    deg = defaultdict(int, {c: int(delta[c]) for c in range(n)})
    size = defaultdict(int, {c: 1 for c in range(n)})

    def qn():
        inner = sum(int(A[i, j]) for i in range(n) for j in range(n) if C[i] == C[j])
        return tw * inner - sum(d * d for d in deg.values())

    trace, q_prev = [], qn()
    for _ in range(max_iters):
        moved = 0
        for v in order:
            a = C[v]
            was_single = size[a] == 1
            deg[a] -= int(delta[v])
            size[a] -= 1
            k = defaultdict(int)
            for u in range(n):
                if u != v and A[v, u]:
                    k[C[u]] += int(A[v, u])
            score = {c: tw * k[c] - int(delta[v]) * deg[c] for c in k}
            stay = tw * k.get(a, 0) - int(delta[v]) * deg[a]
            others = sorted((c for c in k if c != a), key=lambda c: (-score[c], c))
            target = a
            if others and score[others[0]] > stay:
                b = others[0]
                if not (was_single and size[b] == 1 and b > a):
                    target = b
            C[v] = target
            deg[target] += int(delta[v])
            size[target] += 1
            moved += target != a
        q = qn()
        trace.append((moved, q))
        if moved == 0 or Fraction(q - q_prev, tw * tw) < Fraction(*theta):
            break
        q_prev = q
    return np.unique(np.asarray(C), return_inverse=True)[1].astype(np.int32), trace


@pytest.mark.parametrize("seed", range(12))
def test_one_vertex_per_class_is_sequential_local_moving(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 10))
    edges = [(i, j, int(rng.integers(1, 10))) for i in range(n) for j in range(i + 1, n)]
    edges += [(i, i, int(rng.integers(1, 6))) for i in range(n) if rng.random() < 0.3]
    g = gg.from_edges(n, edges)
    color, ncol = oracle.color(g.rp, g.col)
    assert ncol == n  # complete graph: one class per vertex
    theta = (1, 1000) if seed % 2 else (1, 1_000_000)
    labels, trace = sequential_level0(g, theta)
    r = oracle.louvain(g.rp, g.col, g.w, theta=theta, max_levels=1, vertex_following=False,
                       coloring=True)
    assert [(m, q) for _, _, m, q in r.trace] == trace
    if r.levels:
        assert np.array_equal(r.levels[0].labels, labels)
    else:
        assert len(np.unique(labels)) == n


def test_four_cycle_by_hand():
    """C4: 0-1-2-3-0, unit weights, 2W = 8, delta = 2, no vertex following.
    Priorities put 0 before 2 before 1 before 3, so rounds colour {0, 2} with 0 and {1, 3}
    with 1.  Sweep 1, class 0 on singletons: vertex 0 ties G_1 = G_3 = 8 - 4 = 4 > 0, takes
    1 and is vetoed (singletons, 1 > 0); vertex 2 takes 1 (4 > 0, 1 < 2).  Class 1 on
    [0, 1, 1, 3], deg = (2, 4, -, 2): vertex 1 has G_0 = 8 - 4 = 4, G_stay = 8 - 2 * 2 = 4,
    not strictly better, stays; vertex 3 has G_0 = 4 > G_1 = 0 and G_stay = 0, joins 0.
    State [0, 1, 1, 0]: Qn = 8 * 4 - (16 + 16) = 0 from Qn_init = -16.  Sweep 2 moves
    nobody (every G_other = 0 < G_stay = 4).  Level 1 (two vertices, loops 2, link 2,
    delta 4) moves nobody: one level.  Synchronous sweeps instead swap to [0, 1, 0, 1]."""
    g = gg.from_edges(4, [(0, 1, 1), (1, 2, 1), (2, 3, 1), (3, 0, 1)])
    color, ncol = oracle.color(g.rp, g.col)
    assert color.tolist() == [0, 1, 0, 1] and ncol == 2
    r = oracle.louvain(g.rp, g.col, g.w, vertex_following=False, coloring=True)
    assert len(r.levels) == 1
    lev = r.levels[0]
    assert lev.labels.tolist() == [0, 1, 1, 0]
    assert (lev.qn, lev.qn_init, lev.iters) == (0, -16, 2)
    assert r.trace == [(0, 1, 2, 0), (0, 2, 0, 0), (1, 1, 0, 0)]
    s = oracle.louvain(g.rp, g.col, g.w, vertex_following=False)
    assert s.levels[0].labels.tolist() == [0, 1, 0, 1]


@pytest.mark.parametrize("seed", range(6))
def test_coloring_never_beats_brute_force(seed):
    g = gg.erdos_renyi(9, 0.35, 900 + seed, wmax=4, loops=0.1)
    if g.nnz == 0:
        pytest.skip("empty graph")
    best = _all_partitions_qn(g)
    r = oracle.louvain(g.rp, g.col, g.w, coloring=True)
    for lev in r.levels:
        qn, _ = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), lev.labels)
        assert qn == lev.qn <= best


def test_coloring_recovers_planted_cliques():
    k, m = 6, 6
    g = gg.cliques_ring(k, m, 4, 1)
    truth = np.repeat(np.arange(k), m)
    r = oracle.louvain(g.rp, g.col, g.w, coloring=True)
    found = [np.array_equal(np.unique(l.labels, return_inverse=True)[1], truth) for l in r.levels]
    assert any(found) and found[-1]


@pytest.mark.parametrize("seed", range(10))
def test_coloring_levels_theorem1_and_q(seed):
    g = gg.random_small(1600 + seed, n_max=60)
    if g.nnz == 0:
        return
    r = oracle.louvain(g.rp, g.col, g.w, coloring=True, vf_all_levels=bool(seed % 2))
    for a, b in zip(r.levels, r.levels[1:]):
        assert b.n == a.ncomm <= a.n and b.nnz <= a.nnz
    for lev in r.levels:
        qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), lev.labels)
        assert tw == r.tw and qn == lev.qn
