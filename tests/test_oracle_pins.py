"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks one oracle function against something other than itself:
closed forms, an independent library (networkx), a different formula of the same
quantity (pairwise form of Eq. 3, dense P^T A P coarsening), brute force over all
partitions, and hand-worked traces of the Sec. 3.1 rules (tests/golden).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def dense(g):
    """Dense adjacency with loops stored once on the diagonal (Sec. 2 graph model)."""
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for i in range(g.n):
        for t in range(g.rp[i], g.rp[i + 1]):
            A[i, g.col[t]] = g.w[t]
    return A


def rand_partition(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, max(1, k), size=n).astype(np.int32)


# ---------------------------------------------------------------- Eq. 3 ----

@pytest.mark.parametrize("seed", range(12))
def test_modularity_matches_networkx(seed):
    """Eq. 3 against networkx's weighted modularity on loop-free graphs."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.community import modularity as nx_mod
    g = gg.erdos_renyi(18, 0.3, seed, wmax=7, loops=0.0)
    if g.nnz == 0:
        pytest.skip("empty graph")
    C = rand_partition(g.n, 4, seed)
    qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), C)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for i in range(g.n):
        for t in range(g.rp[i], g.rp[i + 1]):
            j = int(g.col[t])
            if j > i:
                G.add_edge(i, j, weight=int(g.w[t]))
    comms = [set(np.flatnonzero(C == c).tolist()) for c in np.unique(C)]
    assert tw == 2 * sum(d["weight"] for _, _, d in G.edges(data=True))
    assert abs(qn / tw ** 2 - nx_mod(G, comms, weight="weight")) < 1e-12


@pytest.mark.parametrize("seed", range(12))
def test_modularity_pairwise_form(seed):
    """Eq. 3 equals the pairwise form (1/2W) sum_ij [A_ij - d_i d_j / 2W] [c_i = c_j]
    (loops included once on the diagonal)."""
    g = gg.erdos_renyi(15, 0.35, 100 + seed, wmax=9, loops=0.3)
    C = rand_partition(g.n, 5, seed)
    qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), C)
    A = dense(g)
    d = A.sum(axis=1)
    same = (C[:, None] == C[None, :])
    expected = tw * int((A * same).sum()) - int((np.outer(d, d) * same).sum())
    assert tw == int(d.sum())
    assert qn == expected


@pytest.mark.parametrize("k,m,w", [(1, 3, 1), (2, 4, 3), (3, 5, 2), (6, 6, 4), (10, 3, 1)])
def test_modularity_disjoint_cliques_closed_form(k, m, w):
    """k disjoint equal cliques, each its own community: Q = 1 - 1/k exactly."""
    g = gg.disjoint_cliques(k, m, w)
    C = np.repeat(np.arange(k), m).astype(np.int32)
    qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), C)
    assert Fraction(qn, tw * tw) == 1 - Fraction(1, k)


@pytest.mark.parametrize("seed", range(6))
def test_modularity_singletons_closed_form(seed):
    """All singletons: Q = (sum of loops)/2W - sum_i (d_i/2W)^2."""
    g = gg.erdos_renyi(20, 0.25, 200 + seed, wmax=5, loops=0.4)
    C = np.arange(g.n, dtype=np.int32)
    qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), C)
    A = dense(g)
    d = A.sum(axis=1)
    assert qn == tw * int(np.trace(A)) - int((d * d).sum())


# ---------------------------------------------------------------- Eq. 4 ----

@pytest.mark.parametrize("seed", range(10))
def test_gain_is_half_modularity_difference(seed):
    """G_b - G_stay == (Qn(after move) - Qn(before)) / 2 for every vertex and every target
    community, including non-neighbouring and empty ones (Eq. 3 vs Eq. 4)."""
    g = gg.erdos_renyi(14, 0.35, 300 + seed, wmax=6, loops=0.3)
    w = g.w.astype(np.int64)
    C = rand_partition(g.n, 5, seed)
    q0, _ = oracle.modularity(g.rp, g.col, w, C)
    for i in range(g.n):
        for b in range(g.n):
            if b == C[i]:
                continue
            C2 = C.copy()
            C2[i] = b
            q1, _ = oracle.modularity(g.rp, g.col, w, C2)
            assert 2 * oracle.gain(g.rp, g.col, w, C, i, b) == q1 - q0, (i, b)


# --------------------------------------------------- Sec. 3.1 hand cases ----

def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked_traces(case):
    g = gg.from_edges(case["n"], [tuple(e) for e in case["edges"]])
    w = g.w.astype(np.int64)
    if case["vertex_following"]:
        C = oracle.vertex_following(g.rp, g.col)
    else:
        C = np.arange(g.n, dtype=np.int32)
    qn, tw = oracle.modularity(g.rp, g.col, w, C)
    assert qn == case["qn_init"]
    for labels, moved, qn_after in case["sweeps"]:
        C, mv = oracle.sweep(g.rp, g.col, w, C)
        assert C.tolist() == labels and mv == moved
        assert oracle.modularity(g.rp, g.col, w, C)[0] == qn_after
    r = oracle.louvain(g.rp, g.col, g.w, vertex_following=case["vertex_following"])
    assert len(r.levels) == len(case["levels"])
    for lev, exp in zip(r.levels, case["levels"]):
        assert lev.labels.tolist() == exp["labels"] and lev.qn == exp["qn"]
    lev0 = [t for t in r.trace if t[0] == 0]
    assert [(t[2], t[3]) for t in lev0] == [(s[1], s[2]) for s in case["sweeps"]]


def test_vertex_following_rules():
    # path 0-1-2-3: ends follow their neighbours (degree 2), middle vertices stay
    g = gg.path(4)
    assert oracle.vertex_following(g.rp, g.col).tolist() == [1, 1, 2, 2]
    # a loop does not count as a neighbour; isolated pair with loops
    g = gg.from_edges(3, [(0, 0, 2), (0, 1, 1), (2, 2, 1)])
    assert oracle.vertex_following(g.rp, g.col).tolist() == [0, 0, 2]
    # star: leaves join the centre
    g = gg.star(3)
    assert oracle.vertex_following(g.rp, g.col).tolist() == [0, 0, 0, 0]


def test_singlet_rule_blocks_swap():
    """Without the singlet rule two singletons would swap labels forever (Sec. 3.1.1)."""
    g = gg.from_edges(2, [(0, 1, 3)])
    C, moved = oracle.sweep(g.rp, g.col, g.w.astype(np.int64), np.arange(2, dtype=np.int32))
    assert C.tolist() == [0, 0] and moved == 1


# ------------------------------------------------ renumber / coarsen ----

@pytest.mark.parametrize("seed", range(5))
def test_renumber_is_order_preserving_compaction(seed):
    C = rand_partition(50, 17, seed)
    new_id, k = oracle.renumber(C)
    uniq, inv = np.unique(C, return_inverse=True)
    assert k == len(uniq)
    assert np.array_equal(new_id[C], inv)


@pytest.mark.parametrize("seed", range(10))
def test_coarsen_equals_dense_projection(seed):
    """A' = P^T A P with P the membership matrix (Sec. 3: loops get intra weight)."""
    g = gg.erdos_renyi(16, 0.3, 400 + seed, wmax=8, loops=0.3)
    C = rand_partition(g.n, 6, seed)
    rp2, col2, w2 = oracle.coarsen(g.rp, g.col, g.w.astype(np.int64), C)
    uniq, inv = np.unique(C, return_inverse=True)
    P = np.zeros((g.n, len(uniq)), np.int64)
    P[np.arange(g.n), inv] = 1
    expected = P.T @ dense(g) @ P
    k = len(uniq)
    got = np.zeros((k, k), np.int64)
    for a in range(k):
        cols = col2[rp2[a]:rp2[a + 1]]
        assert np.all(np.diff(cols) > 0)
        got[a, cols] = w2[rp2[a]:rp2[a + 1]]
    assert np.array_equal(got, expected)


# ----------------------------------------------------------- threshold ----

def test_threshold_exact_against_fractions():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        tw = int(rng.integers(1, 1 << 62)) if rng.random() < 0.5 else int(rng.integers(1, 1000))
        a = int(rng.integers(-(1 << 62), 1 << 62)) * int(rng.integers(1, 1 << 60))
        a = max(min(a, tw * tw), -tw * tw)
        b = a - int(rng.integers(-5, 5)) * (tw * tw // 1_000_000 + int(rng.integers(0, 3)))
        b = max(min(b, tw * tw), -tw * tw)
        num, den = int(rng.integers(0, 10)), int(rng.integers(1, 10_000_000))
        expect = (a - b) * den < num * tw * tw
        assert oracle.below_threshold(a, b, tw, num, den) == expect


# -------------------------------------------------------- whole runs ----

def _all_partitions_qn(g):
    """Max Qn over every partition of the vertex set (restricted growth strings)."""
    n = g.n
    rgs = np.zeros((1, 1), np.int8)
    for pos in range(1, n):
        mx = rgs.max(axis=1)
        reps = (mx + 2).astype(np.int64)
        base = np.repeat(rgs, reps, axis=0)
        nxt = np.concatenate([np.arange(r, dtype=np.int8) for r in reps])
        rgs = np.concatenate([base, nxt[:, None]], axis=1)
    A = dense(g)
    d = A.sum(axis=1)
    tw = int(d.sum())
    inner = np.zeros(len(rgs), np.int64)
    for i in range(n):
        for j in range(n):
            if A[i, j]:
                inner += A[i, j] * (rgs[:, i] == rgs[:, j])
    sq = np.zeros(len(rgs), np.int64)
    for c in range(n):
        dc = ((rgs == c) * d[None, :]).sum(axis=1)
        sq += dc * dc
    return int((tw * inner - sq).max())


@pytest.mark.parametrize("seed", range(8))
def test_louvain_never_beats_brute_force_optimum(seed):
    n = 9 if seed < 6 else 11
    g = gg.erdos_renyi(n, 0.35, 500 + seed, wmax=4, loops=0.1)
    if g.nnz == 0:
        pytest.skip("empty graph")
    r = oracle.louvain(g.rp, g.col, g.w)
    best = _all_partitions_qn(g)
    for lev in r.levels:
        qn, _ = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), lev.labels)
        assert qn == lev.qn
        assert lev.qn <= best


def test_planted_cliques_recovered():
    """6 cliques of 6 (intra weight 4) in a ring of weight-1 bridges."""
    k, m = 6, 6
    g = gg.cliques_ring(k, m, 4, 1)
    truth = np.repeat(np.arange(k), m)
    r = oracle.louvain(g.rp, g.col, g.w)
    found = [np.array_equal(np.unique(l.labels, return_inverse=True)[1], truth) for l in r.levels]
    assert any(found)
    assert found[-1], "clique partition must not be merged later"
    qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), truth.astype(np.int32))
    assert r.levels[-1].qn == qn


@pytest.mark.parametrize("seed", range(10))
def test_levels_preserve_tw_and_q_theorem1(seed):
    """Theorem 1 (N and nnz never grow), TW preserved by coarsening, and the Q of a level's
    partition equals the Q of the singleton partition on the next level's graph."""
    g = gg.random_small(600 + seed, n_max=60)
    if g.nnz == 0:
        return
    r = oracle.louvain(g.rp, g.col, g.w, vertex_following=bool(seed % 2))
    for a, b in zip(r.levels, r.levels[1:]):
        assert b.n <= a.n and b.nnz <= a.nnz
        assert b.n == a.ncomm
        assert b.qn_init == a.qn
    for lev in r.levels:
        qn, tw = oracle.modularity(g.rp, g.col, g.w.astype(np.int64), lev.labels)
        assert tw == r.tw and qn == lev.qn
        assert lev.ncomm == len(np.unique(lev.labels))
        assert lev.labels.min() == 0 and lev.labels.max() == lev.ncomm - 1


@pytest.mark.parametrize("seed", range(10))
def test_fixed_point_is_locally_optimal(seed):
    """When a level ends because no vertex moved, every single-vertex move to a
    neighbouring community has gain <= 0 or is a vetoed singlet move (Eq. 4, Sec. 3.1)."""
    g = gg.random_small(700 + seed, n_max=30)
    if g.nnz == 0:
        return
    r = oracle.louvain(g.rp, g.col, g.w, vertex_following=False, max_levels=1)
    if not r.levels or r.trace[-1][2] != 0:
        return
    C = r.levels[0].labels
    w = g.w.astype(np.int64)
    size = np.bincount(C, minlength=g.n)
    for i in range(g.n):
        nb = {int(C[j]) for j in g.col[g.rp[i]:g.rp[i + 1]] if j != i}
        for b in nb - {int(C[i])}:
            gain = oracle.gain(g.rp, g.col, w, C, i, b)
            vetoed = size[C[i]] == 1 and size[b] == 1 and b > C[i]
            assert gain <= 0 or vetoed


def test_trivial_inputs():
    # no vertices, no edges, isolated vertices, a lone loop
    for g in [gg.from_edges(0, []), gg.from_edges(5, []), gg.from_edges(1, [(0, 0, 3)])]:
        r = oracle.louvain(g.rp, g.col, g.w)
        assert r.levels == []
        assert r.trace == ([] if g.n == 0 else [(0, 1, 0, r.trace[0][3])])


def test_invalid_inputs_rejected():
    g = gg.path(3)
    with pytest.raises(oracle.OracleError):
        oracle.louvain(g.rp, np.array([0, 5, 1, 1], np.int32), g.w)
    with pytest.raises(oracle.OracleError):
        oracle.louvain(g.rp, g.col, np.zeros_like(g.w))


# ------------------------------------------- sweep rule and driver consistency ----

def reference_sweep(g, C):
    """Algorithm 1 body written from the rules, with gains from the pinned oracle.gain:
    candidates are the communities of non-loop neighbours other than C(i); target = argmax
    gain, ties to the smaller label (Sec. 3.1.2); move iff gain > 0 (strict) unless both
    communities are singletons and target > C(i) (Sec. 3.1.1)."""
    w = g.w.astype(np.int64)
    size = np.bincount(C, minlength=g.n)
    out = C.copy()
    for i in range(g.n):
        cands = sorted({int(C[j]) for j in g.col[g.rp[i]:g.rp[i + 1]] if j != i} - {int(C[i])})
        best, best_gain = None, None
        for b in cands:
            gain = oracle.gain(g.rp, g.col, w, C, i, b)
            if best is None or gain > best_gain:
                best, best_gain = b, gain
        if best is None or best_gain <= 0:
            continue
        if size[C[i]] == 1 and size[best] == 1 and best > C[i]:
            continue
        out[i] = best
    return out


@pytest.mark.parametrize("seed", range(12))
def test_sweep_matches_reference_rule(seed):
    g = gg.random_small(800 + seed, n_max=40)
    rng = np.random.default_rng(seed)
    for trial in range(3):
        C = rng.integers(0, max(1, g.n), size=g.n).astype(np.int32) if trial else \
            np.arange(g.n, dtype=np.int32)
        Cn, moved = oracle.sweep(g.rp, g.col, g.w.astype(np.int64), C)
        ref = reference_sweep(g, C)
        assert np.array_equal(Cn, ref)
        assert moved == int((ref != C).sum())


@pytest.mark.parametrize("seed,kind", [(s, k) for s in range(4) for k in ("small", "rmat")])
def test_run_trace_equals_repeated_sweeps(seed, kind):
    """The multi-sweep driver must equal single sweeps applied one after another, each
    followed by Eq. 3; this is the phase loop of Algorithm 1 with the stopping rule."""
    if kind == "small":
        g = gg.random_small(900 + seed, n_max=60)
    else:
        g = gg.rmat(9 + seed % 3, 8, seed=seed)
    vf = bool(seed % 2)
    r = oracle.louvain(g.rp, g.col, g.w, max_levels=1, vertex_following=vf)
    w = g.w.astype(np.int64)
    C = oracle.vertex_following(g.rp, g.col) if vf else np.arange(g.n, dtype=np.int32)
    qn_prev, tw = oracle.modularity(g.rp, g.col, w, C)
    trace = []
    for it in range(1, 1001):
        C, moved = oracle.sweep(g.rp, g.col, w, C)
        qn, _ = oracle.modularity(g.rp, g.col, w, C)
        trace.append((0, it, moved, qn))
        if moved == 0 or (qn - qn_prev) * 1_000_000 < tw * tw:
            break
        qn_prev = qn
    assert r.trace == trace
    if r.levels:
        new_id, _ = oracle.renumber(C)
        assert np.array_equal(r.levels[0].labels, new_id[C])


@pytest.mark.parametrize("seed,theta", [(s, t) for s in range(4) for t in ((1, 100), (1, 10_000))])
def test_relative_threshold_trace(seed, theta):
    """Relative phase test of Algorithm 1 (threshold_mode 1): the phase stops at the first
    sweep with |Q_curr - Q_prev| / |Q_prev| < theta, evaluated here with exact fractions on
    repeated single sweeps, or when nothing moved; Q_prev starts at the initial state's Q."""
    from fractions import Fraction
    g = gg.rmat(9 + seed % 2, 8, seed=40 + seed) if seed % 2 else \
        gg.sbm(400, 40, 0.2, 0.01, 1, 4, seed=seed)
    r = oracle.louvain(g.rp, g.col, g.w, max_levels=1, theta=theta, threshold_mode=1)
    w = g.w.astype(np.int64)
    C = oracle.vertex_following(g.rp, g.col)
    qn_prev, tw = oracle.modularity(g.rp, g.col, w, C)
    th = Fraction(theta[0], theta[1])
    trace = []
    for it in range(1, 1001):
        C, moved = oracle.sweep(g.rp, g.col, w, C)
        qn, _ = oracle.modularity(g.rp, g.col, w, C)
        trace.append((0, it, moved, qn))
        if moved == 0:
            break
        if qn_prev == 0:
            if qn == 0:
                break
        elif abs(Fraction(qn - qn_prev, qn_prev)) < th:
            break
        qn_prev = qn
    assert r.trace == trace
    # the absolute and the relative test are different rules: at least one case differs
    a = oracle.louvain(g.rp, g.col, g.w, max_levels=1, theta=theta)
    assert a.trace[0] == r.trace[0]


def test_relative_threshold_differs_from_absolute():
    g = gg.sbm(600, 30, 0.3, 0.01, 1, 4, seed=5)
    diffs = 0
    for theta in ((1, 10), (1, 100), (1, 1000)):
        a = oracle.louvain(g.rp, g.col, g.w, theta=theta)
        r = oracle.louvain(g.rp, g.col, g.w, theta=theta, threshold_mode=1)
        diffs += a.trace != r.trace
    assert diffs > 0
    with pytest.raises(oracle.OracleError):
        oracle.louvain(g.rp, g.col, g.w, threshold_mode=2)


def test_post_merge_hand_cases():
    """Post-phase merge (Sec. 5.1.2, reading R15), worked by hand with vertex following off
    and one sweep per phase.

    Path 0-1-2, unit weights (2W = 4, delta = 1, 2, 1): from singletons vertex 0 is vetoed
    (target 1 > 0, both singletons), 1 joins 0 (gains to 0 and 2 tie at 2, smaller label),
    2 joins 1, so the phase ends with (0, 0, 1), Qn = 4*2 - (3^2 + 1^2) = -2.  Vertex 2's
    only neighbour community is {0, 1} with gain 4*1 - 1*3 = 1 > 0 (staying: 0), so the
    merge moves it: one community, Qn = 4*4 - 4^2 = 0.

    An isolated pair with loops of weight 10 (2W = 22, delta = 11 each) never merges: the
    move's gain 22*1 - 11*11 is negative, in the phase and in the merge."""
    g = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
    plain = oracle.louvain(g.rp, g.col, g.w, vertex_following=False, max_iters=1, max_levels=1)
    merged = oracle.louvain(g.rp, g.col, g.w, vertex_following=False, max_iters=1, max_levels=1,
                            post_merge=True)
    assert list(plain.levels[0].labels) == [0, 0, 1] and plain.levels[0].qn == -2
    assert list(merged.levels[0].labels) == [0, 0, 0] and merged.levels[0].qn == 0
    assert merged.levels[0].ncomm == 1 and merged.trace == plain.trace
    pair = gg.from_edges(2, [(0, 1, 1), (0, 0, 10), (1, 1, 10)])
    for pm in (False, True):
        r = oracle.louvain(pair.rp, pair.col, pair.w, vertex_following=False, post_merge=pm)
        assert r.levels == [] and r.trace == [(0, 1, 0, 22 * 20 - 2 * 121)]


@pytest.mark.parametrize("seed", range(6))
def test_post_merge_levels_are_consistent(seed):
    """With the merge, every recorded level's Qn is Eq. 3 of its labels, levels nest, and 2W
    and Theorem 1 hold."""
    g = gg.random_small(5000 + seed, n_max=70) if seed % 2 else gg.rmat(9, 8, seed=seed)
    r = oracle.louvain(g.rp, g.col, g.w, post_merge=True, max_iters=2)
    w = g.w.astype(np.int64)
    prev = None
    for lev in r.levels:
        qn, tw = oracle.modularity(g.rp, g.col, w, lev.labels)
        assert qn == lev.qn and tw == r.tw
        if prev is not None:
            first = np.full(int(prev.max()) + 1, -1, np.int64)
            first[prev] = lev.labels
            assert np.array_equal(first[prev], lev.labels)
        prev = lev.labels
