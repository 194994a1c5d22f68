"""Pin of the oracle's outer stopping rule (Algorithm 2, reading R9).

Algorithm 2 repeats phases on the induced graph and stops once a level's modularity gain
falls below the threshold.  Reading R9 fixes the details: a level is recorded when its
phase merged something; from the second level on, the run stops after a level whose Qn
grew by less than theta * (2W)^2 over the previous recorded level (that level stays
recorded).

The expected list of levels is built here independently of the oracle's driver: one
single-level oracle run per level on the graph induced so far (vertex following at level 0,
or at every level when asked), labels composed back to the input vertices here, each
level's Qn checked against Eq. 3 recomputed with numpy integers, and the stopping rule
applied with exact fractions.  The cases are chosen so that the outer stop fires before
the levels run out, and so that two plausible mistakes -- comparing against the level's
own starting Qn instead of the previous level's Qn, or applying the test at level 0 too --
each give a different level list on at least one case.
"""
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle


def _qn_numpy(g, labels):
    """Eq. 3 times (2W)^2 from labels of the input vertices, with numpy integer sums."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rp))
    w = g.w.astype(np.int64)
    internal = int(w[labels[rows] == labels[g.col]].sum())
    dvert = np.zeros(g.n, np.int64)
    np.add.at(dvert, rows, w)
    dcomm = np.zeros(int(labels.max()) + 1, np.int64)
    np.add.at(dcomm, labels, dvert)
    tw = int(dvert.sum())
    return tw * internal - sum(int(x) * int(x) for x in dcomm), tw


def _stars(groups=4, stars=3, leaves=5, hub_w=20, bridge_w=1):
    """Stars whose hubs form heavy cliques per group, groups joined in a ring: vertex
    following settles the leaves before the first sweep, so level 0 gains almost nothing
    over its starting state while level 1 still merges the groups."""
    edges, n, hubs = [], 0, []
    for _ in range(groups):
        gh = []
        for _ in range(stars):
            h = n
            n += 1
            gh.append(h)
            for _ in range(leaves):
                edges.append((h, n, 1))
                n += 1
        edges += [(gh[a], gh[b], hub_w) for a in range(len(gh)) for b in range(a + 1, len(gh))]
        hubs.append(gh)
    edges += [(hubs[k][0], hubs[(k + 1) % groups][-1], bridge_w) for k in range(groups)]
    return gg.from_edges(n, edges, "stars")


def _levels_one_at_a_time(g, theta, vf_all):
    """Every level the phases reach (no outer stop): (composed labels, Qn, Qn at the
    level's start) per level, from single-level oracle runs on the induced graphs."""
    rp, col, w = g.rp, g.col, g.w.astype(np.int64)
    composed = np.arange(g.n, dtype=np.int32)
    out = []
    for level in range(64):
        r = oracle.louvain(rp, col, w, theta=theta, max_levels=1,
                           vertex_following=(level == 0 or vf_all))
        if not r.levels:  # nothing merged: no new level
            break
        lab = r.levels[0].labels
        composed = lab[composed]
        qn, tw = _qn_numpy(g, composed)
        assert qn == r.levels[0].qn  # Eq. 3 on the input graph equals the level's Qn
        out.append((composed.copy(), qn, r.levels[0].qn_init))
        rp, col, w = oracle.coarsen(rp, col, w, lab)
    return out, int(g.w.astype(np.int64).sum())


def _stop(levels, tw, theta, rule):
    """Number of recorded levels under a stopping rule, applied with exact fractions."""
    th = Fraction(theta[0], theta[1])
    for l, (_, qn, qn_start) in enumerate(levels):
        if rule == "paper":
            stop = l >= 1 and Fraction(qn - levels[l - 1][1], tw * tw) < th
        elif rule == "against_level_start":
            stop = l >= 1 and Fraction(qn - qn_start, tw * tw) < th
        else:  # "from_level_0": the test also at level 0, against its starting state
            ref = qn_start if l == 0 else levels[l - 1][1]
            stop = Fraction(qn - ref, tw * tw) < th
        if stop:
            return l + 1
    return len(levels)


# (name, graph, vertex following at every level, theta); in every case but "stars" the
# outer stop fires before the levels run out ("stars" ends because level 1 merges all)
CASES = [
    ("random_small_16", lambda: gg.random_small(16, n_max=60), True, (1, 30)),
    ("random_small_31", lambda: gg.random_small(31, n_max=60), True, (1, 1000)),
    ("random_small_19", lambda: gg.random_small(19, n_max=60), True, (1, 100)),
    ("random_small_12", lambda: gg.random_small(12, n_max=60), False, (1, 10)),
    ("stars", _stars, False, (1, 10)),
    ("rmat12", lambda: gg.rmat(12, 16, seed=12), False, (1, 100)),
]
RUN_OUT = {"stars"}


@pytest.fixture(scope="module")
def outcomes():
    res = {}
    for name, build, vf_all, theta in CASES:
        g = build()
        levels, tw = _levels_one_at_a_time(g, theta, vf_all)
        res[name] = (g, vf_all, theta, levels,
                     {rule: _stop(levels, tw, theta, rule)
                      for rule in ("paper", "against_level_start", "from_level_0")})
    return res


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_outer_stop_matches_algorithm_2(outcomes, name):
    g, vf_all, theta, levels, stops = outcomes[name]
    expect = stops["paper"]
    if name not in RUN_OUT:
        assert expect < len(levels), "the outer stop must fire before the levels run out"
    r = oracle.louvain(g.rp, g.col, g.w, theta=theta, vf_all_levels=vf_all)
    assert len(r.levels) == expect
    for l in range(expect):
        assert np.array_equal(r.levels[l].labels, levels[l][0])
        assert r.levels[l].qn == levels[l][1]


def test_cases_tell_the_rules_apart(outcomes):
    """Each plausible mistake changes the level list of at least one case."""
    for wrong in ("against_level_start", "from_level_0"):
        assert any(s[wrong] != s["paper"] for *_, s in outcomes.values()), wrong
