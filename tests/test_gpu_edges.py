"""louvain_csr_from_edges: the symmetric CSR of an undirected edge list built on the GPU
(Sec. 5.1.2 neighbour computation), compared entry for entry with its plain definition
written in numpy: both directions of every non-loop edge, a loop once, equal (row, column)
entries merged by adding weights, rows sorted by column."""
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


def reference_csr(n, u, v, w):
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    w = np.ones(len(u), np.int64) if w is None else np.asarray(w, np.int64)
    loop = u == v
    rows = np.concatenate([u, v[~loop]])
    cols = np.concatenate([v, u[~loop]])
    ws = np.concatenate([w, w[~loop]])
    keys = rows * n + cols
    uk, inv = np.unique(keys, return_inverse=True)
    wsum = np.bincount(inv, weights=ws, minlength=len(uk)).astype(np.int64)
    r = uk // n
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return np.cumsum(rp), (uk % n).astype(np.int32), wsum.astype(np.int32)


def check(lv, torch, n, u, v, w, device):
    h = lv.Louvain(0)
    if device:
        d = torch.device("cuda:0")
        args = [torch.from_numpy(np.asarray(x, np.int32)).to(d) if x is not None else None
                for x in (u, v, w)]
    else:
        args = [None if x is None else np.asarray(x, np.int32) for x in (u, v, w)]
    rp, col, ww = h.csr_from_edges(n, *args)
    erp, ecol, ew = reference_csr(n, u, v, w)
    assert np.array_equal(rp.cpu().numpy(), erp)
    assert np.array_equal(col.cpu().numpy(), ecol)
    assert np.array_equal(ww.cpu().numpy(), ew)
    return rp, col, ww


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("device", [True, False])
def test_random_edge_lists(torch, lv, seed, device):
    rng = np.random.default_rng(seed)
    n = [1, 7, 1024, 5000, 65537, 300000][seed]
    m = [3, 40, 9000, 30000, 200000, 1000000][seed]
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    dup = rng.integers(0, m, m // 5)   # repeated edges, half of them reversed
    u = np.concatenate([u, u[dup[::2]], v[dup[1::2]]])
    v = np.concatenate([v, v[dup[::2]], u[dup[1::2]]])
    w = rng.integers(1, 17, len(u)) if seed % 2 == 0 else None
    check(lv, torch, n, u, v, w, device)


def test_rmat_edge_list_rebuilds_its_csr_and_runs(torch, lv):
    """The upper triangle of a generated CSR, shuffled, gives back exactly that CSR, and
    Louvain on it is the oracle's run."""
    g = gg.rmat(16, 16, seed=16)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    keep = rows <= g.col
    rng = np.random.default_rng(1)
    perm = rng.permutation(int(keep.sum()))
    u, v, w = rows[keep][perm], g.col[keep][perm], g.w[keep][perm]
    flip = rng.random(len(u)) < 0.5
    u, v = np.where(flip, v, u), np.where(flip, u, v)
    rp, col, ww = check(lv, torch, g.n, u, v, w, True)
    assert np.array_equal(rp.cpu().numpy(), g.rp) and np.array_equal(col.cpu().numpy(), g.col)
    res = lv.Louvain(0).run(rp, col, ww)
    ref = oracle.louvain(g.rp, g.col, g.w)
    assert res.num_levels == len(ref.levels)
    for l, rl in enumerate(ref.levels):
        assert np.array_equal(res.labels(l), rl.labels) and res.level(l).qn == rl.qn


def test_edge_cases_and_errors(torch, lv):
    h = lv.Louvain(0)
    # no edges; isolated vertices; a single loop counted once
    check(lv, torch, 5, [], [], None, False)
    check(lv, torch, 3, [2, 2], [2, 2], [4, 5], True)
    with pytest.raises(lv.LouvainError) as e:
        h.csr_from_edges(4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    assert e.value.code == lv.louvain.ERR_INDEX_RANGE
    with pytest.raises(lv.LouvainError) as e:
        h.csr_from_edges(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                         np.array([3, 0], np.int32))
    assert e.value.code == lv.louvain.ERR_BAD_WEIGHT
    big = np.array([2 ** 30 + 1, 2 ** 30 + 1], np.int32)  # merged: above 2^31 - 1
    with pytest.raises(lv.LouvainError) as e:
        h.csr_from_edges(3, np.array([0, 1], np.int32), np.array([1, 0], np.int32), big)
    assert e.value.code == lv.louvain.ERR_TOO_LARGE
    check(lv, torch, 3, [0, 1], [1, 2], [5, 7], True)  # the handle stays usable
