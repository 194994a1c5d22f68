"""Checkpoint / resume: a run that keeps the graph induced after each level can be resumed
from any of them, and the resumed run must reproduce the uninterrupted run's later levels
exactly (labels through the saved level's labels, Qn, iterations, trace, edge visits)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_1805_10904_gb300 as m
    m.load()
    return m


def sorted_rows(rp, col, w):
    out_c, out_w = col.copy(), w.copy()
    for i in range(len(rp) - 1):
        a, b = rp[i], rp[i + 1]
        o = np.argsort(col[a:b], kind="stable")
        out_c[a:b], out_w[a:b] = col[a:b][o], w[a:b][o]
    return out_c, out_w


def check_resume(lv, g, **kw):
    import torch
    d = [torch.from_numpy(a).cuda() for a in (g.rp, g.col, g.w)]
    full = lv.Louvain(0, keep_coarse=True, **kw).run(*d)
    assert full.num_levels >= 2
    h = lv.Louvain(0, **kw)
    checked = 0
    for s in range(1, full.num_levels + 1):
        cg = full.coarse_graph(s - 1)
        if s == full.num_levels and cg is None:
            break  # the run stopped at its last level (outer test or max_levels)
        assert cg is not None
        rp, col, w = cg
        # the saved graph is the induced graph of the saved labels (rows in any order)
        ref = oracle.coarsen(g.rp, g.col, g.w, full.labels(s - 1)) if s == 1 else None
        if ref is not None:
            c1, w1 = sorted_rows(rp, col, w.astype(np.int64))
            assert np.array_equal(rp, ref[0]) and np.array_equal(c1, ref[1])
            assert np.array_equal(w1, np.asarray(ref[2], np.int64))
        res = h.resume(s, full.level(s - 1).qn, rp, col, w)
        assert res.num_levels == full.num_levels - s
        base = full.labels(s - 1)
        for k in range(res.num_levels):
            assert res.level(k) == full.level(s + k)
            assert np.array_equal(res.labels(k)[base], full.labels(s + k))
        assert res.trace() == [t for t in full.trace() if t[0] >= s]
        checked += 1
    return checked


def test_resume_reproduces_later_levels(lv):
    assert check_resume(lv, gg.rmat(13, 16, seed=13)) >= 1


def test_resume_with_int64_coarse_weights(lv):
    """Community degrees above 2^31 - 1 make the induced graphs carry int64 weights (every
    vertex's weighted degree is near 2^29 here, so a community of four already needs them)."""
    b = gg.sbm(3000, 60, 0.1, 0.004, 1, 4, seed=2)
    heavy = gg.Graph(b.rp, b.col, (b.w.astype(np.int64) * (1 << 24)).astype(np.int32), "heavy")
    import torch
    full = lv.Louvain(0, keep_coarse=True).run(*[torch.from_numpy(a).cuda()
                                                  for a in (heavy.rp, heavy.col, heavy.w)])
    assert full.coarse_graph(0)[2].dtype == np.int64
    check_resume(lv, heavy)


def test_resume_with_variants(lv):
    check_resume(lv, gg.sbm(2048, 64, 0.15, 0.003, 1, 4, seed=5), vf_all_levels=True,
                 post_merge=True, max_levels=4)


def test_no_checkpoint_without_keep_coarse(lv):
    import torch
    g = gg.rmat(11, 16, seed=1)
    r = lv.Louvain(0).run(*[torch.from_numpy(a).cuda() for a in (g.rp, g.col, g.w)])
    assert r.num_levels >= 1 and r.coarse_graph(0) is None
    with pytest.raises(lv.LouvainError):
        lv.Louvain(0).resume(0, 0, g.rp, g.col, g.w)
