"""louvain_modularity_noalloc: modularity without device allocation, for callers that
cannot allocate GPU memory while they run (memory reserved up front by another framework,
or code that must avoid the synchronisation of cudaMalloc/cudaFree).

The entry point is called through the C ABI twice in a row on the same device; both calls
must reproduce, exactly, the modularity that louvain_run reports for each recorded level
(so the second call proves the shared scratch array is cleared between calls), and the
oracle's Eq. 3 on random partitions that leave labels unused, with and without weights.
A call after the first one on a device must leave the device's free memory unchanged.
Kept in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

Q_RTOL = 1e-12


def _noalloc(lib):
    f = lib.louvain_modularity_noalloc
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P]
    f.restype = ctypes.c_int
    return f


def _call(f, torch, n, rp, col, w, labels_dev):
    qn = np.zeros(2, np.int64)
    tw = ctypes.c_int64()
    q = ctypes.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(n, rp.data_ptr(), col.data_ptr(), None if w is None else w.data_ptr(),
           labels_dev.data_ptr(), ctypes.c_void_p(stream), qn.ctypes.data,
           ctypes.addressof(tw), ctypes.addressof(q))
    value = (int(qn[0]) << 64) | (int(qn[1]) & 0xFFFFFFFFFFFFFFFF)
    return rc, value, tw.value, q.value


@pytest.mark.parametrize("kind", ["planted", "rmat"])
def test_noalloc_modularity_matches_louvain_run(kind):
    torch = pytest.importorskip("torch")
    import paper_1805_10904_gb300 as lv
    lib = lv.load()
    f = _noalloc(lib)
    if kind == "planted":
        g = gg.sbm(4096, 128, 0.10, 0.002, 1, 4, seed=1)
    else:
        g = gg.rmat(13, 16, seed=5)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rp).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    res = lv.Louvain(0).run(rp, col, w)
    assert res.num_levels > 0
    for l in range(res.num_levels):
        lev = res.level(l)
        labels = torch.from_numpy(res.labels(l)).to(dev)
        for _ in range(2):  # two calls in a row share the same scratch array
            rc, qn, tw, q = _call(f, torch, g.n, rp, col, w, labels)
            assert rc == 0
            assert qn == lev.qn and tw == res.tw
            assert abs(q - lev.q) <= Q_RTOL * max(1.0, abs(lev.q))


def test_noalloc_singletons_and_limits():
    torch = pytest.importorskip("torch")
    import paper_1805_10904_gb300 as lv
    lib = lv.load()
    f = _noalloc(lib)
    g = gg.from_edges(5, [(0, 1, 2), (1, 2, 3), (3, 3, 4)])
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rp).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    singletons = torch.arange(5, dtype=torch.int32, device=dev)
    # all singletons: Qn = 2W * (sum of loops) - sum_i delta_i^2
    deg = np.array([2, 5, 3, 4, 0])
    tw = int(deg.sum())
    for _ in range(2):
        rc, qn, tw_got, _ = _call(f, torch, 5, rp, col, w, singletons)
        assert rc == 0 and tw_got == tw
        assert qn == tw * 4 - int((deg * deg).sum())
    # a label outside [0, n) is reported, and the next call is correct again
    bad = singletons.clone()
    bad[2] = 7
    rc, _, _, _ = _call(f, torch, 5, rp, col, w, bad)
    assert rc == 5
    rc, qn, _, _ = _call(f, torch, 5, rp, col, w, singletons)
    assert rc == 0 and qn == tw * 4 - int((deg * deg).sum())
    # more vertices than the static array holds: rejected before any device work
    rc = f(4194305, rp.data_ptr(), col.data_ptr(), w.data_ptr(), singletons.data_ptr(),
           None, None, None, None)
    assert rc == 12


@pytest.mark.parametrize("weighted", [True, False])
def test_noalloc_matches_oracle_on_random_partitions(weighted):
    """Random labels drawn from [0, n) leave many labels unused; NULL weights mean 1."""
    torch = pytest.importorskip("torch")
    import paper_1805_10904_gb300 as lv
    f = _noalloc(lv.load())
    g = gg.rmat(12, 16, seed=7)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rp).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w).to(dev) if weighted else None
    rng = np.random.default_rng(11)
    for ncomm in (1, 7, 300, g.n):
        labels = rng.integers(0, ncomm, size=g.n).astype(np.int32)
        # spread the used labels over [0, n) so that most labels stay unused
        labels = (labels * (g.n // ncomm)).astype(np.int32)
        ref_qn, ref_tw = oracle.modularity(g.rp, g.col, g.w if weighted else None, labels)
        d_labels = torch.from_numpy(labels).to(dev)
        for _ in range(2):
            rc, qn, tw, q = _call(f, torch, g.n, rp, col, w, d_labels)
            assert rc == 0
            assert qn == ref_qn and tw == ref_tw
            ref_q = float(ref_qn) / float(ref_tw * ref_tw)
            assert abs(q - ref_q) <= Q_RTOL * max(1.0, abs(ref_q))


def test_noalloc_later_calls_allocate_nothing():
    torch = pytest.importorskip("torch")
    import paper_1805_10904_gb300 as lv
    f = _noalloc(lv.load())
    g = gg.sbm(2048, 64, 0.2, 0.005, 1, 4, seed=3)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rp).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    labels = torch.from_numpy((np.arange(g.n) // 64).astype(np.int32)).to(dev)
    rc, first, _, _ = _call(f, torch, g.n, rp, col, w, labels)  # the set-up call
    assert rc == 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(dev)
    for _ in range(2):
        rc, qn, _, _ = _call(f, torch, g.n, rp, col, w, labels)
        assert rc == 0 and qn == first
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert free_after == free_before
