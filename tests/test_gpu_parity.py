"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Labels are integers decided by exact integer gains, so every level's labels, Qn
(exact int128), Q (double computed the same way on both sides), sweep counts and the
per-sweep trace (moved count, Qn) must be identical.  The relative tolerance on Q
stated for this method is 1e-12; both sides convert the same int128 values, so the
check below is equality, which implies it.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

Q_RTOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def lv():
    import paper_1805_10904_gb300 as m
    m.load()
    return m


def to_dev(torch, g):
    d = torch.device("cuda:0")
    return (torch.from_numpy(g.rp).to(d), torch.from_numpy(g.col).to(d),
            torch.from_numpy(g.w).to(d))


def assert_parity(res, ref, check_trace=True):
    assert res.num_levels == len(ref.levels)
    for l, rl in enumerate(ref.levels):
        lev = res.level(l)
        lab = res.labels(l)
        assert np.array_equal(lab, rl.labels), f"labels differ at level {l}"
        assert lev.ncomm == rl.ncomm and lev.qn == rl.qn and lev.qn_init == rl.qn_init
        assert lev.iters == rl.iters and lev.n == rl.n and lev.nnz == rl.nnz
        assert lev.q == rl.q or abs(lev.q - rl.q) <= Q_RTOL * abs(rl.q)
    if check_trace:
        assert res.trace() == ref.trace
    c, _ = res.counters()
    assert c[0] == ref.edge_visits


def run_both(torch, lv, g, **kw):
    okw = {k: kw[k] for k in ("theta", "max_iters", "max_levels", "vertex_following",
                              "vf_all_levels", "threshold_mode", "post_merge") if k in kw}
    ref = oracle.louvain(g.rp, g.col, g.w, **okw)
    h = lv.Louvain(0, **kw)
    res = h.run(*to_dev(torch, g))
    return res, ref


BIN_CONFIGS = [
    {},                                                          # default bins
    {"bins": (0, 0, 0, 0, 0, 12288)},                            # every row in one CTA
    {"bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32},           # every bin, many chunked rows
    {"bins": (0, 0, 0, 0, 0, 1), "chunk_entries": 32},           # rows above 16 chunked
    {"force_int128": True},
    {"wide_sums": True, "bins": (2, 4, 8, 16, 32, 64), "chunk_entries": 64},
    {"force_int128": True, "wide_sums": True, "bins": (0, 0, 0, 0, 0, 1), "chunk_entries": 32},
    {"bins": (8, 32, 128, 512, 2048, 12288), "chunk_entries": 128},
    {"bins": (0, 0, 0, 0, 0, 2)},                                # clusters of 2..16 CTAs
    {"bins": (1, 2, 3, 4, 5, 6), "wide_sums": True, "force_int128": True, "chunk_entries": 64},
    {"cuda_graphs": False},                                      # one host round trip per sweep
    {"sweep_streams": 0},                                        # bins one after another
    {"sweep_streams": 2, "cuda_graphs": False, "bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32},
    {"cuda_graphs": False, "bins": (0, 0, 0, 0, 0, 2), "chunk_entries": 32},
]


@pytest.mark.parametrize("seed", range(40))
def test_fuzz_small_graphs(torch, lv, seed):
    g = gg.random_small(1000 + seed, n_max=80)
    kw = dict(BIN_CONFIGS[seed % len(BIN_CONFIGS)])
    kw["vertex_following"] = seed % 3 != 0
    kw["vf_all_levels"] = seed % 5 == 0
    res, ref = run_both(torch, lv, g, **kw)
    assert_parity(res, ref)


@pytest.mark.parametrize("cfg", range(len(BIN_CONFIGS)))
def test_planted_partition_4096(torch, lv, cfg):
    """Planted partition: 4,096 vertices, 32 blocks of 128, p_in 0.10, p_out 0.002,
    weights uniform in [1, 4], threshold 1e-6, full multi-level run."""
    g = gg.sbm(4096, 128, 0.10, 0.002, 1, 4, seed=1)
    res, ref = run_both(torch, lv, g, **BIN_CONFIGS[cfg])
    assert_parity(res, ref)


@pytest.mark.parametrize("scale,cfg", [(10, 0), (12, 0), (13, 1), (14, 2), (12, 4), (15, 0),
                                       (14, 3), (13, 5), (12, 6), (15, 7), (16, 0), (13, 8),
                                       (14, 9), (17, 0)])
def test_rmat_medium(torch, lv, scale, cfg):
    """R-MAT graphs (a=.57, b=c=.19): hubs spanning many chunks, isolated vertices,
    several tiles of every scan and a ragged tail."""
    g = gg.rmat(scale, 16, seed=100 + scale)
    res, ref = run_both(torch, lv, g, **BIN_CONFIGS[cfg])
    assert_parity(res, ref)


@pytest.mark.parametrize("n,cfg", [(20_000, 0), (7_777, 2), (30_001, 1), (12_345, 5)])
def test_chung_lu(torch, lv, n, cfg):
    g = gg.chung_lu(n, 2.1, 10.0, 1, 8, seed=n)
    res, ref = run_both(torch, lv, g, **BIN_CONFIGS[cfg])
    assert_parity(res, ref)


def test_sbm_ragged_blocks(torch, lv):
    g = gg.sbm(10_007, 300, 0.05, 0.0005, 1, 8, seed=9)
    res, ref = run_both(torch, lv, g)
    assert_parity(res, ref)


@pytest.mark.parametrize("theta,max_iters,max_levels", [((1, 1000), 1000, 64), ((0, 1), 3, 2),
                                                        ((1, 10), 1000, 64), ((1, 10**6), 1, 64)])
def test_thresholds_and_caps(torch, lv, theta, max_iters, max_levels):
    g = gg.rmat(12, 16, seed=77)
    res, ref = run_both(torch, lv, g, theta=theta, max_iters=max_iters, max_levels=max_levels)
    assert_parity(res, ref)
    if not ref.hit_iter_cap:
        assert not any(res.level(l).hit_iter_cap for l in range(res.num_levels))


def test_hand_worked_cases(torch, lv):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        g = gg.from_edges(case["n"], [tuple(e) for e in case["edges"]])
        h = lv.Louvain(0, vertex_following=case["vertex_following"])
        res = h.run(*to_dev(torch, g))
        assert res.num_levels == len(case["levels"])
        for l, exp in enumerate(case["levels"]):
            assert res.labels(l).tolist() == exp["labels"]
            assert res.level(l).qn == exp["qn"]
        lev0 = [(t[2], t[3]) for t in res.trace() if t[0] == 0]
        assert lev0 == [(s[1], s[2]) for s in case["sweeps"]]


def test_edge_cases(torch, lv):
    h = lv.Louvain(0)
    for g in [gg.from_edges(0, []), gg.from_edges(1, []), gg.from_edges(6, []),
              gg.from_edges(1, [(0, 0, 5)]), gg.from_edges(2, [(0, 1, 1)]),
              gg.from_edges(3, [(0, 0, 2), (1, 1, 3), (2, 2, 1)]), gg.star(200),
              gg.from_edges(4, [(0, 1, 2**31 - 1), (2, 3, 2**31 - 1), (1, 2, 1)])]:
        ref = oracle.louvain(g.rp, g.col, g.w)
        res = h.run(*to_dev(torch, g))
        assert_parity(res, ref)


def test_host_pointers_match_device_pointers(torch, lv):
    g = gg.rmat(13, 16, seed=5)
    h = lv.Louvain(0)
    a = h.run(*to_dev(torch, g))
    b = h.run(g.rp, g.col, g.w)
    assert a.num_levels == b.num_levels
    for l in range(a.num_levels):
        assert np.array_equal(a.labels(l), b.labels(l))
        assert a.level(l).qn == b.level(l).qn


def test_unweighted_means_all_ones(torch, lv):
    g = gg.rmat(11, 8, seed=3)
    ones = np.ones_like(g.w)
    ref = oracle.louvain(g.rp, g.col, ones)
    h = lv.Louvain(0)
    rp, col, _ = to_dev(torch, g)
    res = h.run(rp, col, None)
    assert_parity(res, ref)


def test_deterministic_and_allocator_independent(torch, lv):
    g = gg.rmat(14, 16, seed=8)
    a = lv.Louvain(0, torch_alloc=True).run(*to_dev(torch, g))
    b = lv.Louvain(0, torch_alloc=False).run(*to_dev(torch, g))
    c = lv.Louvain(0).run(*to_dev(torch, g))
    for r in (b, c):
        assert r.num_levels == a.num_levels
        for l in range(a.num_levels):
            assert np.array_equal(a.labels(l), r.labels(l))
        assert r.trace() == a.trace()


def test_invalid_inputs_are_reported_and_handle_survives(torch, lv):
    h = lv.Louvain(0, checks=2)
    g = gg.path(5)
    rp, col, w = to_dev(torch, g)
    bad_col = col.clone()
    bad_col[3] = 99
    with pytest.raises(lv.LouvainError) as e:
        h.run(rp, bad_col, w)
    assert e.value.code == 5
    bad_w = w.clone()
    bad_w[0] = 0
    with pytest.raises(lv.LouvainError) as e:
        h.run(rp, col, bad_w)
    assert e.value.code == 4
    bad_rp = rp.clone()
    bad_rp[2] = 0
    with pytest.raises(lv.LouvainError) as e:
        h.run(bad_rp, col, w)
    assert e.value.code == 5
    asym_w = w.clone()
    asym_w[0] = 7
    with pytest.raises(lv.LouvainError) as e:
        h.run(rp, col, asym_w)
    assert e.value.code == 2
    dup = gg.Graph(np.array([0, 2, 3], np.int64), np.array([1, 1, 0], np.int32),
                   np.array([1, 1, 1], np.int32))
    with pytest.raises(lv.LouvainError) as e:
        h.run(*to_dev(torch, dup))
    assert e.value.code in (2, 3)
    # the handle still works
    res = h.run(rp, col, w)
    ref = oracle.louvain(g.rp, g.col, g.w)
    assert_parity(res, ref)


@pytest.mark.parametrize("graphs", [True, False])
def test_sweep_loop_modes_run_as_configured(torch, lv, graphs):
    """cuda_graphs=True runs every sweep but the first of each phase (table-free, launched
    on its own) inside the device-side loop (a CUDA graph with a while node),
    cuda_graphs=False one sweep per host round trip; both give the oracle's result."""
    g = gg.rmat(13, 16, seed=9)
    res, ref = run_both(torch, lv, g, cuda_graphs=graphs)
    assert_parity(res, ref)
    in_graph, host_loop, steps, captures = res.exec_info()[:4]
    assert steps >= res.num_levels
    phases = sum(1 for rec in res.trace() if rec[1] == 1)
    if graphs:
        assert host_loop == phases and in_graph == res.counters()[0][1] - phases
        assert captures >= 1
    else:
        assert in_graph == 0 and host_loop == res.counters()[0][1] and captures == 0


def test_autotuned_bins_give_the_same_result(torch, lv):
    """The autotuner only picks which kernel handles a row: a run with autotune = 1 matches
    the oracle, the first call tunes, a second call on the same (n, nnz) reuses the choice,
    and the bins louvain_autotune returns are a valid configuration giving the same result."""
    g = gg.rmat(14, 16, seed=21)
    ref = oracle.louvain(g.rp, g.col, g.w)
    h = lv.Louvain(0, autotune=True)
    d = to_dev(torch, g)
    first = h.run(*d)
    assert_parity(first, ref)
    assert first.exec_info()[4] > 0 and first.exec_info()[5] == 0
    second = h.run(*d)
    assert_parity(second, ref)
    assert second.exec_info()[4] == 0 and second.exec_info()[5] == 1
    h2 = lv.Louvain(0)
    bins, chunk, ms, trials = h2.autotune(g.rp, g.col, g.w)  # host arrays
    assert trials > 0 and ms > 0
    assert 0 <= bins[0] <= bins[1] <= bins[2] <= bins[3] <= bins[4] <= bins[5] <= 12288
    assert chunk in (1024, 2048, 4096)
    assert_parity(lv.Louvain(0, bins=bins, chunk_entries=chunk).run(*d), ref)
    assert h2.autotune(*d)[3] == 0  # cached on the handle


@pytest.mark.parametrize("theta", [(1, 1_000_000), (1, 1000), (1, 20)])
@pytest.mark.parametrize("kind", ["sbm", "rmat", "small"])
def test_relative_threshold_mode(torch, lv, theta, kind):
    """threshold_mode 1: the relative phase test of Algorithm 1 on the device controller."""
    if kind == "sbm":
        g = gg.sbm(2048, 64, 0.15, 0.003, 1, 4, seed=3)
    elif kind == "rmat":
        g = gg.rmat(13, 16, seed=31)
    else:
        g = gg.random_small(4242, n_max=60)
    res, ref = run_both(torch, lv, g, theta=theta, threshold_mode=1)
    assert_parity(res, ref)


@pytest.mark.parametrize("kw", [{}, {"max_iters": 1}, {"max_iters": 2, "vertex_following": False},
                                {"theta": (1, 50), "force_int128": True},
                                {"bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32, "max_iters": 2}])
@pytest.mark.parametrize("kind", ["sbm", "rmat", "small", "path"])
def test_post_merge_mode(torch, lv, kw, kind):
    """post_merge: the Sec. 5.1.2 merge after every phase, on the device."""
    if kind == "sbm":
        g = gg.sbm(2048, 64, 0.15, 0.003, 1, 4, seed=8)
    elif kind == "rmat":
        g = gg.rmat(13, 16, seed=37)
    elif kind == "small":
        g = gg.random_small(777, n_max=60)
    else:
        g = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
    res, ref = run_both(torch, lv, g, post_merge=True, **kw)
    assert_parity(res, ref)


# Heavy weights put 2W far above 2^32 while every weighted degree stays small or large:
# the level's widths follow its largest weighted degree d_max (32-bit table sums when
# d_max < 2^32, int64 gains when d_max * 2W <= 2^62), so these graphs run the width
# combinations that 2W alone would never pick.
HEAVY = [
    # (weights, expected: d_max < 2^32, d_max * 2W <= 2^62)
    ((1 << 16, 1 << 20), (True, True)),        # 2W ~ 2^35: int64 gains, 32-bit sums
    ((1 << 25, 1 << 26), (True, False)),       # int128 gains, 32-bit sums
    ((1 << 29, (1 << 31) - 1), (False, False)),  # int128 gains, 64-bit sums
]


@pytest.mark.parametrize("weights,expect", HEAVY)
@pytest.mark.parametrize("cfg", [{}, {"bins": (1, 2, 3, 4, 5, 6), "chunk_entries": 32}])
def test_heavy_weights_per_level_widths(torch, lv, weights, expect, cfg):
    g = gg.sbm(4096, 128, 0.10, 0.002, weights[0], weights[1], seed=9)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    dmax = int(np.bincount(rows, weights=g.w.astype(np.float64)).max())
    tw = int(g.w.astype(np.int64).sum())
    assert tw > 2 ** 32
    assert (dmax < 2 ** 32, dmax * tw <= 2 ** 62) == expect
    res, ref = run_both(torch, lv, g, **cfg)
    assert_parity(res, ref)


@pytest.mark.parametrize("shift", [(1, 0), (0, 3), (2, 1)])
def test_unaligned_column_and_weight_arrays(torch, lv, shift):
    """Column and weight arrays that start 4, 8 or 12 bytes past a 16-byte boundary (views
    into larger buffers) give the same result in every kernel path."""
    g = gg.rmat(14, 16, seed=31)
    d = torch.device("cuda:0")

    def view(a, s):
        buf = torch.zeros(a.size + s, dtype=torch.int32, device=d)
        buf[s:] = torch.from_numpy(a).to(d)
        return buf[s:]

    rp = torch.from_numpy(g.rp).to(d)
    col, w = view(g.col, shift[0]), view(g.w, shift[1])
    assert col.data_ptr() % 16 or w.data_ptr() % 16
    ref = oracle.louvain(g.rp, g.col, g.w)
    for cfg in ({}, {"bins": (0, 0, 0, 0, 0, 12288)}, {"sweep_streams": 0, "cuda_graphs": False}):
        assert_parity(lv.Louvain(0, **cfg).run(rp, col, w), ref)
