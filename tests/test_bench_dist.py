"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): each rank reports its own
time and work; rank 0 must see the max time and the summed work, as in a torchrun launch."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    t = bench.reduce_max(10.0 + rank, w)
    v = bench.reduce_sum(100.0 * (rank + 1), w)
    out.put((rank, t, v))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 11.0 and v == 300.0


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(2.0, 1) == 2.0


def test_roofline_traffic_only_for_the_captured_kernel_and_bins():
    """bench.py reports the committed DRAM-traffic figure only while the kernel source and
    the bin layout match the capture; anything else gives None (no stale number)."""
    import json
    import bench
    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")) as f:
        kernels = json.load(f)["kernels"]
    assert kernels
    import hashlib
    src = os.path.join(os.path.dirname(bench.__file__), "paper_1805_10904_gb300", "csrc",
                       "k_move_impl.cuh")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    for name, rec in kernels.items():
        bins, chunk = rec["bins"], rec["chunk_entries"]
        expected = rec["dram_bytes_per_launch_full"] if sha == rec["source_sha256"] else None
        assert bench.kernel_traffic(name, bins, chunk) == expected
        assert bench.kernel_traffic(name, bins[:-1] + [bins[-1] // 2], chunk) is None
        assert bench.kernel_traffic(name, bins, chunk // 2) is None
    other = next(k for k in ("k_move_cta<128>", "k_move_cta<256>", "k_move_cta<1024>")
                 if k not in kernels)
    assert bench.kernel_traffic(other, bins, chunk) is None
