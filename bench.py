"""Benchmark: multi-level synchronous Louvain on the largest single graph, R-MAT scale 26.

One step = one full multi-level run (every local-moving sweep, renumbering and graph
induction of every level) of the library on the same synthetic graph:
R-MAT scale 26 (67,108,864 vertices, 16 * 2^26 sampled pairs, a=0.57 b=0.19 c=0.19),
symmetrised, loops and duplicates dropped, int32 weights uniform in [1, 16], seed 26
(2.1e9 stored entries; 2W above 2^32, so int128 gains and 64-bit table sums).
`--scale 22` runs the R-MAT scale-22 graph instead.

Metric: local-move edge-visits/s = sum over phases of (sweeps applied) * (stored
entries of that phase's graph), divided by the device time of the run.

Prints one JSON line.  With torchrun (N > 1) every rank runs its own replica on its
own GPU (no data-path collective; weak scaling) and rank 0 reports the max time.
`--impl reference` times the CPU oracle (single thread) on a bounded sample of the
same workload instead: the full multi-level run on the subgraph induced by one aligned
block of vertices (rows and columns in [r0, r0 + 2^block_bits)).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "local-move edge-visits/s, HBM % of peak; batched graphs/s vs plain (bit-exact)"
UNIT = "edge-visits/s"
def workload(scale: int) -> str:
    return (f"R-MAT scale {scale} ({1 << scale:,} vertices, edge factor 16, a=0.57 b=0.19 "
            "c=0.19), symmetrised, duplicates and self-loops dropped, int32 weights uniform in "
            f"[1,16], int32 ids, seed {scale}; full multi-level run to threshold 1e-6; "
            "autotuned degree bins")
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 1024 * 1024
# kernel of every bin slot (louvain_result_bin_stats): the table kernels, then the
# first-sweep kernels of the same bins (bins 5-9 share the 1024-thread CTA kernel there)
KERNEL_NAMES = ["k_move_small", "k_move_group<8>", "k_move_group<32>", "k_move_cta<128>",
                "k_move_cta<256>", "k_move_cta<1024>", "k_move_cluster<2>", "k_move_cluster<4>",
                "k_move_cluster<8>", "k_move_cluster<16>", "k_move_huge",
                "k_move_small<first>", "k_move_group_first<8>", "k_move_group_first<32>",
                "k_move_cta_first<128>", "k_move_cta_first<256>", "k_move_cta_first<1024>",
                "k_move_cta_first<1024> (bin 6)", "k_move_cta_first<1024> (bin 7)",
                "k_move_cta_first<1024> (bin 8)", "k_move_cta_first<1024> (bin 9)",
                "k_move_huge (first sweep)"]


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--scale", type=int, default=26, help="R-MAT scale (26 is the workload)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--sample-bits", type=int, default=20,
                   help="CPU sample: vertex block of 2^bits vertices (induced subgraph)")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer arm (profiling)")
    p.add_argument("--no-autotune", action="store_true",
                   help="use the default degree bins instead of tuning them (profiling)")
    p.add_argument("--batch-graphs", type=int, default=512,
                   help="also time the mixed batch workload of this many graphs, batched vs "
                        "one graph at a time (0: skip)")
    p.add_argument("--batch-only", action="store_true",
                   help="time only the batch workload (its own JSON line)")
    p.add_argument("--serve-requests", type=int, default=2000,
                   help="also run the serving workload with this many requests (0: skip)")
    p.add_argument("--serve-only", action="store_true",
                   help="run only the serving workload (its own JSON line)")
    p.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    p.add_argument("--no-edges", action="store_true",
                   help="skip timing the edge-list to CSR conversion")
    p.add_argument("--edges-scale", type=int, default=22,
                   help="R-MAT scale of the edge-list conversion leg")
    p.add_argument("--serve-budget-gb", type=float, default=120.0)
    p.add_argument("--serve-slots", type=int, default=256)
    return p.parse_args(argv)


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity when world == 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- helpers

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_traffic(kernel_name: str, bins=None, chunk=None):
    """DRAM bytes per launch of the kernel from the committed ncu summary, or None when
    the summary is missing or was taken on a different kernel source or bin layout."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    src = os.path.join(ROOT, "paper_1805_10904_gb300", "csrc", "k_move_impl.cuh")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    entry = rec.get("kernels", {}).get(kernel_name)
    if not entry or entry.get("source_sha256") != sha:
        return None
    if bins is not None and (list(entry.get("bins", [])) != list(bins) or
                             entry.get("chunk_entries") != chunk):
        return None
    return entry.get("dram_bytes_per_launch_full")


def host_cpu():
    """Host CPU model (from /proc/cpuinfo) and logical core count."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    if not model or model.startswith("0x"):  # Arm: /proc/cpuinfo gives only a part code
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip() or model
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    import platform
    return {"model": model or platform.processor() or platform.machine(),
            "arch": platform.machine(), "logical_cores": os.cpu_count()}


def make_graph(scale: int):
    import graphgen as gg
    return gg.rmat(scale, 16, 0.57, 0.19, 0.19, 1, 16, seed=scale)


# ---------------------------------------------------------------- CPU oracle timing

def sample_block(scale: int, bits: int):
    """First vertex of the CPU sample's block: the aligned block of 2^bits vertices whose
    index is the top bit of the vertex id (vertices [2^(scale-1), 2^(scale-1) + 2^bits)),
    a block of typical density (one R-MAT level in the (1,1) quadrant)."""
    return 1 << (scale - 1) if bits < scale else 0


def induced_block(g, r0: int, bits: int):
    """Subgraph induced by vertices [r0, r0 + 2^bits) of g, renumbered from 0: the rows of
    the block with the entries whose column lies in the block (symmetric, rows sorted)."""
    import numpy as np
    import graphgen as gg
    r1 = min(g.n, r0 + (1 << bits))
    e0, e1 = int(g.rp[r0]), int(g.rp[r1])
    col = np.asarray(g.col[e0:e1])
    keep = (col >= r0) & (col < r1)
    rows = np.repeat(np.arange(r1 - r0, dtype=np.int64), np.diff(g.rp[r0:r1 + 1]))
    rp = np.zeros(r1 - r0 + 1, np.int64)
    np.add.at(rp, rows[keep] + 1, 1)
    np.cumsum(rp, out=rp)
    return gg.Graph(rp, (col[keep] - r0).astype(np.int32),
                    np.ascontiguousarray(np.asarray(g.w[e0:e1])[keep]), f"block{r0}")


def time_oracle(sample):
    """Single-threaded oracle: the full multi-level run on the sample graph."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.louvain(sample.rp, sample.col, sample.w)
    dt = time.perf_counter() - t0
    visits = r.edge_visits
    return visits / dt, dt, visits


def time_omp(sample, threads: int):
    """The OpenMP CPU Louvain (cpu_omp) on the sample graph with `threads` threads; its
    result is checked equal to the oracle's in tests/test_cpu_omp.py."""
    import cpu_omp
    t0 = time.perf_counter()
    r = cpu_omp.louvain(sample.rp, sample.col, sample.w, threads=threads)
    dt = time.perf_counter() - t0
    return r.edge_visits / dt, dt, r.edge_visits


def sample_text(scale, bits, sample):
    r0 = sample_block(scale, bits)
    return (f"full multi-level oracle run (defaults as the GPU run) on the subgraph of the "
            f"workload graph induced by vertices [{r0:,}, {r0 + (1 << bits):,}) "
            f"({sample.n:,} vertices, {sample.nnz:,} entries), single thread, per step")


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    g = make_graph(args.scale)
    sample_g = induced_block(g, sample_block(args.scale, args.sample_bits), args.sample_bits)
    del g
    sample = sample_text(args.scale, args.sample_bits, sample_g)
    for _ in range(args.warmup):
        time_oracle(sample_g)
    times, visits_total = [], 0
    for _ in range(args.steps):
        _, dt, v = time_oracle(sample_g)
        times.append(dt)
        visits_total += v
    value = visits_total / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": workload(args.scale), "graph_n": 1 << args.scale,
                   "sample_n": sample_g.n, "sample_nnz": sample_g.nnz,
                   "parallelism": "single host thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host_cpu": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- native arm

def run_e2e(args, g, lv, local, stream, world, dev, bins, chunk):
    """Same metric through the C ABI with pinned host buffers: the H2D copy of the graph
    and the D2H copy of every level's labels are inside the timed region.  The handle copies
    each recorded level's labels to pinned host memory while the later levels run
    (host_labels), and every level's labels are read there.  The handle uses the bins the
    timed runs' autotuner chose (the choice it would cache)."""
    import torch
    rp_h = torch.from_numpy(g.rp).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    w_h = torch.from_numpy(g.w).pin_memory()
    h2 = lv.Louvain(local, profile=False, bins=bins, chunk_entries=chunk, host_labels=True)
    for _ in range(max(1, args.warmup)):
        r = h2.run(rp_h, col_h, w_h, stream=stream.cuda_stream)
        for l in range(r.num_levels):
            r.labels(l, copy=False)
        r.close()
    barrier(world)
    e2e_s, e2e_visits, d2h = 0.0, 0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = h2.run(rp_h, col_h, w_h, stream=stream.cuda_stream)
        out = [r.labels(l, copy=False) for l in range(r.num_levels)]
        e2e_s += time.perf_counter() - t0
        e2e_visits += int(r.counters()[0][0])
        d2h = sum(a.nbytes for a in out)
        del out  # views into the result's pinned copy
        r.close()
    h2.close()
    del rp_h, col_h, w_h
    e2e_max = reduce_max(e2e_s, world, dev)
    e2e_all = reduce_sum(float(e2e_visits), world, dev)
    h2d = g.rp.nbytes + g.col.nbytes + g.w.nbytes
    return {"value": e2e_all / e2e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


BATCH_WORKLOAD = ("mixed batch: graph sizes log-uniform in [1K, 200K] vertices; even graphs "
                  "planted partition (block size log-uniform 32-512, average degree 8-40, "
                  "80% inside blocks), odd graphs Chung-Lu power law (exponent 2.1, average "
                  "degree 10); int32 weights uniform in [1, 8]; seed 512; stacked "
                  "block-diagonal CSR; full multi-level run per graph to threshold 1e-6")


def run_batch_workload(args, lv, dev, stream, steps, warmup):
    """Graphs/s of louvain_run_batch over the mixed workload against louvain_run on the
    same graphs one at a time (inputs resident in HBM for both), and whether every
    graph's result is identical in both forms."""
    import numpy as np
    import torch
    import graphgen as gg
    graphs = gg.batch_mix(args.batch_graphs, seed=512)
    vptr, eptr, rp, col, w = lv.stack_graphs([(g.rp, g.col, g.w) for g in graphs])
    d_rp, d_col, d_w = (torch.from_numpy(a).to(dev) for a in (rp, col, w))
    singles = [tuple(torch.from_numpy(a).to(dev) for a in (g.rp, g.col, g.w)) for g in graphs]
    h = lv.Louvain(dev.index, profile=False)

    def batched():
        return h.run_batch(vptr, d_rp, d_col, d_w, graph_eptr=eptr, stream=stream.cuda_stream)

    def plain():
        return [h.run(*t, stream=stream.cuda_stream) for t in singles]

    def timed(fn):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        out = fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1), out

    for _ in range(warmup):
        for r in batched():
            r.close()
        for r in plain():
            r.close()
    t_b, t_p, kernels = [], [], 0
    identical = True
    for k in range(steps):
        ms, rb = timed(batched)
        t_b.append(ms)
        kernels += int(rb[0].counters()[0][4]) if rb else 0
        ms, rp_ = timed(plain)
        t_p.append(ms)
        if k == 0:  # compare every graph's levels, labels and trace in both forms
            for a, b in zip(rb, rp_):
                if a.num_levels != b.num_levels or a.trace() != b.trace():
                    identical = False
                    break
                for l in range(a.num_levels):
                    if a.level(l) != b.level(l) or not np.array_equal(a.labels(l), b.labels(l)):
                        identical = False
                        break
        for r in rb + rp_:
            r.close()
    nb = sum(t_b) / len(t_b)
    npl = sum(t_p) / len(t_p)
    return {
        "workload": BATCH_WORKLOAD, "graphs": len(graphs), "total_vertices": int(vptr[-1]),
        "total_entries": int(eptr[-1]), "steps": steps,
        "batched_ms_per_step": nb, "plain_ms_per_step": npl,
        "graphs_per_s_batched": len(graphs) / (nb / 1000.0),
        "graphs_per_s_plain": len(graphs) / (npl / 1000.0),
        "speedup": npl / nb, "identical_to_plain": identical,
        "gpu_launches_per_batched_step": kernels // max(1, steps),
    }


SERVE_WORKLOAD = ("serving: Poisson arrivals; half R-MAT graphs of scale uniform in 10-21 (edge "
                  "factor 16, a=0.57 b=0.19 c=0.19), half planted partitions as in the mixed "
                  "batch; int32 weights uniform in [1, 16]; requests drawn with replacement "
                  "from a pool of 48 distinct graphs (2 R-MAT per scale, 24 planted "
                  "partitions); HBM admission budget and slot count as stated")


def serve_pool(seed=4):
    import numpy as np
    import graphgen as gg
    rmat = {s: [gg.rmat(s, 16, 0.57, 0.19, 0.19, 1, 16, seed=gg.graph_seed(seed, 100 * s + k))
                for k in range(2)] for s in range(10, 22)}
    sbm = []
    for p in gg.batch_mix_params(48, seed=seed)[0::2]:
        _, n, b, p_in, p_out, gs = p
        sbm.append(gg.sbm(n, b, p_in, p_out, 1, 16, gs))
    return rmat, sbm


def run_serve_workload(args, lv, dev):
    """Requests arrive as a Poisson stream and are served by the request loop; reports
    p50/p99 submit-to-finish latency and graphs/s, against the same requests run one at a
    time with louvain_run, and checks a sample of results against their plain runs."""
    import threading
    import numpy as np
    import torch
    import graphgen as gg
    rmat, sbm = serve_pool()
    rng = np.random.Generator(np.random.PCG64(gg.graph_seed(4, 0)))
    nreq = args.serve_requests
    picks = []
    for k in range(nreq):
        if rng.random() < 0.5:
            s = int(rng.integers(10, 22))
            picks.append(rmat[s][int(rng.integers(0, 2))])
        else:
            picks.append(sbm[int(rng.integers(0, len(sbm)))])
    gaps = rng.exponential(1.0 / args.serve_rate, size=nreq)
    h = lv.Louvain(dev.index, torch_alloc=False)
    # warm-up: a few requests through the loop
    h.serve_open(int(args.serve_budget_gb * (1 << 30)), args.serve_slots)
    for t in [h.submit(g.rp, g.col, g.w) for g in (rmat[14][0], sbm[0], rmat[18][1])]:
        h.poll(t, -1).close()
    tickets = [None] * nreq
    t_sub = [0.0] * nreq

    def producer():
        t0 = time.perf_counter()
        due = 0.0
        for k, g in enumerate(picks):
            due += gaps[k]
            wait = t0 + due - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            t_sub[k] = time.perf_counter()
            tickets[k] = h.submit(g.rp, g.col, g.w)

    th = threading.Thread(target=producer)
    start = time.perf_counter()
    th.start()
    lat, waits, t_fin = [], [], []
    sample = {}
    for k in range(nreq):
        while tickets[k] is None:
            time.sleep(0.0005)
        r = h.poll(tickets[k], -1)
        t_fin.append(time.perf_counter())
        _, tm = r.counters()
        lat.append(float(tm[3]))
        waits.append(float(tm[2]))
        if k % max(1, nreq // 16) == 0:
            sample[k] = [(r.level(l).qn, r.labels(l)) for l in range(r.num_levels)]
        r.close()
    th.join()
    span = max(t_fin) - start
    # saturation: every request submitted at once, graphs/s of the loop at full load
    t0 = time.perf_counter()
    burst = [h.submit(g.rp, g.col, g.w) for g in picks]
    for t in burst:
        h.poll(t, -1).close()
    burst_s = time.perf_counter() - t0
    h.serve_close()
    # the same requests one at a time, inputs resident on the device
    uniq = {id(g): tuple(torch.from_numpy(a).to(dev) for a in (g.rp, g.col, g.w)) for g in picks}
    hp = lv.Louvain(dev.index)
    for g in (rmat[14][0], sbm[0]):
        hp.run(*uniq.get(id(g), tuple(torch.from_numpy(a).to(dev) for a in (g.rp, g.col, g.w))))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    identical = True
    for k, g in enumerate(picks):
        r = hp.run(*uniq[id(g)])
        if k in sample:
            got = [(r.level(l).qn, r.labels(l)) for l in range(r.num_levels)]
            identical = identical and len(got) == len(sample[k]) and all(
                a[0] == b[0] and np.array_equal(a[1], b[1]) for a, b in zip(got, sample[k]))
        r.close()
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - t0
    lat = np.asarray(lat)
    return {
        "workload": SERVE_WORKLOAD, "requests": nreq, "rate_per_s": args.serve_rate,
        "budget_gb": args.serve_budget_gb, "slots": args.serve_slots,
        "total_entries": int(sum(g.nnz for g in picks)),
        "latency_ms_p50": float(np.percentile(lat, 50)),
        "latency_ms_p99": float(np.percentile(lat, 99)),
        "admission_wait_ms_p99": float(np.percentile(np.asarray(waits), 99)),
        "graphs_per_s_served": nreq / span, "served_span_s": span,
        "graphs_per_s_saturated": nreq / burst_s, "saturated_span_s": burst_s,
        "graphs_per_s_plain": nreq / plain_s, "plain_span_s": plain_s,
        "saturated_vs_plain": plain_s / burst_s,
        "identical_to_plain_sample": identical, "sample_size": len(sample),
    }


def run_edges_workload(lv, g, dev, stream, reps=5):
    """Edge-list input (Sec. 5.1.2 neighbour computation): the workload graph's undirected
    edges (one per pair, loops once) in a seeded random order and orientation, resident in
    HBM, converted to the symmetric CSR by louvain_csr_from_edges; checks the result equals
    the generated CSR and reports input edges/s."""
    import numpy as np
    import torch
    rows = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.rp))
    keep = rows <= g.col
    rng = np.random.Generator(np.random.PCG64(2205))
    perm = rng.permutation(int(keep.sum()))
    u, v, w = rows[keep][perm], g.col[keep][perm], g.w[keep][perm]
    flip = rng.random(len(u)) < 0.5
    u, v = np.where(flip, v, u), np.where(flip, u, v)
    du, dv, dw = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (u, v, w))
    h = lv.Louvain(dev.index)
    rp, col, ww = h.csr_from_edges(g.n, du, dv, dw, stream=stream.cuda_stream)
    same = (np.array_equal(rp.cpu().numpy(), g.rp) and np.array_equal(col.cpu().numpy(), g.col)
            and np.array_equal(ww.cpu().numpy(), g.w))
    del rp, col, ww
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = h.csr_from_edges(g.n, du, dv, dw, stream=stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        del out
    ms = statistics.median(times)
    return {"edges": int(len(u)), "csr_entries": int(g.nnz), "ms": ms,
            "edges_per_s": len(u) / (ms / 1000.0), "identical_to_generated_csr": bool(same),
            "note": "median of %d calls, inputs on the device; each call allocates its "
                    "scratch and synchronises once" % reps}


def run_native(args):
    import numpy as np
    import torch

    import paper_1805_10904_gb300 as lv

    world, rank, local = dist_env()
    dist = dist_init(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.batch_only:
        stream = torch.cuda.current_stream(dev)
        b = run_batch_workload(args, lv, dev, stream, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"batch": b}), flush=True)
        return 0
    if args.serve_only:
        sv = run_serve_workload(args, lv, dev)
        if rank == 0:
            print(json.dumps({"serve": sv}), flush=True)
        return 0
    g = make_graph(args.scale)
    rp = torch.from_numpy(g.rp).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    stream = torch.cuda.current_stream(dev)
    # the library's default mode: sweeps as CUDA graphs, the bins of a sweep on concurrent
    # streams, bins chosen by the autotuner during the warm-up
    h = lv.Louvain(local, profile=False, autotune=not args.no_autotune)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def step():
        return h.run(rp, col, w, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step().close()
    torch.cuda.synchronize(dev)
    if args.no_autotune:
        tuned_bins, tuned_chunk = (8, 32, 128, 512, 2048, 12288), 4096
    else:
        tuned_bins, tuned_chunk, _, _ = h.autotune(rp, col, w)  # the warm-up's cached choice

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    step_ms, visits, launches = [], 0, 0
    levels = None
    for _ in range(args.steps):
        flush.fill_(1)  # L2 flush between timed steps (untimed)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        res = step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        c, _ = res.counters()
        visits += int(c[0])
        launches += int(c[4])
        if levels is None:
            levels = [(l.n, l.nnz, l.iters, l.ncomm, round(l.q, 6)) for l in res.levels()]
            run_bytes = {"local_move": int(c[2]), "coarsen": int(res.coarsen_stats()[1])}
        res.close()
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    total_ms = sum(step_ms)
    max_ms = reduce_max(total_ms, world, dev)
    all_visits = reduce_sum(float(visits), world, dev)

    # kernel times: the same runs profiled (per-bin CUDA events on each bin's stream), with
    # the bins one after another so that every kernel is timed alone, same tuned bins
    hp = lv.Louvain(local, profile=True, sweep_streams=0, bins=tuned_bins,
                    chunk_entries=tuned_chunk)
    hp.run(rp, col, w, stream=stream.cuda_stream).close()
    prof_steps = 3
    dom = {"time_ms": 0.0, "bytes": 0, "launches": 0, "id": None}
    bins_acc, coarsen_ms, coarsen_bytes, prof_ms = {}, 0.0, 0, 0.0
    for _ in range(prof_steps):
        flush.fill_(1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        res = hp.run(rp, col, w, stream=stream.cuda_stream)
        ev1.record(stream)
        ev1.synchronize()
        prof_ms += ev0.elapsed_time(ev1)
        c, t = res.counters()
        dom["time_ms"] += float(t[4])
        dom["bytes"] += int(c[6])
        dom["launches"] += int(c[5])
        dom["id"] = int(c[7])
        coarsen_ms += float(t[1])
        coarsen_bytes += int(res.coarsen_stats()[1])
        for b, st in enumerate(res.bin_stats()):
            agg = bins_acc.setdefault(b, {"time_ms": 0.0, "launches": 0, "alg_bytes": 0})
            for key in agg:
                agg[key] += st[key]
        res.close()

    hp.close()
    h.close()
    del rp, col, w, flush
    torch.cuda.empty_cache()
    # end-to-end through the C ABI with pinned host buffers: H2D inside, labels D2H inside
    e2e = (run_e2e(args, g, lv, local, stream, world, dev, tuned_bins, tuned_chunk)
           if not args.no_e2e else None)
    torch.cuda.empty_cache()
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        # the oracle on a bounded sample of the workload graph, one host thread
        sample_g = induced_block(g, sample_block(args.scale, args.sample_bits), args.sample_bits)
        v, dt, vis = time_oracle(sample_g)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": sample_text(args.scale, args.sample_bits, sample_g) +
                         f": {vis:,} edge visits in {dt:.1f} s",
               "host_cpu": host_cpu()}
        # this project's OpenMP synchronous Louvain on the same sample (same results as the
        # oracle), at 8 threads as in the paper's CPU comparison and at every host core
        omp = {}
        for th in sorted({8, os.cpu_count() or 1}):
            v2, dt2, _ = time_omp(sample_g, th)
            omp[f"threads_{th}"] = {"value": v2, "unit": UNIT, "cores": th,
                                    "seconds": round(dt2, 3)}
        cpu["omp"] = omp
    graph_n, graph_nnz = g.n, g.nnz
    del g
    batch = (run_batch_workload(args, lv, dev, stream, 2, 1) if args.batch_graphs > 0
             else None)
    torch.cuda.empty_cache()
    serve = run_serve_workload(args, lv, dev) if args.serve_requests > 0 else None
    torch.cuda.empty_cache()
    edges = None
    if not args.no_edges:
        ge = make_graph(args.edges_scale)
        edges = run_edges_workload(lv, ge, dev, stream)
        edges["workload"] = f"R-MAT scale {args.edges_scale} (seed {args.edges_scale})"
        del ge

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_hbm_peak()
    roofline = None
    if dom["time_ms"] > 0 and dom["launches"] > 0:
        achieved = dom["bytes"] / (dom["time_ms"] / 1000.0) / 1e9
        name = KERNEL_NAMES[dom["id"]]
        if dom["id"] == 5 and tuned_bins[5] <= 6144:
            name = "k_move_cta<512>"  # bin 5 with an 8K-slot table (1024 threads if 64-bit)
        traffic = kernel_traffic(name, tuned_bins, tuned_chunk)
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic,
                    "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                    "avg_launch_ms": dom["time_ms"] / dom["launches"]}

    value = all_visits / (max_ms / 1000.0)
    ms_step = max_ms / args.steps
    roofline_coarsen = None
    if coarsen_ms > 0:
        ach = coarsen_bytes / (coarsen_ms / 1000.0) / 1e9
        roofline_coarsen = {"bound": "hbm", "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                            "unit": "GB/s", "frac": ach / peak,
                            "bytes_per_step": coarsen_bytes // prof_steps,
                            "ms_per_step": coarsen_ms / prof_steps,
                            "note": "graph induction of all levels: algorithmic bytes "
                                    "(louvain_result_coarsen_stats) over its device time in the "
                                    "profiled runs"}
    step_bytes = run_bytes["local_move"] + run_bytes["coarsen"]
    roofline_step = {"bound": "hbm", "bytes_local_move": run_bytes["local_move"],
                     "bytes_coarsen": run_bytes["coarsen"], "ms_per_step": ms_step,
                     "achieved": step_bytes / (ms_step / 1000.0) / 1e9,
                     "achieved_local_move": run_bytes["local_move"] / (ms_step / 1000.0) / 1e9,
                     "peak": peak, "unit": "GB/s",
                     "frac": step_bytes / (ms_step / 1000.0) / 1e9 / peak,
                     "note": "whole run: algorithmic bytes of every sweep and induction over "
                             "the timed step (includes binning, renumbering and host syncs)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": workload(args.scale), "graph_n": graph_n,
                   "graph_nnz": graph_nnz,
                   "levels": levels, "parallelism": "replicas" if world > 1 else "single",
                   "bins": list(tuned_bins), "chunk_entries": tuned_chunk,
                   "l2": "L2 flushed between timed steps (258 MB write); CSR "
                         f"{(graph_nnz * 8 + graph_n * 8) / 1e9:.1f} GB > L2"},
        "roofline": roofline, "roofline_step": roofline_step,
        "roofline_coarsen": roofline_coarsen, "cpu_baseline": cpu,
        "kernels_ms_per_step": {
            (KERNEL_NAMES[b] if b != 5 or tuned_bins[5] > 6144 else "k_move_cta<512>"): {"ms": round(a["time_ms"] / prof_steps, 4),
                              "launches": a["launches"] // prof_steps,
                              "GB/s": round(a["alg_bytes"] / (a["time_ms"] / 1000.0) / 1e9, 1)
                              if a["time_ms"] > 0 else None}
            for b, a in sorted(bins_acc.items()) if a["launches"]},
        "coarsen_ms_per_step": round(coarsen_ms / prof_steps, 4),
        "kernel_timing": {"runs": prof_steps, "ms_per_run": prof_ms / prof_steps,
                          "note": "kernels_ms_per_step, coarsen_ms_per_step and the roofline "
                                  "come from profiled runs right after the timed region: "
                                  "per-bin CUDA events on each kernel's stream, bins one after "
                                  "another (timed alone), same bins; the timed steps run the "
                                  "default mode (CUDA-graph sweep loops, bins on 4 concurrent "
                                  "streams)"},
        "e2e": e2e,
        "batch": batch, "serve": serve, "edges": edges,
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
