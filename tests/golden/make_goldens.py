"""Write the stored oracle results of the full-size workloads (tests/golden/full_*.json).

    python tests/golden/make_goldens.py rmat22 batch512 rmat26 [--workers N] [--scratch DIR]

Calls only the CPU oracle (``oracle/``) and the input generators (``graphgen/``); no
value in these files comes from the CUDA library.  Every run uses the oracle's defaults,
which are also the library's: theta = 1/10^6 (absolute phase and level tests, exact),
at most 1000 sweeps per phase and 64 levels, vertex following before level 0 only.

R-MAT scale 26 takes tens of minutes of one core; with ``--scratch DIR`` the graph is
generated in a child process and saved there (about 17 GB), and the oracle reads it
memory-mapped, holding about 55 GB of host memory at its peak.  The 512-graph batch runs
its graphs in parallel worker processes (spawned, one oracle call per graph).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import fullsize as fs  # noqa: E402


def oracle_record(g, full_trace: bool):
    """Run the oracle on graph g and summarise every recorded level and the trace."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.louvain(g.rp, g.col, g.w)
    dt = time.perf_counter() - t0
    rec = {
        "input_digest": fs.input_digest(g.rp, g.col, g.w),
        "n": int(g.n), "nnz": int(g.nnz), "tw": int(r.tw),
        "edge_visits": int(r.edge_visits), "sweeps": int(r.sweeps),
        "hit_iter_cap": bool(r.hit_iter_cap),
        "levels": [[fs.labels_digest(l.labels), int(l.ncomm), int(l.qn), int(l.qn_init),
                    int(l.iters), int(l.n), int(l.nnz)] for l in r.levels],
        "trace_digest": fs.trace_digest(r.trace),
        "oracle_seconds": round(dt, 2),
    }
    if full_trace:
        rec["trace"] = [[int(a), int(b), int(c), int(d)] for a, b, c, d in r.trace]
    return rec


def _batch_one(args):
    k, params = args
    sys.path[:0] = [ROOT, HERE]
    g = fs.batch_graph(params)
    rec = oracle_record(g, full_trace=False)
    rec["graph"] = k
    rec["kind"] = params[0]
    return rec


def write(name: str, body: dict):
    graphs = body.pop("graphs")
    head = {"_about": ("Oracle results of a full-size synthetic workload, written by "
                       "tests/golden/make_goldens.py (CPU oracle only). Digests are the first "
                       "128 bits of SHA-256: of the input CSR, of the int32 little-endian "
                       "label array of the input vertices after each recorded level, and of "
                       "the sweep trace (level, sweep, moved, Qn per sweep, Algorithm 1). qn "
                       "is (2W)^2 * Q (Eq. 3) as an exact integer."),
            "workload": name, **body, "level_fields": fs.LEVEL_FIELDS}
    tmp = fs.path(name) + ".tmp"
    with open(tmp, "w") as f:
        # one graph per line keeps the file small and its diffs readable
        text = json.dumps(head, indent=1)
        f.write(text[:-2] + ',\n "graphs": [\n')
        f.write(",\n".join(json.dumps(g, separators=(",", ":")) for g in graphs))
        f.write("\n ]\n}\n")
    os.replace(tmp, fs.path(name))
    print(f"wrote {fs.path(name)}", flush=True)


def _generate_to_disk(scale: int, folder: str):
    """Child process: generate the R-MAT graph and save its arrays as .npy files."""
    sys.path[:0] = [ROOT, HERE]
    import numpy as np
    g = fs.rmat_graph(scale)
    for key in ("rp", "col", "w"):
        np.save(os.path.join(folder, f"{key}.npy"), getattr(g, key))


def make_rmat(name: str, scratch: str = ""):
    scale = fs.RMAT[name]
    t0 = time.perf_counter()
    if scratch:
        # generate in a child process and memory-map the saved arrays: the input's pages
        # are then file-backed and can be evicted while the oracle holds its own copy
        import numpy as np
        import graphgen
        folder = os.path.join(scratch, name)
        os.makedirs(folder, exist_ok=True)
        proc = mp.get_context("spawn").Process(target=_generate_to_disk, args=(scale, folder))
        proc.start()
        proc.join()
        if proc.exitcode != 0:
            raise RuntimeError(f"generating {name} failed")
        arrays = [np.load(os.path.join(folder, f"{k}.npy"), mmap_mode="r")
                  for k in ("rp", "col", "w")]
        g = graphgen.Graph(*arrays, name)
    else:
        g = fs.rmat_graph(scale)
    print(f"{name}: generated n={g.n} nnz={g.nnz} in {time.perf_counter() - t0:.1f} s", flush=True)
    rec = oracle_record(g, full_trace=True)
    print(f"{name}: oracle {rec['oracle_seconds']} s, {len(rec['levels'])} levels", flush=True)
    write(name, {"generator": (f"R-MAT scale {scale}, edge factor 16, a=0.57 b=0.19 c=0.19, "
                               f"symmetrised, loops and duplicates dropped, int32 weights "
                               f"uniform in [1,16], seed {scale}"),
                 "graphs": [rec]})


def make_batch(name: str, workers: int):
    params = fs.batch_params(name)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        recs = pool.map(_batch_one, list(enumerate(params)), chunksize=1)
    recs.sort(key=lambda r: r["graph"])
    print(f"{name}: {len(recs)} graphs in {time.perf_counter() - t0:.1f} s", flush=True)
    count, seed = fs.BATCH[name]
    write(name, {"generator": (f"{count} graphs of graphgen.batch_mix_params(seed={seed}): "
                               "sizes log-uniform in [1000, 200000]; even graphs planted "
                               "partition, odd graphs Chung-Lu (exponent 2.1, mean degree 10); "
                               "int32 weights uniform in [1, 8]"),
                 "graphs": recs})


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+", choices=sorted(list(fs.RMAT) + list(fs.BATCH)))
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--scratch", default="",
                    help="folder for the R-MAT arrays (memory-mapped during the oracle run)")
    args = ap.parse_args(argv)
    for name in args.names:
        if name in fs.RMAT:
            make_rmat(name, args.scratch)
        else:
            make_batch(name, args.workers)


if __name__ == "__main__":
    main()
