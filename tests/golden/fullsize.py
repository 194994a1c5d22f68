"""Full-size workloads whose oracle results are stored in this folder, and the digests
that compare them.

Each workload is a seeded synthetic graph (or a family of graphs) built by ``graphgen``;
the stored records are written by ``make_goldens.py``, which runs only the CPU oracle on
them.  The GPU tests rebuild the same graphs, check that the input digest equals the
stored one (so a generator that drifted between machines fails loudly instead of
comparing different graphs), run the library in the benchmark's launch configuration and
compare every recorded level, the sweep trace and the counters with the record.

Nothing here computes any part of community detection: these are input builders and
SHA-256 digests of arrays.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# R-MAT (a=0.57, b=c=0.19), edge factor 16, weights uniform in [1, 16], seed = scale
RMAT = {"rmat22": 22, "rmat26": 26}
# mixed batch: 512 graphs, log-uniform sizes in [1K, 200K], planted partitions and
# Chung-Lu power-law graphs alternating, weights uniform in [1, 8], seed 512
BATCH = {"batch512": (512, 512)}


def path(name: str) -> str:
    return os.path.join(HERE, f"full_{name}.json")


def load(name: str):
    """The stored record of workload `name`, or None when it has not been written."""
    try:
        with open(path(name)) as f:
            return json.load(f)
    except OSError:
        return None


def rmat_graph(scale: int):
    import graphgen as gg
    return gg.rmat(scale, 16, 0.57, 0.19, 0.19, 1, 16, seed=scale)


def batch_params(name: str):
    import graphgen as gg
    count, seed = BATCH[name]
    return gg.batch_mix_params(count, seed=seed)


def batch_graph(params):
    import graphgen as gg
    return gg.batch_mix_graph(params)


# per recorded level: these fields, in this order
LEVEL_FIELDS = ["labels_digest", "ncomm", "qn", "qn_init", "iters", "n", "nnz"]


def _sha(*arrays) -> str:
    """First 128 bits of SHA-256 over the arrays' bytes, as hex."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:32]


def input_digest(rp, col, w) -> str:
    """Digest of row offsets (int64 LE), columns (int32 LE) and weights (int32 LE)."""
    return _sha(np.asarray(rp, "<i8"), np.asarray(col, "<i4"), np.asarray(w, "<i4"))


def labels_digest(labels) -> str:
    return _sha(np.asarray(labels, "<i4"))


def trace_digest(trace) -> str:
    """Digest of the sweep trace [(level, sweep, moved, Qn), ...] as decimal text."""
    text = ";".join(f"{a},{b},{c},{d}" for a, b, c, d in trace)
    return hashlib.sha256(text.encode()).hexdigest()[:32]
