"""Write the stored expected results of the large named workloads.

Every value here comes from the CPU oracle (oracle/) run on the seeded
generator's graph; nothing comes from the GPU engine. Each file also records a
fingerprint of the graph so that a test can confirm the generator produced the
same graph on another machine.

    python tests/golden/make_golden.py er_2000 chunglu_1m ...

Per workload, <name>.json holds: fingerprint (n, m, sha256 of row_ptr and
col), count, hash, hist, max_size, degeneracy, per-width totals of tree nodes
and bitset word operations (oracle_mce_work: W = ceil(|P0|/32) words per row;
the integer-pipe roofline's algorithmic work), the oracle's wall time and
thread count.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402


def fingerprint(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, np.int32).tobytes())
    h.update(np.ascontiguousarray(g.col, np.int32).tobytes())
    return {"n": g.n, "m": g.m, "sha256": h.hexdigest()}


def later_degree(g, rank):
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    return np.bincount(src[rank[g.col] > rank[src]], minlength=g.n)


def make(name, threads=0):
    g = gen.workload(name)
    core, rank, order, rounds = oracle.peel(g.row_ptr, g.col)
    t0 = time.time()
    r = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, threads=threads)
    t_mce = time.time() - t0
    rn, rw = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_IP, threads=threads)
    W = (later_degree(g, rank) + 31) // 32
    by_w_nodes, by_w_work = {}, {}
    for w in np.unique(W):
        sel = W == w
        by_w_nodes[int(w)] = int(rn[sel].astype(np.uint64).sum())
        by_w_work[int(w)] = int(rw[sel].astype(np.uint64).sum())
    out = {
        "workload": name,
        "source": "CPU oracle (oracle/oracle.c), pivot from P u X_P, on gen.workload(%r)" % name,
        "fingerprint": fingerprint(g),
        "count": r.count,
        "hash": "0x%016x" % r.hash,
        "max_size": r.max_size,
        "hist": [int(x) for x in r.hist],
        "degeneracy": int(core.max()) if g.n else 0,
        "peel_rounds": rounds,
        "tree_nodes": int(rn.astype(np.uint64).sum()),
        "word_ops": int(rw.astype(np.uint64).sum()),
        "nodes_by_W": by_w_nodes,
        "word_ops_by_W": by_w_work,
        "oracle_seconds": round(t_mce, 2),
        "oracle_threads": threads if threads > 0 else oracle.default_threads(),
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["count"], out["hash"], "%.1fs" % t_mce, flush=True)


if __name__ == "__main__":
    for name in sys.argv[1:]:
        make(name)
