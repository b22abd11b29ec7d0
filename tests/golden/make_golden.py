"""Write the stored expected results of the large named workloads.

Every value here comes from the CPU oracle (oracle/) run on the seeded
generator's graph; nothing comes from the GPU engine. Each file also records a
fingerprint of the graph so that a test can confirm the generator produced the
same graph on another machine.

    python tests/golden/make_golden.py er_2000 chunglu_1m ...
    python tests/golden/make_golden.py work batch_4096   # adds per-width work to a batch file
    python tests/golden/make_golden.py roots rmat_22     # per-root results of a banded root sample
    python tests/golden/make_golden.py subset rmat_22 8  # every root with at most 8 words per row

Batched workloads (batch_*) store per-graph count, hash, largest size and
histogram instead (see make_batch). Per single-graph workload, <name>.json holds: fingerprint (n, m, sha256 of row_ptr and
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


def make_batch(name, threads=0):
    """Per-graph results of a batched workload. Each graph is a G(n,p) part
    plus, for some, a disjoint Moon-Moser block; the parts are separate
    components, so per-graph results are the sums of the parts':
      * G(n,p) part: count and hash from one oracle run over all such roots
        (per-root results summed per graph, hashes on the batch's ids), and
        the histogram from the part alone (sizes do not depend on ids);
      * Moon-Moser block: oracle_multipartite (all transversals enumerated).
    """
    b = gen.workload(name)
    gp, mm = b.graph_ptr, b.mm_sizes
    G = len(gp) - 1
    gnp_roots = np.concatenate([np.arange(gp[i], gp[i + 1] - mm[i], dtype=np.int32) for i in range(G)])
    t0 = time.time()
    r = oracle.mce(b.row_ptr, b.col, mode=oracle.PIVOT_IP, threads=threads, roots=gnp_roots, per_root=True)
    graphs = []
    total_c, total_h = 0, 0
    for i in range(G):
        a, z = int(gp[i]), int(gp[i + 1])
        ng = z - a - int(mm[i])
        cnt = int(r.root_count[a:a + ng].astype(np.uint64).sum())
        hsh = int(r.root_hash[a:a + ng].astype(object).sum()) & ((1 << 64) - 1)
        # the part alone (ids 0..ng-1) for its histogram
        rp = b.row_ptr[a:a + ng + 1] - b.row_ptr[a]
        col = b.col[b.row_ptr[a]:b.row_ptr[a + ng]] - a
        part = oracle.mce(rp, col, mode=oracle.PIVOT_IP, threads=1)
        assert part.count == cnt
        hist = {int(k): int(v) for k, v in enumerate(part.hist) if v}
        if mm[i]:
            k = int(mm[i]) // 3
            c2, h2 = oracle.multipartite(a + ng, k, 3)
            cnt += c2
            hsh = (hsh + h2) & ((1 << 64) - 1)
            hist[k] = hist.get(k, 0) + c2
        graphs.append({"count": cnt, "hash": "0x%016x" % hsh, "max_size": max(hist) if hist else 0,
                       "hist": {str(k): v for k, v in sorted(hist.items())}})
        total_c += cnt
        total_h = (total_h + hsh) & ((1 << 64) - 1)
    out = {"workload": name,
           "source": "CPU oracle: Bron-Kerbosch (pivot from P u X_P) on the G(n,p) parts, "
                     "oracle_multipartite on the Moon-Moser blocks, on gen.workload(%r)" % name,
           "fingerprint": fingerprint(b), "graph_ptr_sha256": hashlib.sha256(gp.astype(np.int32).tobytes()).hexdigest(),
           "G": G, "count": total_c, "hash": "0x%016x" % total_h, "graphs": graphs,
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f)
    print(name, total_c, out["hash"], "%.1fs" % out["oracle_seconds"], flush=True)


RMAT_BANDS = [(1, 1), (2, 2), (3, 4), (5, 8), (9, 12), (13, 16), (17, 20), (21, 24), (25, 28), (29, 31)]


def make_root_sample(name, per_band=40, node_cap=200000, wide_from=9, wide_draw=48, wide_cap=4000000, threads=0,
                     seed=17):
    """Per-root oracle results for a seeded sample of roots in every row-width
    band W = ceil(|P0| / 32) of a graph too large to enumerate whole. Within a
    band, 8 x per_band roots are drawn at random (wide_draw in the bands from
    W = wide_from on, whose subtrees are far larger) and walked by the oracle
    with a cap of node_cap (wide_cap) Bron-Kerbosch calls per root
    (oracle_mce_capped); of the roots that finish, per_band are kept at
    random, with their count, hash and tree nodes (pivot from P u X_P). A band
    where no drawn root finishes is left out."""
    g = gen.workload(name)
    core, rank, order, rounds = oracle.peel(g.row_ptr, g.col)
    outd = later_degree(g, rank)
    W = (outd + 31) // 32
    rs = np.random.default_rng(seed)
    t0 = time.time()
    chosen, bands = [], {}
    cnt, hsh, nds = [], [], []
    for lo, hi in RMAT_BANDS:
        ids = np.nonzero((W >= lo) & (W <= hi))[0].astype(np.int32)
        if len(ids) == 0:
            continue
        wide = lo >= wide_from
        draw = wide_draw if wide else 8 * per_band
        cand = np.sort(rs.choice(ids, size=min(len(ids), draw), replace=False)).astype(np.int32)
        c, h, nd = oracle.capped(g.row_ptr, g.col, cand, wide_cap if wide else node_cap, mode=oracle.PIVOT_IP,
                                 threads=threads)
        ok = cand[nd[cand] != np.iinfo(np.uint64).max]
        pick = np.sort(rs.choice(ok, size=min(len(ok), per_band), replace=False)).astype(np.int32)
        chosen.append(pick)
        cnt.append(c[pick])
        hsh.append(h[pick])
        nds.append(nd[pick])
        bands["%d-%d" % (lo, hi)] = {"roots_in_band": int(len(ids)), "drawn": int(len(cand)),
                                    "finished_within_cap": int(len(ok)), "stored": int(len(pick))}
        print(name, lo, hi, bands["%d-%d" % (lo, hi)], "%.0fs" % (time.time() - t0), flush=True)
    roots = np.concatenate(chosen)
    rc, rh, rn = np.concatenate(cnt), np.concatenate(hsh), np.concatenate(nds)
    out = {"workload": name,
           "source": "CPU oracle (oracle/oracle.c, oracle_mce_capped), pivot from P u X_P, per root, on a seeded "
                     "sample of gen.workload(%r) roots in every row-width band (tests/golden/make_golden.py)" % name,
           "fingerprint": fingerprint(g), "selection": {"per_band": per_band, "node_cap": node_cap,
                                                        "wide_from": wide_from, "wide_draw": wide_draw,
                                                        "wide_cap": wide_cap, "seed": seed, "bands": bands},
           "roots": roots.tolist(), "W": W[roots].tolist(),
           "root_count": rc.astype(np.uint64).tolist(),
           "root_hash": ["0x%016x" % int(x) for x in rh],
           "root_nodes": rn.astype(np.uint64).tolist(),
           "count": int(rc.astype(np.uint64).sum()),
           "hash": "0x%016x" % (int(sum(int(x) for x in rh)) & ((1 << 64) - 1)),
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, name + "_roots.json"), "w") as f:
        json.dump(out, f)
    print(name, "sample of", len(roots), "roots:", out["count"], "cliques", "%.0fs" % out["oracle_seconds"])


def make_subset(name, max_w, threads=0):
    """Oracle results of every first-level subtree whose root has at most
    max_w words per row (|P0| <= 32 max_w; roots without later neighbours
    included): count, hash, histogram, tree nodes and per-width work (pivot
    from P u X_P), written to <name>_w<max_w>.json."""
    g = gen.workload(name)
    core, rank, order, rounds = oracle.peel(g.row_ptr, g.col)
    outd = later_degree(g, rank)
    W = (outd + 31) // 32
    roots = np.nonzero(W <= max_w)[0].astype(np.int32)
    t0 = time.time()
    hl = int(outd.max()) + 2
    r = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, threads=threads, roots=roots, hist_len=hl)
    t_mce = time.time() - t0
    rn, rw = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_IP, threads=threads, roots=roots)
    by_w_nodes, by_w_work = {}, {}
    for w in np.unique(W[roots]):
        sel = np.zeros(g.n, bool)
        sel[roots] = True
        sel &= W == w
        by_w_nodes[int(w)] = int(rn[sel].astype(np.uint64).sum())
        by_w_work[int(w)] = int(rw[sel].astype(np.uint64).sum())
    out = {"workload": "%s_w%d" % (name, max_w),
           "source": "CPU oracle (oracle/oracle.c), pivot from P u X_P, on the roots of gen.workload(%r) with at "
                     "most %d words per row" % (name, max_w),
           "fingerprint": fingerprint(g), "max_w": max_w, "roots": int(len(roots)),
           "count": r.count, "hash": "0x%016x" % r.hash, "max_size": r.max_size,
           "hist": [int(x) for x in r.hist], "degeneracy": int(core.max()),
           "tree_nodes": int(sum(by_w_nodes.values())), "word_ops": int(sum(by_w_work.values())),
           "nodes_by_W": by_w_nodes, "word_ops_by_W": by_w_work,
           "oracle_seconds": round(t_mce, 2), "oracle_threads": threads if threads > 0 else oracle.default_threads()}
    with open(os.path.join(HERE, "%s_w%d.json" % (name, max_w)), "w") as f:
        json.dump(out, f, indent=1)
    print(out["workload"], out["count"], out["hash"], "%.1fs" % t_mce, flush=True)


def add_batch_work(name, threads=0):
    """Add the oracle's tree nodes and bitset word-ops per row width W to a
    stored batch file (pivot from P u X_P): the G(n,p) parts by one oracle
    walk over their roots; each Moon-Moser block by a walk of one block of
    that size alone, times the number of such blocks (a block's subtrees do
    not depend on where its ids start: its peel order is the same)."""
    b = gen.workload(name)
    gp, mm = b.graph_ptr, b.mm_sizes
    G = len(gp) - 1
    path = os.path.join(HERE, name + ".json")
    with open(path) as f:
        out = json.load(f)
    assert out["fingerprint"] == fingerprint(b)
    t0 = time.time()
    gnp_roots = np.concatenate([np.arange(gp[i], gp[i + 1] - mm[i], dtype=np.int32) for i in range(G)])
    core, rank, order, rounds = oracle.peel(b.row_ptr, b.col)
    rn, rw = oracle.work(b.row_ptr, b.col, mode=oracle.PIVOT_IP, threads=threads, roots=gnp_roots)
    W = (later_degree(b, rank) + 31) // 32
    by_w_nodes, by_w_work = {}, {}

    def add(w, nodes, work):
        by_w_nodes[w] = by_w_nodes.get(w, 0) + int(nodes)
        by_w_work[w] = by_w_work.get(w, 0) + int(work)

    sel = np.zeros(b.n, bool)
    sel[gnp_roots] = True
    for w in np.unique(W[sel]):
        s = sel & (W == w)
        add(int(w), rn[s].astype(np.uint64).sum(), rw[s].astype(np.uint64).sum())
    for size in sorted(set(int(x) for x in mm if x)):
        blk = gen.moon_moser(size // 3)
        bn, bw = oracle.work(blk.row_ptr, blk.col, mode=oracle.PIVOT_IP, threads=threads)
        _, brank, _, _ = oracle.peel(blk.row_ptr, blk.col)
        bW = (later_degree(blk, brank) + 31) // 32
        times = int((mm == size).sum())
        for w in np.unique(bW):
            s = bW == w
            add(int(w), int(bn[s].astype(np.uint64).sum()) * times, int(bw[s].astype(np.uint64).sum()) * times)
    out["tree_nodes_ip"] = sum(by_w_nodes.values())
    out["word_ops"] = sum(by_w_work.values())
    out["nodes_by_W"] = {str(k): v for k, v in sorted(by_w_nodes.items())}
    out["word_ops_by_W"] = {str(k): v for k, v in sorted(by_w_work.items())}
    out["work_seconds"] = round(time.time() - t0, 1)
    with open(path, "w") as f:
        json.dump(out, f)
    print(name, "tree nodes", out["tree_nodes_ip"], "word-ops", out["word_ops"], "%.1fs" % out["work_seconds"])


if __name__ == "__main__":
    args = sys.argv[1:]
    if args and args[0] == "work":
        for name in args[1:]:
            add_batch_work(name)
        sys.exit(0)
    if args and args[0] == "subset":
        make_subset(args[1], int(args[2]))
        sys.exit(0)
    if args and args[0] == "roots":
        for name in args[1:]:
            make_root_sample(name)
        sys.exit(0)
    for name in args:
        if name.startswith("batch_"):
            make_batch(name)
        else:
            make(name)
