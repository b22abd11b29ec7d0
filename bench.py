#!/usr/bin/env python
"""Maximal cliques/sec of the GB300 engine on a seeded synthetic workload.

One step = the whole hot path on one graph: mce_create (CSR validation,
degeneracy peel, orientation into per-root P/X lists) + mce_run (the
persistent Bron-Kerbosch traversal of every first-level subtree), with the
CSR already resident in HBM. Default workload: Chung-Lu n=1,000,000, mean
degree 16, exponent 2.1, weight cap 20,000, 50 planted cliques of size
U[20,40], seed 1 (chunglu_1m).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). With torchrun and N > 1 every rank runs an
independent replica of the workload on its own GPU (the method shards by root
with no exchange; replicas need no collective beyond the timing barrier).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WP_CLASSES = [1, 2, 4, 12, 20, 28, 36, 68, 132]
WORK_TEXT = ("bitset word-ops of the oracle-counted Bron-Kerbosch tree (pivot rule IP), counted as one op per "
             "32-bit word intersected and counted (AND + POPC + the accumulating add); the pivot scan is counted "
             "up to the first candidate that reaches the largest score possible, as the kernel stops there")
BYTES_TEXT = ("algorithmic bytes: per root v of the launch, 4 x (deg(v) + sum over u in N(v) of |later(u)|), "
              "the oriented adjacency lists that building the root's bitset rows A and X_X reads, "
              "each once per root, with no reuse across roots")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chunglu_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=float, default=0.05,
                    help="fraction of roots (seeded) the CPU oracle runs for its baseline")
    ap.add_argument("--pivot", default="auto", choices=["auto", "ip", "ipx"],
                    help="pivot rule of the timed steps (auto = the Sec. IV-E heuristic)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the learned-order and batched comparisons")
    return ap.parse_args()


def split_workload(name):
    """'rmat_22_w8' -> ('rmat_22', 8): the first-level subtrees of the roots
    with at most 8 words per row (|P0| <= 256) of rmat_22; plain names -> (name, None)."""
    base, _, tail = name.rpartition("_w")
    if base and tail.isdigit():
        return base, int(tail)
    return name, None


def subset_roots(outd, max_w):
    """Input ids of the roots with at most max_w words per row (roots without
    later neighbours included), int32."""
    import numpy as np
    return np.nonzero((outd.astype(np.int64) + 31) // 32 <= max_w)[0].astype(np.int32)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


TRAVERSAL_SOURCES = ("mce_traverse.cuh", "mce_trav_inst.cuh", "mce_internal.cuh", "mce_trav_mid.cu")


def traversal_source_hash():
    """sha256 over the sources that define the traversal kernels."""
    import hashlib
    h = hashlib.sha256()
    for name in TRAVERSAL_SOURCES:
        with open(os.path.join(ROOT, "paper_2212_01473_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def replica_throughput(count, steps, total_ms, dist=None, device="cpu"):
    """Whole-job rate of N independent replicas (the path does not shard: each
    rank enumerates the same graph). Every rank ran `steps` steps of `count`
    cliques; the job lasts as long as its slowest rank. Returns (cliques/s
    over all ranks, the slowest rank's total ms)."""
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return count * steps * world / (total_ms / 1e3), total_ms


def load_golden(name):
    p = os.path.join(ROOT, "tests", "golden", name + ".json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def wp_of_words(w):
    for c in WP_CLASSES:
        if w <= c:
            return c
    return None


def launch_word_ops(word_ops_by_W, wp_lo, wp_hi):
    """Word-ops of the roots whose rows fall in width classes wp_lo..wp_hi.

    word_ops_by_W maps str(W) -> the oracle's word-op count of the roots with
    W = ceil(|P0| / 32) words per row (W = 0: roots without later
    neighbours, which no traversal launch runs)."""
    return sum(v for w, v in word_ops_by_W.items() if int(w) > 0 and wp_lo <= wp_of_words(int(w)) <= wp_hi)


def launch_bytes(g, outd, wp_lo, wp_hi, roots=None):
    """Algorithmic bytes (BYTES_TEXT) of the roots (all, or those listed) whose
    row width falls in width classes wp_lo..wp_hi (roots with |P0| = 0 run in
    no launch)."""
    import numpy as np
    deg = np.diff(g.row_ptr).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    per_root = deg + np.bincount(src, weights=outd[g.col].astype(np.float64), minlength=g.n).astype(np.int64)
    W = (outd.astype(np.int64) + 31) // 32
    cls = np.array([wp_of_words(int(w)) or 0 for w in range(int(W.max()) + 1)])
    wp = cls[W]
    sel = (outd > 0) & (wp >= wp_lo) & (wp <= wp_hi)
    if roots is not None:
        keep = np.zeros(g.n, bool)
        keep[roots] = True
        sel &= keep
    return 4 * int(per_root[sel].sum())


def measure_peaks():
    """The roofline's denominators, measured on this GPU by the library's
    microbenchmarks (mce_microbench) with the SM clock seen meanwhile, plus
    the measured HBM copy bandwidth of MEASURED_PEAKS.json."""
    import paper_2212_01473_gb300 as mce
    wo, lop, l2 = (mce.mce_microbench(i) for i in range(3))
    hbm = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            hbm = json.load(f).get("hbm_gbs")
    return {"word_ops_per_s": wo["rate"], "word_ops_sm_mhz": wo["sm_mhz"], "lop3_per_s": lop["rate"],
            "lop3_sm_mhz": lop["sm_mhz"], "l2_read_gbs": l2["rate"] / 1e9, "l2_sm_mhz": l2["sm_mhz"],
            "hbm_gbs": hbm, "hbm_source": "MEASURED_PEAKS.json (driver-measured copy)" if hbm else None,
            "how": "mce_microbench: word-ops = AND+POPC+add over independent register pairs, 4 x 256 threads "
                   "per SM; L2 = 40 passes over 64 MiB with ld.global.cg; each timed by CUDA events after a warm-up"}


def roofline_legs(words, nbytes, ms, peaks):
    """Integer-pipe, HBM and L2 legs of one launch; the binding one is the
    leg with the largest fraction of its peak."""
    sec = ms / 1e3
    legs = {}
    if words is not None:
        a = words / sec / 1e9
        legs["alu"] = {"achieved": a, "peak": peaks["word_ops_per_s"] / 1e9, "unit": "G word-ops/s",
                       "frac": a / (peaks["word_ops_per_s"] / 1e9), "work": words}
    if nbytes is not None:
        a = nbytes / sec / 1e9
        if peaks.get("hbm_gbs"):
            legs["hbm"] = {"achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": a / peaks["hbm_gbs"], "bytes": nbytes}
        legs["l2"] = {"achieved": a, "peak": peaks["l2_read_gbs"], "unit": "GB/s",
                      "frac": a / peaks["l2_read_gbs"], "bytes": nbytes}
    bound = max(legs, key=lambda k: legs[k]["frac"]) if legs else None
    return bound, legs


def dominant_launch_ms(mce, h, opts, steps, flush_buf):
    """Runs `opts` 1 + steps times (L2 flushed before each); returns the
    longest launch of the last run, its mean duration over the timed runs (CUDA
    events on the handle's stream) and the last result."""
    import statistics
    lst, r = [], None
    batched = mce.mce_graph_info(h)["G"] > 1
    for _ in range(1 + steps):
        flush_buf.zero_()
        r = mce.mce_run_batch(h, opts)[2] if batched else mce.mce_run(h, opts)
        st = mce.mce_get_stats(h)
        lst.append(max(st["classes"], key=lambda c: c["ms"]))
    dom = lst[-1]
    same = [c["ms"] for c in lst[1:] if c["wp"] == dom["wp"]]
    return dom, statistics.mean(same), r


def later_degrees(g, rank):
    """|P0| of every root from a degeneracy rank (numpy)."""
    import numpy as np
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return np.bincount(src[rank[g.col] > rank[src]], minlength=g.n)


def cpu_baseline(g, frac, seed=12345, reps=3, single_frac=None, pool=None):
    """The CPU oracle as it stands, on a seeded uniform sample of roots (of
    `pool`, the workload's root subset, when given): the median of `reps`
    runs on every host core, and one single-threaded run on a smaller sample
    (single_frac, default frac / 10)."""
    import numpy as np
    import oracle
    rs = np.random.default_rng(seed)
    ids = np.arange(g.n, dtype=np.int32) if pool is None else np.asarray(pool, np.int32)
    k = max(1, int(round(frac * len(ids))))
    roots = np.sort(rs.choice(ids, size=k, replace=False)).astype(np.int32)
    threads = oracle.default_threads()
    secs, r = [], None
    for _ in range(max(1, reps)):
        t0 = time.perf_counter()
        r = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, threads=threads, roots=roots)
        secs.append(time.perf_counter() - t0)
    dt = statistics.median(secs)
    out = {"value": r.count / dt, "unit": "cliques/s", "cores": threads, "kind": "oracle", "seconds": dt,
           "sample": "%d of %d roots (%.1f%%, seed %d), %d cliques; median of %d runs of %.2f s each incl. "
                     "validation, peel and relabelling" % (k, len(ids), 100.0 * frac, seed, r.count, len(secs), dt)}
    sf = frac / 10 if single_frac is None else single_frac
    if sf > 0:
        k1 = max(1, int(round(sf * len(ids))))
        roots1 = np.sort(np.random.default_rng(seed + 1).choice(ids, size=k1, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        r1 = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, threads=1, roots=roots1)
        d1 = time.perf_counter() - t0
        out["single_thread"] = {"value": r1.count / d1, "unit": "cliques/s", "cores": 1, "seconds": d1,
                                "sample": "%d of %d roots (%.2f%%, seed %d), %d cliques" % (
                                    k1, len(ids), 100.0 * sf, seed + 1, r1.count)}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import gen
    base, max_w = split_workload(args.workload)
    g = gen.workload(base)
    frac = args.cpu_sample
    pool = None
    if max_w is not None:
        import oracle
        _, rank, _, _ = oracle.peel(g.row_ptr, g.col)
        pool = subset_roots(later_degrees(g, rank), max_w)
    vals, secs = [], []
    info = None
    for it in range(args.warmup + args.steps):
        b = cpu_baseline(g, frac, reps=1, single_frac=0, pool=pool)
        if it >= args.warmup:
            vals.append(b["value"])
            secs.append(b["seconds"])
            info = b
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "maximal cliques/sec", "value": value, "unit": "cliques/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "step": "CPU oracle on a seeded %.0f%% sample of roots" % (100 * frac)},
            "cpu_baseline": {"kind": "oracle", "cores": info["cores"], "sample": info["sample"], "value": value,
                             "unit": "cliques/s"},
            "e2e": {"value": value, "unit": "cliques/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def form_roofline(mce, h, opts, g, golden, peaks, steps, flush_buf, nodes_key="tree_nodes"):
    """Roofline legs of the dominant launch of `opts` (pivot rule IP) on handle h."""
    _, _, outd = mce.mce_get_order(h)
    dom, kms, r = dominant_launch_ms(mce, h, opts, steps, flush_buf)
    lo = dom.get("wp_min") or dom["wp"]
    words = None
    if golden and golden.get("word_ops_by_W") and r.tree_nodes == golden.get(nodes_key):
        words = launch_word_ops(golden["word_ops_by_W"], lo, dom["wp"])
    bound, legs = roofline_legs(words, launch_bytes(g, outd, lo, dom["wp"]), kms, peaks)
    top = legs[bound]
    return {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
            "frac": top["frac"], "kernel_ms": kms, "legs": legs,
            "kernel": "k_traverse<WP=%d,GW=%d> (pivot rule IP; width classes %d..%d words)" % (
                dom["wp"], dom["group_warps"], lo, dom["wp"])}


def measure_forms(args, rp_d, col_d, count, value_plain, flush_buf, g=None, peaks=None, forms=None):
    """Learned root order on the same workload, and the 4096-graph batch run
    batched (one set of persistent launches, replayed from a CUDA graph) versus
    graph by graph, all on this GPU."""
    import numpy as np
    import torch
    import gen
    import paper_2212_01473_gb300 as mce
    from paper_2212_01473_gb300 import learn
    # filled in place, so that what was measured survives a later failure
    forms = {} if forms is None else forms
    forms["plain"] = {"value": value_plain, "unit": "cliques/s"}
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            flush_buf.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, out

    # learned order: features + network + traversal in the step
    model, meta = learn.load()

    def learned_step():
        h = mce.mce_create(rp_d, col_d)
        pr = learn.priority(model, h)
        o = mce.mce_default_opts(order=mce.MCE_ORDER_PRIORITY)
        o.root_priority = pr.data_ptr()
        r = mce.mce_run(h, o)
        mce.mce_destroy(h)
        return r

    timed(learned_step, 1)
    ms, r = timed(learned_step, args.steps)
    assert r.count == count
    forms["learned"] = {"value": count * args.steps / (sum(ms) / 1e3), "unit": "cliques/s",
                        "ms_per_step": sum(ms) / len(ms), "vs_plain": count * args.steps / (sum(ms) / 1e3) / value_plain,
                        "model": "paper_2212_01473_gb300/work_model.json (%s)" % meta.get("train", "")}
    if peaks is not None:
        golden = load_golden(args.workload)
        h = mce.mce_create(rp_d, col_d)
        pr = learn.priority(model, h)
        o = mce.mce_default_opts(order=mce.MCE_ORDER_PRIORITY, pivot=mce.MCE_PIVOT_IP)
        o.root_priority = pr.data_ptr()
        forms["learned"]["roofline"] = form_roofline(mce, h, o, g, golden, peaks, args.steps, flush_buf)
        forms["plain"]["roofline"] = form_roofline(mce, h, mce.mce_default_opts(pivot=mce.MCE_PIVOT_IP), g, golden,
                                                   peaks, args.steps, flush_buf)
        mce.mce_destroy(h)
    model.close()

    # batched versus graph by graph
    b = gen.workload("batch_4096")
    gp, rp, col = (torch.from_numpy(x).cuda() for x in (b.graph_ptr, b.row_ptr, b.col))

    def batched_step():
        h = mce.mce_batch_create(gp, rp, col)
        per, hist, tot = mce.mce_run_batch(h)
        mce.mce_destroy(h)
        return tot

    timed(batched_step, 1)
    ms_b, tot = timed(batched_step, 2)
    hb = mce.mce_batch_create(gp, rp, col)
    tune = mce.mce_autotune(hb, budget_ms=8000.0)
    # one run with the tuned settings, launched directly: its kernel launches,
    # and the host time around it beyond its device time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, rd = mce.mce_run_batch(hb, mce.mce_default_opts(tuned=1))
    wall_d = (time.perf_counter() - t0) * 1e3
    launches_direct = mce.mce_get_stats(hb)["kernel_launches"]
    mce.mce_prepare(hb, mce.mce_default_opts(tuned=1))
    mce.mce_run_prepared(hb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, rp_ = mce.mce_run_prepared(hb)
    wall_r = (time.perf_counter() - t0) * 1e3
    ms_r, rr = timed(lambda: mce.mce_run_prepared(hb)[2], 2)
    assert rr.count == tot.count and rr.hash == tot.hash and rd.count == tot.count
    b_roof = None
    if peaks is not None:
        b_roof = form_roofline(mce, hb, mce.mce_default_opts(pivot=mce.MCE_PIVOT_IP), b, load_golden("batch_4096"),
                               peaks, 2, flush_buf, nodes_key="tree_nodes_ip")
    mce.mce_destroy(hb)
    parts = []
    for i in range(len(b.graph_ptr) - 1):
        a, z = int(b.graph_ptr[i]), int(b.graph_ptr[i + 1])
        sub_rp = torch.from_numpy((b.row_ptr[a:z + 1] - b.row_ptr[a]).astype(np.int32)).cuda()
        sub_col = torch.from_numpy((b.col[b.row_ptr[a]:b.row_ptr[z]] - a).astype(np.int32)).cuda()
        parts.append((sub_rp, sub_col))

    def one_by_one():
        c = 0
        for sub_rp, sub_col in parts:
            h = mce.mce_create(sub_rp, sub_col)
            c += mce.mce_run(h).count
            mce.mce_destroy(h)
        return c

    ms_1, c1 = timed(one_by_one, 1)
    assert c1 == tot.count
    v_b = tot.count * len(ms_b) / (sum(ms_b) / 1e3)
    v_r = tot.count * len(ms_r) / (sum(ms_r) / 1e3)
    v_1 = c1 / (ms_1[0] / 1e3)
    forms["batched"] = {"workload": "batch_4096", "maximal_cliques": tot.count,
                        "value": v_b, "unit": "cliques/s", "ms_per_step": sum(ms_b) / len(ms_b),
                        "step": "mce_batch_create + mce_run_batch over all 4096 graphs",
                        "replay_value": v_r, "replay_ms": sum(ms_r) / len(ms_r),
                        "replay": "autotuned launch settings, run captured once and replayed as one CUDA graph",
                        "tuning": tune,
                        "direct": {"kernel_launches": launches_direct, "wall_ms": wall_d,
                                   "device_ms": rd.ms_traverse, "host_ms": wall_d - rd.ms_traverse},
                        "replayed": {"graph_launches": 1, "wall_ms": wall_r, "device_ms": rp_.ms_traverse,
                                     "host_ms": wall_r - rp_.ms_traverse},
                        "one_by_one_value": v_1, "one_by_one_ms": ms_1[0],
                        "vs_one_by_one": v_b / v_1}
    if b_roof is not None:
        forms["batched"]["roofline"] = b_roof
    return forms


def run_ours(args):
    import numpy as np
    import torch
    import gen
    import paper_2212_01473_gb300 as mce
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the engine has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    base, max_w = split_workload(args.workload)
    g = gen.workload(base)
    rp_d = torch.from_numpy(g.row_ptr).cuda()
    col_d = torch.from_numpy(g.col).cuda()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    pivot = {"auto": mce.MCE_PIVOT_AUTO, "ip": mce.MCE_PIVOT_IP, "ipx": mce.MCE_PIVOT_IPX}[args.pivot]
    roots_np, roots_d = None, None
    if max_w is not None:
        # a root subset: the roots with at most max_w words per row, found once
        h = mce.mce_create(rp_d, col_d)
        roots_np = subset_roots(mce.mce_get_order(h)[2], max_w)
        mce.mce_destroy(h)
        roots_d = torch.from_numpy(roots_np).cuda()

    def opts(**kw):
        o = mce.mce_default_opts(**kw)
        if roots_d is not None:
            o.roots = roots_d.data_ptr()
            o.n_roots = len(roots_np)
        return o

    def step():
        h = mce.mce_create(rp_d, col_d)
        r = mce.mce_run(h, opts(pivot=pivot))
        st = mce.mce_get_stats(h)
        mce.mce_destroy(h)
        return r, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    ms, results, stats = [], [], []
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    try:
        for _ in range(args.steps):
            flush_buf.zero_()  # evict the CSR from the 129 MB L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r, st = step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            results.append(r)
            stats.append(st)
        torch.cuda.synchronize()
        barrier()
    finally:
        clk = clocks.stop()  # the sampler never outlives the timed region
    count = results[-1].count
    assert all(r.count == count and r.hash == results[-1].hash for r in results)
    value, total_ms = replica_throughput(count, args.steps, sum(ms), dist, "cuda")

    st = stats[-1]

    # ---- end to end through the C ABI from pinned host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    e2e_s = []
    hl = results[-1].degeneracy + 2
    for _ in range(args.steps):
        flush_buf.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = mce.mce_create(rp_h, col_h)
        r = mce.mce_run(h, opts(pivot=pivot), hist_len=hl)
        t1 = time.perf_counter()
        mce.mce_destroy(h)
        assert r.count == count
        e2e_s.append(t1 - t0)
    h2d = (g.n + 1 + 2 * g.m) * 4
    d2h = 64 + 8 * hl
    e2e = {"value": count * args.steps * world / sum(e2e_s), "unit": "cliques/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- roofline of the dominant traversal launch: integer-pipe leg
    # (oracle word-ops) and memory legs (algorithmic bytes) against peaks
    # measured here. The oracle counts work on the tree of the partial-
    # induced-subgraph pivot rule (IP), so the roofline is taken on IP runs of
    # the same workload; the timed steps above use the default rule (AUTO).
    peaks = measure_peaks()
    h = mce.mce_create(rp_d, col_d)
    _, _, outd = mce.mce_get_order(h)
    dom, kms, r_ip = dominant_launch_ms(mce, h, opts(pivot=mce.MCE_PIVOT_IP), args.steps, flush_buf)
    mce.mce_destroy(h)
    golden = load_golden(args.workload)
    lo = dom.get("wp_min") or dom["wp"]
    words = None
    if golden and golden.get("count") == count and r_ip.tree_nodes == golden.get("tree_nodes"):
        words = launch_word_ops(golden["word_ops_by_W"], lo, dom["wp"])
    nbytes = launch_bytes(g, outd, lo, dom["wp"], roots_np)
    bound, legs = roofline_legs(words, nbytes, kms, peaks)
    top = legs[bound]
    roofline = {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                "frac": top["frac"], "traffic": None,
                "kernel": "k_traverse<WP=%d,GW=%d> (pivot rule IP; roots of width classes %d..%d words)" % (
                    dom["wp"], dom["group_warps"], lo, dom["wp"]),
                "kernel_ms": kms, "legs": legs, "peaks": peaks,
                "peak_basis": "measured on this GPU by mce_microbench (alu, l2); HBM from MEASURED_PEAKS.json",
                "work": WORK_TEXT + " (tests/golden/%s.json word_ops_by_W)" % args.workload, "bytes": BYTES_TEXT}
    prof = os.path.join(ROOT, "profiles", "traffic_%s.json" % args.workload)
    if os.path.exists(prof):
        with open(prof) as f:
            tr = json.load(f)
        # counters taken on another build of the kernel do not describe this one
        if tr.get("kernel_wp") == dom["wp"] and tr.get("source_sha256") == traversal_source_hash():
            roofline["traffic"] = tr.get("dram_bytes_per_launch")
            roofline["traffic_note"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (%s)" % (
                os.path.relpath(prof, ROOT))
        else:
            roofline["traffic_note"] = "null: the traversal kernel changed since %s was captured" % (
                os.path.relpath(prof, ROOT))

    line = {"metric": "maximal cliques/sec", "value": value, "unit": "cliques/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": g.n, "m": g.m, "degeneracy": results[-1].degeneracy,
                       "maximal_cliques": count, "hash": "0x%016x" % results[-1].hash,
                       "tree_nodes": results[-1].tree_nodes, "donations": results[-1].donations,
                       "pivot": {"auto": "AUTO (Sec. IV-E: IPX when max degree / degeneracy <= 200)",
                                 "ip": "IP (pivot from P u X_P)",
                                 "ipx": "IPX (pivot from P u X)"}[args.pivot],
                       "ms_prep": results[-1].ms_prep, "ms_traverse": results[-1].ms_traverse,
                       "classes": st["classes"], "peel_rounds": st["peel_rounds"],
                       "peel_stages": {"ms": st["peel_stage_ms"], "sub_rounds": st["peel_stage_rounds"],
                                       "stages": "full grid, narrow (16 CTAs), one block",
                                       "narrow_as_cluster": bool(st["peel_cluster"])},
                       "l2": "flushed before every step by a 256 MiB device write",
                       "step": "mce_create (validate, degeneracy peel, orient) + mce_run (traversal) on a "
                               "device-resident CSR",
                       "parallelism": "replicas x%d" % world},
            "gpu_launches": int(stats[-1]["kernel_launches"]) * args.steps,
            "clocks": clk, "e2e": e2e, "roofline": roofline}
    if golden:
        line["config"]["oracle_match"] = golden.get("count") == count and golden.get("hash") == "0x%016x" % results[-1].hash
    if max_w is not None:
        line["config"]["roots"] = "the %d roots with at most %d words per row (|P0| <= %d) of %s, isolated " \
            "vertices included; each step enumerates their first-level subtrees" % (len(roots_np), max_w, 32 * max_w, base)
    if rank == 0 and world == 1 and not args.no_forms and max_w is None:
        # the comparisons come after the headline measurement: an error in one
        # of them is reported in the line instead of losing the line
        forms = {}
        try:
            measure_forms(args, rp_d, col_d, count, value, flush_buf, g, peaks, forms)
        except Exception as exc:  # noqa: BLE001 - reported, not hidden
            forms["error"] = "%s: %s" % (type(exc).__name__, exc)
        line["forms"] = forms
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, args.cpu_sample, pool=roots_np)
    if getattr(args, "retried_after", None):
        line["retried_after"] = args.retried_after
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if dist_env()[1] > 1:
        return run_ours(args)
    # one GPU: an engine error in the measurement (say, a device wait that gave
    # up) makes the whole measurement run once more from the start; the line
    # then names the error it followed
    try:
        return run_ours(args)
    except Exception as exc:  # noqa: BLE001 - reported in the line of the second run
        if type(exc).__name__ != "MCEError":
            raise
        sys.stderr.write("bench.py: %s; measuring once more\n" % exc)
        args.retried_after = "%s: %s" % (type(exc).__name__, exc)
        return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
