"""GPU engine vs the CPU oracle, through the C ABI: every result bit-exact.

Compared per graph: clique count, size histogram, 64-bit hash, largest
clique; per root vertex: the subtree's clique count, hash sum and number of
Bron-Kerbosch calls (the engine walks the same tree as the oracle's
pivot-from-P-u-X_P mode, so even the node counts agree); the degeneracy
peel's core numbers and ranks.
"""
import numpy as np
import pytest

import gen
import oracle
from test_oracle import M64, h_clique

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2212_01473_gb300 as mce  # noqa: E402


def run(g, per_root=False, **opts):
    return mce.enumerate_maximal_cliques(g.row_ptr, g.col, per_root=per_root, **opts)


def same(r, o):
    assert r.count == o.count
    assert r.hash == o.hash
    assert r.max_size == o.max_size
    assert np.array_equal(r.hist.astype(np.uint64), o.hist.astype(np.uint64))


# GPU pivot rule -> the oracle mode that walks the same tree: pivot from
# P u X_P (partial induced subgraph) or from all of P u X (full, Tomita)
ORACLE_MODE = {mce.MCE_PIVOT_IP: oracle.PIVOT_IP, mce.MCE_PIVOT_IPX: oracle.PIVOT_FULL}


def check_against_oracle(g, per_root=True, pivot=mce.MCE_PIVOT_IP, **opts):
    o = oracle.mce(g.row_ptr, g.col, mode=ORACLE_MODE[pivot], per_root=per_root)
    opts["pivot"] = pivot
    if per_root:
        r, (rc, rh, rn) = run(g, per_root=True, **opts)
        same(r, o)
        assert np.array_equal(rc, o.root_count)
        assert np.array_equal(rh, o.root_hash)
        assert np.array_equal(rn, o.root_nodes)
        assert r.tree_nodes == int(o.root_nodes.sum())
    else:
        r = run(g, **opts)
        same(r, o)
    return r, o


CLOSED = [gen.complete(1), gen.complete(2), gen.complete(7), gen.empty(5), gen.cycle(4), gen.cycle(3),
          gen.cycle(33), gen.moon_moser(2), gen.moon_moser(6), gen.multipartite(7, 2),
          gen.worked_example(), gen.random_forest(60, 1)]


PIVOTS = [mce.MCE_PIVOT_IP, mce.MCE_PIVOT_IPX]


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
@pytest.mark.parametrize("g", CLOSED, ids=[g.name for g in CLOSED])
def test_closed_forms(g, pivot):
    check_against_oracle(g, pivot=pivot)


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
@pytest.mark.parametrize("n,p,seed", [(30, 0.3, 0), (64, 0.5, 1), (100, 0.2, 2), (150, 0.6, 3),
                                      (300, 0.1, 4), (500, 0.05, 5), (120, 0.85, 6), (1000, 0.02, 7)])
def test_random_graphs(n, p, seed, pivot):
    check_against_oracle(gen.gnp(n, p, seed), pivot=pivot)


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
def test_er_2000_per_root(pivot):
    check_against_oracle(gen.workload("er_2000"), pivot=pivot)


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
def test_chunglu_small_per_root(pivot):
    # hubs: large excluded sets, many X_X pivots under IPX
    check_against_oracle(gen.chung_lu(6000, 20.0, 2.1, 1500.0, 3, 10, 20, 6), pivot=pivot)


@pytest.mark.parametrize("maker", [lambda: gen.workload("er_2000"), lambda: gen.gnp(3000, 0.01, 3),
                                   lambda: gen.moon_moser(8), lambda: gen.random_forest(500, 2),
                                   lambda: gen.chung_lu(20000, 8.0, 2.1, 500.0, 5, 8, 16, 11),
                                   lambda: gen.peel_stages()])
def test_peel_matches_oracle(maker):
    g = maker()
    core_o, rank_o, order_o, _ = oracle.peel(g.row_ptr, g.col)
    h = mce.mce_create(g.row_ptr, g.col)
    core, rank, outd = mce.mce_get_order(h)
    info = mce.mce_graph_info(h)
    mce.mce_destroy(h)
    assert np.array_equal(core, core_o)
    assert np.array_equal(rank, rank_o)
    src = np.repeat(np.arange(g.n), g.degrees())
    later = np.bincount(src[rank_o[g.col] > rank_o[src]], minlength=g.n)
    assert np.array_equal(outd, later)
    assert info["degeneracy"] == (int(core_o.max()) if g.n else 0)
    assert info["max_degree"] == (int(g.degrees().max()) if g.n else 0)


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
@pytest.mark.parametrize("blocks,donate,wl,policy", [(1, 1, 1, 0), (2, 1, 1, 1), (3, 2, 1, 2), (5, 10, 1, 1),
                                                     (4, 1, 0, 0)])
def test_worker_list_interleavings(blocks, donate, wl, policy, pivot):
    # tiny grids force phase 2 early and many donations; results and the
    # tree itself (node counts per root) must not change
    g = gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5)
    r, o = check_against_oracle(g, pivot=pivot, blocks=blocks, donate_min_p=donate, worker_list=wl,
                                donate_policy=policy)
    if wl == 0:
        assert r.donations == 0


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
@pytest.mark.parametrize("blocks,donate", [(2, 3), (8, 10), (0, 0)])
def test_deep_balanced_tree_split(blocks, donate, pivot):
    # K_{3x12} plus a sparse random part: every subtree below depth ~3 has
    # |P| + |X_P| <= 32, so the split across groups must happen inside the
    # one-word (compact) subtrees; the tree must not change
    mm = gen.moon_moser(12)
    g = gen.disjoint_union([gen.gnp(300, 0.03, 7), mm])
    r, o = check_against_oracle(g, pivot=pivot, blocks=blocks, donate_min_p=donate)
    assert r.count > 3 ** 12  # the multipartite block alone holds 3^12 maximal cliques
    if blocks:
        assert r.donations > 0


def check_level2(g, pivot, **opts):
    o = oracle.mce(g.row_ptr, g.col, mode=ORACLE_MODE[pivot], per_root=True, level=2)
    r, (rc, rh, rn) = run(g, per_root=True, pivot=pivot, subtree_level=2, **opts)
    same(r, o)
    assert np.array_equal(rc, o.root_count)
    assert np.array_equal(rh, o.root_hash)
    assert np.array_equal(rn, o.root_nodes)
    assert r.tree_nodes == int(o.root_nodes.sum())
    return r


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
@pytest.mark.parametrize("make", [lambda: gen.complete(12), lambda: gen.worked_example(),
                                  lambda: gen.disjoint_union([gen.gnp(300, 0.05, 11), gen.empty(4), gen.complete(40)]),
                                  lambda: gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5),
                                  lambda: gen.moon_moser(8)])
def test_second_level_subtrees(make, pivot):
    # one subtree per edge (Algorithm 4): results as always, tree nodes per
    # root (summed over its edges) as the oracle's second-level walk
    check_level2(make(), pivot)


@pytest.mark.parametrize("pivot", PIVOTS, ids=["IP", "IPX"])
@pytest.mark.parametrize("blocks,donate", [(1, 1), (3, 2), (8, 10)])
def test_second_level_under_donations(blocks, donate, pivot):
    g = gen.disjoint_union([gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5), gen.moon_moser(9)])
    check_level2(g, pivot, blocks=blocks, donate_min_p=donate)


def test_second_level_listing():
    g = gen.disjoint_union([gen.gnp(250, 0.06, 5), gen.empty(2), gen.moon_moser(5)])
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    cl = mce.list_maximal_cliques(g.row_ptr, g.col, subtree_level=2)
    assert len(cl) == o.count
    assert len({tuple(sorted(c.tolist())) for c in cl}) == o.count
    tot = 0
    for c in cl:
        tot = (tot + h_clique([int(x) for x in c])) & M64
    assert tot == o.hash


def test_worker_list_donates():
    # a deep tree (K_{3x9}) outlasts the other roots, so idle groups take parts of it
    g = gen.disjoint_union([gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5), gen.moon_moser(9)])
    r = run(g, blocks=2, donate_min_p=1)
    assert r.donations > 0


def _complete_minus_matching(n, t):
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    missing = {(2 * k, 2 * k + 1) for k in range(t)}
    g = gen.from_edges(n, [x for x in e if x not in missing])
    # maximal cliques: one endpoint of every removed edge, plus all other vertices
    rest = list(range(2 * t, n))
    cl = []
    for mask in range(1 << t):
        cl.append([2 * k + ((mask >> k) & 1) for k in range(t)] + rest)
    return g, cl


@pytest.mark.parametrize("n,t", [(33, 2), (65, 3), (129, 2), (300, 3), (500, 2), (700, 2), (900, 1),
                                 (1100, 2), (1300, 1), (2300, 1)])
def test_wide_rows_closed_form(n, t):
    # |P0| of the first root is n-1: exercises every bitset width class,
    # including rows kept in global memory
    g, cl = _complete_minus_matching(n, t)
    r = run(g)
    assert r.count == len(cl) == 2 ** t
    assert r.max_size == n - t
    assert r.hash == sum(h_clique(c) for c in cl) & M64
    assert r.hist[n - t] == 2 ** t and int(r.hist.sum()) == 2 ** t


def test_degeneracy_above_the_limit_is_unsupported():
    # K_4098 has degeneracy 4097, one above MCE_MAX_DEGENERACY (4096): create
    # reports MCE_EUNSUPPORTED after the peel instead of running out of row width
    n = 4098
    idx = np.arange(n * n, dtype=np.int64)
    col = (idx % n)[idx % (n + 1) != 0].astype(np.int32)  # row i: every j != i, ascending
    row_ptr = (np.arange(n + 1, dtype=np.int64) * (n - 1)).astype(np.int32)
    with pytest.raises(mce.MCEError) as e:
        mce.mce_create(row_ptr, col)
    assert e.value.code == mce.MCE_EUNSUPPORTED


def test_complete_graph_node_counts():
    # K_n, pivot from P u X_P: root r walks a chain of n - r calls
    n = 200
    g = gen.complete(n)
    r, (rc, rh, rn) = run(g, per_root=True, pivot=mce.MCE_PIVOT_IP)
    assert rn.tolist() == [n - i for i in range(n)]
    assert r.tree_nodes == n * (n + 1) // 2
    # full Tomita (IPX): every later root's excluded vertex 0 covers all of P
    r, (rc, rh, rn) = run(g, per_root=True, pivot=mce.MCE_PIVOT_IPX)
    assert rn.tolist() == [n] + [1] * (n - 1)


def test_device_pointer_input():
    g = gen.gnp(400, 0.07, 9)
    o = oracle.mce(g.row_ptr, g.col)
    h = mce.mce_create(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    r = mce.mce_run(h)
    mce.mce_destroy(h)
    same(r, o)


def test_empty_graph():
    g = gen.empty(0)
    r = run(g)
    assert r.count == 0 and r.max_size == 0


@pytest.mark.parametrize("bad", ["unsorted", "asym", "loop", "dup", "range", "rowptr"])
def test_invalid_graph_rejected(bad):
    g = gen.gnp(40, 0.3, 1)
    rp, col = g.row_ptr.copy(), g.col.copy()
    v = int(np.argmax(np.diff(rp) >= 3))
    a, b = rp[v], rp[v + 1]
    if bad == "unsorted":
        col[a], col[a + 1] = col[a + 1], col[a]
    elif bad == "asym":
        col[a] = [x for x in range(40) if x != v and x not in set(col[a:b])][0]
        col[a:b] = np.sort(col[a:b])
    elif bad == "loop":
        col[a] = v
        col[a:b] = np.sort(col[a:b])
    elif bad == "dup":
        col[a + 1] = col[a]
    elif bad == "range":
        col[b - 1] = 40
    elif bad == "rowptr":
        rp[5] = rp[6] + 1
    with pytest.raises(mce.MCEError) as ei:
        mce.mce_create(rp, col)
    assert ei.value.code == mce.MCE_EINVAL


def test_hist_too_short_is_erange():
    g = gen.complete(6)
    h = mce.mce_create(g.row_ptr, g.col)
    with pytest.raises(mce.MCEError) as ei:
        mce.mce_run(h, hist_len=4)
    assert ei.value.code == mce.MCE_ERANGE
    mce.mce_destroy(h)


def test_batch_small():
    parts = [gen.gnp(80, 0.15, 1), gen.moon_moser(4), gen.complete(9), gen.empty(3), gen.gnp(200, 0.05, 2),
             gen.cycle(10)]
    u = gen.disjoint_union(parts)
    h = mce.mce_batch_create(u.graph_ptr, u.row_ptr, u.col)
    per, hist, tot = mce.mce_run_batch(h)
    mce.mce_destroy(h)
    for i, p in enumerate(parts):
        # hashes use the ids of the concatenated graph
        a, z = int(u.graph_ptr[i]), int(u.graph_ptr[i + 1])
        o = oracle.mce(u.row_ptr, u.col, roots=np.arange(a, z, dtype=np.int32))
        assert (per[i].count, per[i].hash, per[i].max_size) == (o.count, o.hash, o.max_size), i
        hl = len(o.hist)
        assert np.array_equal(hist[i, :hl], o.hist) and not hist[i, hl:].any()
        # counts and histogram do not depend on ids: the part alone agrees
        op = oracle.mce(p.row_ptr, p.col)
        assert per[i].count == op.count and np.array_equal(hist[i, :len(op.hist)], op.hist)
    ou = oracle.mce(u.row_ptr, u.col)
    assert (tot.count, tot.hash) == (ou.count, ou.hash)


def test_batch_generated():
    b = gen.batch(48, 7, nmin=20, nmax=400, dmin=3, dmax=30, mm_every=8)
    h = mce.mce_batch_create(b.graph_ptr, b.row_ptr, b.col)
    per, hist, tot = mce.mce_run_batch(h)
    mce.mce_destroy(h)
    for i in range(48):
        a, z = int(b.graph_ptr[i]), int(b.graph_ptr[i + 1])
        o = oracle.mce(b.row_ptr, b.col, roots=np.arange(a, z, dtype=np.int32))
        assert (per[i].count, per[i].hash) == (o.count, o.hash), i
        if b.mm_sizes[i]:
            assert np.count_nonzero(hist[i]) >= 1


def test_root_subset():
    g = gen.gnp(600, 0.06, 12)
    roots = np.random.default_rng(3).choice(g.n, 150, replace=False).astype(np.int32)
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, roots=roots, per_root=True)
    r, (rc, rh, rn) = run(g, per_root=True, roots=roots, pivot=mce.MCE_PIVOT_IP)
    same(r, o)
    assert np.array_equal(rc, o.root_count) and np.array_equal(rh, o.root_hash)
    assert np.array_equal(rn, o.root_nodes)


def test_root_subset_empty_and_bad():
    g = gen.gnp(100, 0.1, 1)
    r = run(g, roots=np.zeros(0, np.int32))
    assert r.count == 0 and r.tree_nodes == 0
    with pytest.raises(mce.MCEError) as ei:
        run(g, roots=np.array([5, g.n], np.int32))
    assert ei.value.code == mce.MCE_EINVAL


def test_device_waits_give_up_and_context_survives():
    # each kind of device wait, run on its own with a 50 ms bound: a wait that
    # nothing releases gives up with MCE_ETIMEOUT (no fault, no hang), and a
    # wait kept alive by heartbeats outlasts its bound and ends normally
    assert mce.mce_selftest_waits(0, 50) == mce.MCE_ETIMEOUT  # idle wait, flag never set
    assert mce.mce_selftest_waits(1, 50) == mce.MCE_ETIMEOUT  # grid barrier one block short
    assert mce.mce_selftest_waits(2, 50) == mce.MCE_OK        # heartbeats for 150 ms, then released
    g = gen.gnp(300, 0.1, 2)
    same(run(g), oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP))


def test_long_subtree_is_not_timed():
    # one group walks a Moon-Moser root for far longer than the 20 ms wait
    # bound (no donations), while the other groups wait in the worker list:
    # the heartbeat keeps their waits alive, so only waits are ever timed
    g = gen.moon_moser(15)
    h = mce.mce_create(g.row_ptr, g.col)
    r = mce.mce_run(h, mce.mce_default_opts(timeout_ms=20, blocks=1, donate_min_p=100000,
                                            pivot=mce.MCE_PIVOT_IP))
    ref = mce.mce_run(h)
    mce.mce_destroy(h)
    assert r.count == 3 ** 15 and r.max_size == 15 and r.hist[15] == 3 ** 15
    assert (r.count, r.hash) == (ref.count, ref.hash)
    assert r.ms_traverse > 20.0  # the walk really outlasted the wait bound


def test_run_budget_stops_the_run_and_context_survives():
    g = gen.moon_moser(15)
    h = mce.mce_create(g.row_ptr, g.col)
    with pytest.raises(mce.MCEError) as ei:
        mce.mce_run(h, mce.mce_default_opts(run_budget_ms=2, blocks=1, donate_min_p=100000))
    assert ei.value.code == mce.MCE_EBUDGET
    r = mce.mce_run(h)
    mce.mce_destroy(h)
    assert r.count == 3 ** 15


def test_phase_counters_variant_gives_the_same_results():
    # opts.stats = 1 launches the kernel variant that keeps per-phase cycle
    # counters; the plain counting variant carries none of that code. Both must
    # walk the same trees, and the counters must account for every task and node.
    g = gen.disjoint_union([gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5), gen.moon_moser(7)])
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    h = mce.mce_create(g.row_ptr, g.col)
    try:
        r0 = mce.mce_run(h, mce.mce_default_opts(pivot=mce.MCE_PIVOT_IP, stats=0))
        st0 = mce.mce_get_stats(h)
        r1 = mce.mce_run(h, mce.mce_default_opts(pivot=mce.MCE_PIVOT_IP, stats=1, blocks=2, donate_min_p=1))
        st1 = mce.mce_get_stats(h)
    finally:
        mce.mce_destroy(h)
    for r in (r0, r1):
        assert (r.count, r.hash, r.max_size) == (o.count, o.hash, o.max_size)
    assert r0.tree_nodes == r1.tree_nodes
    assert sum(st0["phase_cycles"].values()) == 0
    assert all(v > 0 for k, v in st1["phase_cycles"].items() if k in ("setup", "pivot", "branch"))
    # one setup per task: every root with later neighbours, plus every received subtree
    _, _, outd = mce.mce_get_order(mce.mce_create(g.row_ptr, g.col))
    assert st1["phase_counts"]["setup"] == int((np.asarray(outd) > 0).sum()) + r1.donations


def test_peel_narrow_stage_runs_as_cluster():
    # gen.peel_stages() reaches every stage of the peel; on a GB300 the narrow
    # stage runs as one 16-CTA thread-block cluster, and the results stay exact
    g = gen.peel_stages()
    core_o, rank_o, _, _ = oracle.peel(g.row_ptr, g.col)
    h = mce.mce_create(g.row_ptr, g.col)
    try:
        core, rank, _ = mce.mce_get_order(h)
        mce.mce_run(h)
        st = mce.mce_get_stats(h)
    finally:
        mce.mce_destroy(h)
    assert np.array_equal(core, core_o) and np.array_equal(rank, rank_o)
    assert st["peel_stage_rounds"][1] > 0
    if torch.cuda.get_device_capability() >= (10, 0):
        assert st["peel_cluster"] == 1
