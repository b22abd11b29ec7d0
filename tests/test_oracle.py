"""Pins for the CPU oracle: closed forms, the paper's worked example, brute
force over all vertex subsets, cross-checks between Algorithms 1 and 2,
permutation invariance, disjoint-union additivity and the degeneracy
peel's properties. None of these expected values comes from the GPU engine,
and none re-calls the oracle's own routines to produce an expected value."""
import itertools
import json
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


# ----- independent restatement of the clique hash (definition, not the oracle's code)
def _mix(z):
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def h_clique(ids):
    s = sum(_mix(int(c) + 1) for c in ids) & M64
    return _mix(s + len(ids) * 0x9E3779B97F4A7C15)


def summarise(cliques):
    cliques = [tuple(sorted(c)) for c in cliques]
    hist = {}
    for c in cliques:
        hist[len(c)] = hist.get(len(c), 0) + 1
    return len(cliques), hist, sum(h_clique(c) for c in cliques) & M64


def hist_dict(arr):
    return {k: int(v) for k, v in enumerate(arr) if v}


def brute_force(g):
    """All maximal cliques by enumerating every vertex subset (n <= 16)."""
    n = g.n
    assert n <= 16
    adj = np.zeros(n, np.int64)
    for v in range(n):
        for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            adj[v] |= 1 << int(u)
    S = np.arange(1 << n, dtype=np.int64)
    clique = np.ones(S.shape, bool)
    for v in range(n):
        inS = (S >> v) & 1 == 1
        clique &= ~inS | ((S & ~(adj[v] | (1 << v))) == 0)
    maximal = clique.copy()
    for w in range(n):
        inS = (S >> w) & 1 == 1
        maximal &= inS | ((S & ~adj[w]) != 0)
    out = []
    for s in S[maximal]:
        out.append([v for v in range(n) if (int(s) >> v) & 1])
    return out


def run_all_modes(g):
    return [oracle.mce(g.row_ptr, g.col, mode=m, threads=2) for m in
            (oracle.PIVOT_FULL, oracle.PIVOT_IP, oracle.NO_PIVOT)]


def check(g, cliques):
    cnt, hist, hsh = summarise(cliques)
    for r in run_all_modes(g):
        assert r.count == cnt
        assert hist_dict(r.hist) == hist
        assert r.hash == hsh


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13])
def test_complete_graph(n):
    check(gen.complete(n), [list(range(n))])


@pytest.mark.parametrize("n", [0, 1, 4, 17])
def test_empty_graph(n):
    check(gen.empty(n), [[v] for v in range(n)])


@pytest.mark.parametrize("n", [4, 5, 9, 30])
def test_cycle(n):
    check(gen.cycle(n), [[i, (i + 1) % n] for i in range(n)])


def test_triangle_is_cycle_3():
    check(gen.cycle(3), [[0, 1, 2]])


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 7])
def test_moon_moser(k):
    # K_{3,...,3}: a maximal clique picks exactly one vertex from each part
    g = gen.moon_moser(k)
    cl = [list(p) for p in itertools.product(*[range(3 * i, 3 * i + 3) for i in range(k)])]
    assert len(cl) == 3 ** k
    check(g, cl)


@pytest.mark.parametrize("k", [1, 3, 5, 8])
def test_cocktail_party(k):
    g = gen.multipartite(k, 2)
    cl = [list(p) for p in itertools.product(*[range(2 * i, 2 * i + 2) for i in range(k)])]
    assert len(cl) == 2 ** k
    check(g, cl)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forest(seed):
    g = gen.random_forest(40, seed)
    deg = g.degrees()
    cl = [[v] for v in range(g.n) if deg[v] == 0]
    for v in range(g.n):
        for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            if v < u:
                cl.append([v, int(u)])
    check(g, cl)


def test_worked_example_golden():
    with open(os.path.join(GOLDEN, "worked_example.json")) as f:
        fx = json.load(f)
    idx = {name: i for i, name in enumerate(fx["vertices"])}
    g = gen.from_edges(len(idx), [(idx[a], idx[b]) for a, b in fx["edges"]])
    deg = g.degrees()
    assert int(deg.argmax()) == idx[fx["max_degree_vertex"]] and deg.max() == fx["max_degree"]
    check(g, [[idx[v] for v in c] for c in fx["maximal_cliques"]])
    assert g.n == len(gen.worked_example().row_ptr) - 1
    assert np.array_equal(g.col, gen.worked_example().col)


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("n,p,seed", [(n, p, s) for n in (6, 11, 16) for p in (0.1, 0.3, 0.5, 0.7, 0.9)
                                      for s in (0, 1)])
def test_brute_force(n, p, seed):
    g = gen.small_gnp(n, p, seed)
    check(g, brute_force(g))


# ------------------------------------------------------- cross-checks / invariants

@pytest.mark.parametrize("seed", range(4))
def test_algorithms_agree_midsize(seed):
    g = gen.gnp(300, 0.08 + 0.04 * seed, seed)
    full, ip, nopiv = run_all_modes(g)
    for r in (ip, nopiv):
        assert (r.count, r.hash, r.max_size) == (full.count, full.hash, full.max_size)
        assert np.array_equal(r.hist, full.hist)


@pytest.mark.parametrize("seed", range(3))
def test_permutation_invariance(seed):
    g = gen.gnp(120, 0.15, seed)
    perm = np.random.default_rng(seed).permutation(g.n)
    gp = gen.relabel(g, perm)
    a = oracle.mce(g.row_ptr, g.col)
    b = oracle.mce(gp.row_ptr, gp.col)
    assert a.count == b.count and np.array_equal(a.hist, b.hist)
    # small case: the permuted cliques' hash equals the hash of the mapped cliques
    g = gen.small_gnp(14, 0.5, seed)
    perm = np.random.default_rng(seed + 10).permutation(g.n)
    gp = gen.relabel(g, perm)
    mapped = [[int(perm[v]) for v in c] for c in brute_force(g)]
    assert oracle.mce(gp.row_ptr, gp.col).hash == summarise(mapped)[2]


def test_disjoint_union_additive():
    parts = [gen.gnp(80, 0.2, 5), gen.moon_moser(4), gen.complete(6), gen.empty(3)]
    u = gen.disjoint_union(parts)
    ru = oracle.mce(u.row_ptr, u.col)
    tot_c, tot_h, hist = 0, 0, {}
    for gpart, off in zip(parts, u.graph_ptr[:-1]):
        # shift ids: build the part's graph with ids offset, through from_edges
        src = np.repeat(np.arange(gpart.n), gpart.degrees())
        e = np.stack([src, gpart.col], 1)
        shifted = gen.from_edges(u.n, (e + int(off)).tolist())
        # isolated vertices of other parts would add size-1 cliques; restrict via roots
        r = oracle.mce(shifted.row_ptr, shifted.col,
                       roots=np.arange(off, off + gpart.n, dtype=np.int32))
        tot_c += r.count
        tot_h = (tot_h + r.hash) & M64
        for k, v in hist_dict(r.hist).items():
            hist[k] = hist.get(k, 0) + v
    assert ru.count == tot_c and ru.hash == tot_h and hist_dict(ru.hist) == hist


def test_per_root_sums_match_totals():
    g = gen.gnp(500, 0.05, 9)
    r = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, per_root=True)
    assert int(r.root_count.sum()) == r.count
    assert int(r.root_hash.astype(object).sum()) & M64 == r.hash
    sub = np.array([3, 77, 499, 0], np.int32)
    rs = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, roots=sub, per_root=True)
    assert rs.count == int(r.root_count[sub].sum())
    assert np.array_equal(rs.root_nodes[sub], r.root_nodes[sub])


@pytest.mark.parametrize("n", [2, 5, 9])
def test_node_counts_complete_graph(n):
    # K_n: the peel removes every vertex in one sub-round, ranks = ids.
    # Full Tomita: root 0 walks a chain of n calls; every later root's X holds
    # vertex 0, adjacent to all of P, so it is the pivot and no branch exists.
    g = gen.complete(n)
    full = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_FULL, per_root=True)
    assert full.root_nodes.tolist() == [n] + [1] * (n - 1)
    # pivot restricted to P u X_P: root r walks a chain of n - r calls
    ip = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, per_root=True)
    assert ip.root_nodes.tolist() == [n - r for r in range(n)]
    assert ip.root_count.tolist() == [1] + [0] * (n - 1)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_node_counts_moon_moser(k):
    # K_{3x k} is regular, so the peel keeps ids as ranks. Root v of part
    # p = v // 3 has P0 = the later parts, X0 = the earlier parts. With P a
    # K_{3x m} and X_P empty, the pivot is P's first vertex and its part gives
    # three branches, each again K_{3x (m-1)} with X_P empty (a part's
    # vertices are not adjacent): T(m) = 1 + 3 T(m-1), T(0) = 1.
    T = lambda m: (3 ** (m + 1) - 1) // 2
    g = gen.moon_moser(k)
    # full Tomita: an earlier part's vertex is adjacent to all of P, so every
    # root past part 0 stops at once
    full = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_FULL, per_root=True)
    assert full.root_nodes.tolist() == [T(k - 1) if v < 3 else 1 for v in range(3 * k)]
    # pivot from P u X_P: the earlier parts (X_X) never become pivots
    ip = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, per_root=True)
    assert ip.root_nodes.tolist() == [T(k - 1 - v // 3) for v in range(3 * k)]
    # no pivot: one call per clique of the later parts, 4 choices per part
    nop = oracle.mce(g.row_ptr, g.col, mode=oracle.NO_PIVOT, per_root=True)
    assert nop.root_nodes.tolist() == [4 ** (k - 1 - v // 3) for v in range(3 * k)]
    assert int(nop.root_nodes.sum()) == 4 ** k - 1
    for o in (full, ip, nop):
        assert o.count == 3 ** k


def _py_tomita_nodes(g, mode):
    """Per input vertex: (calls, maximal cliques) of its first-level subtree.

    Independent of oracle.c: Algorithm 2 written over Python sets, taking
    only the degeneracy order from the (separately pinned) oracle peel. The
    pivot maximises |P n N(u)| over P u X_P, or over all of X too under full
    Tomita; ties go to the smallest rank; branches run in ascending rank."""
    _, rank, order, _ = oracle.peel(g.row_ptr, g.col)
    n = g.n
    adj = [set() for _ in range(n)]
    for v in range(n):
        for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            adj[rank[v]].add(int(rank[u]))
    calls = np.zeros(n, np.int64)
    found = np.zeros(n, np.int64)

    def walk(root, P, XP, XX):
        calls[root] += 1
        if not P and not XP and not XX:
            found[root] += 1
            return
        if not P:
            return
        cands = P | XP | (XX if mode == oracle.PIVOT_FULL else set())
        pivot, best = None, -1
        for u in sorted(cands):
            score = len(P & adj[u])
            if score > best:
                pivot, best = u, score
        for v in sorted(P - adj[pivot]):
            walk(root, P & adj[v], XP & adj[v], XX & adj[v])
            P = P - {v}
            XP = XP | {v}

    for r in range(n):
        walk(r, {u for u in adj[r] if u > r}, set(), {u for u in adj[r] if u < r})
    by_id_calls, by_id_found = np.zeros(n, np.int64), np.zeros(n, np.int64)
    by_id_calls[order] = calls
    by_id_found[order] = found
    return by_id_calls, by_id_found


@pytest.mark.parametrize("mode", [oracle.PIVOT_FULL, oracle.PIVOT_IP])
@pytest.mark.parametrize("n,p,seed", [(14, 0.4, 1), (24, 0.3, 2), (30, 0.5, 3), (40, 0.2, 4)])
def test_node_counts_match_python_tomita(n, p, seed, mode):
    # pins the tie rule and the pivot domains on irregular graphs, where the
    # closed forms above cannot reach
    g = gen.small_gnp(n, p, seed)
    calls, found = _py_tomita_nodes(g, mode)
    o = oracle.mce(g.row_ptr, g.col, mode=mode, per_root=True)
    assert o.root_nodes.astype(np.int64).tolist() == calls.tolist()
    assert o.root_count.astype(np.int64).tolist() == found.tolist()


def _words(p):
    return (p + 31) // 32


@pytest.mark.parametrize("n", [1, 2, 5, 33, 70])
def test_work_counter_complete_graph(n):
    # The roofline's numerator: per node with P non-empty, W = ceil(|P0|/32)
    # word-ops per pivot candidate scanned (ascending rank, up to the first
    # that reaches the largest possible score), W for the branch set and 2W
    # per branch. K_n, pivot from P u X_P: root r walks a chain of
    # p0 = n - 1 - r nodes whose first candidate reaches |P| - 1 and leaves
    # one branch: 4W each. Full Tomita: a later root scans vertex 0 of X_X,
    # which reaches |P| and leaves no branch: 2W.
    g = gen.complete(n)
    _, ip = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    _, full = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_FULL)
    chain = [4 * (n - 1 - r) * _words(n - 1 - r) for r in range(n)]
    assert ip.tolist() == chain
    assert full.tolist() == chain[:1] + [2 * _words(n - 1 - r) for r in range(1, n)]


@pytest.mark.parametrize("k", [1, 2, 3, 5, 12])
def test_work_counter_moon_moser(k):
    # K_{3x k}: at a node whose P is a K_{3x m} (X_P empty), every candidate
    # scores 3m - 3, short of the bound 3m - 1, so all 3m are scanned; the
    # pivot's part gives 3 branches: W (3m + 7). A root of part p has 3^d
    # such nodes at depth d with m = k - 1 - p - d. Full Tomita: roots past
    # part 0 scan one vertex of X_X and stop (2W).
    def tree(m):
        return _words(3 * m) * sum(3 ** d * (3 * (m - d) + 7) for d in range(m))
    g = gen.moon_moser(k)
    _, ip = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    _, full = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_FULL)
    assert ip.tolist() == [tree(k - 1 - v // 3) for v in range(3 * k)]
    assert full.tolist() == [tree(k - 1) if v < 3 else 2 * _words(3 * (k - 1 - v // 3)) for v in range(3 * k)]


@pytest.mark.parametrize("n", [2, 3, 6, 10])
def test_second_level_node_counts_complete_graph(n):
    # K_n, one subtree per edge (i, j), i < j (Algorithm 4): X = {0..j-1} - {i}.
    # Full Tomita: only edge (0, 1) has X empty and walks a chain of n - 1
    # calls; every other edge node has a pivot in X adjacent to all of P.
    g = gen.complete(n)
    full = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_FULL, per_root=True, level=2)
    assert int(full.root_nodes.sum()) == n * (n - 1) // 2 + n - 2
    assert full.root_nodes[0] == (n - 1) + (n - 2)  # edges (0, 1) .. (0, n-1)
    # pivot from P u X_P: edge (j-1, j) has X_P empty and walks n - j calls,
    # the others stop at once: (n-1)^2 in all
    ip = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, per_root=True, level=2)
    assert int(ip.root_nodes.sum()) == (n - 1) ** 2
    assert ip.root_nodes.tolist() == [(n - 1 - j - 1 + 1) + (n - 2 - j) for j in range(n - 1)] + [0]
    # no pivot: edge (i, j) spans all 2^(n-1-j) subsets of the vertices after j
    nop = oracle.mce(g.row_ptr, g.col, mode=oracle.NO_PIVOT, per_root=True, level=2)
    assert int(nop.root_nodes.sum()) == 2 ** n - n - 1
    for o in (full, ip, nop):
        assert o.count == 1 and o.root_count.tolist() == [1] + [0] * (n - 1)


@pytest.mark.parametrize("seed", range(6))
def test_second_level_same_cliques(seed):
    # edge subtrees partition M(G) minus the isolated vertices, which are
    # cliques of their own: every result equals the first-level walk's
    g = gen.disjoint_union([gen.small_gnp(35, 0.25, seed), gen.empty(3), gen.moon_moser(3)])
    for mode in (oracle.PIVOT_FULL, oracle.PIVOT_IP, oracle.NO_PIVOT):
        a = oracle.mce(g.row_ptr, g.col, mode=mode, per_root=True)
        b = oracle.mce(g.row_ptr, g.col, mode=mode, per_root=True, level=2)
        assert (a.count, a.hash, a.max_size) == (b.count, b.hash, b.max_size)
        assert np.array_equal(a.hist, b.hist)
        assert np.array_equal(a.root_count, b.root_count) and np.array_equal(a.root_hash, b.root_hash)


# ------------------------------------------------------------ degeneracy peel

def naive_cores(g):
    """Sequential min-degree peel (Matula-Beck), O(n^2): core numbers."""
    n = g.n
    deg = g.degrees().astype(np.int64)
    alive = np.ones(n, bool)
    core = np.zeros(n, np.int64)
    k = 0
    for _ in range(n):
        d = np.where(alive, deg, np.iinfo(np.int64).max)
        v = int(d.argmin())
        k = max(k, int(deg[v]))
        core[v] = k
        alive[v] = False
        for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            deg[u] -= 1
    return core


@pytest.mark.parametrize("maker", [lambda: gen.workload("er_2000"), lambda: gen.gnp(400, 0.05, 3),
                                   lambda: gen.moon_moser(5), gen.worked_example,
                                   lambda: gen.random_forest(100, 4), lambda: gen.cycle(12)])
def test_peel_properties(maker):
    g = maker()
    core, rank, order, rounds = oracle.peel(g.row_ptr, g.col)
    assert np.array_equal(core, naive_cores(g))
    assert np.array_equal(np.sort(rank), np.arange(g.n))
    assert np.array_equal(order[rank], np.arange(g.n))
    src = np.repeat(np.arange(g.n), g.degrees())
    later = np.bincount(src[rank[g.col] > rank[src]], minlength=g.n)
    assert (later <= core).all()           # |P| <= core(v) <= d (Sec. II-C)
    # core is non-decreasing along the order
    assert (np.diff(core[order]) >= 0).all()
    assert rounds >= 1 or g.n == 0


def test_worked_example_order():
    # Sec. II-C: after degeneracy ordering A has no later neighbours. Our
    # tie-break (ascending id within a peel sub-round) removes E and F first
    # (core 2), then A, B, C, D together (core 3); A's later neighbours are
    # B, C, D, which is within the degeneracy d = 3.
    g = gen.worked_example()
    core, rank, order, _ = oracle.peel(g.row_ptr, g.col)
    assert core.tolist() == [3, 3, 3, 3, 2, 2]
    assert order.tolist() == [4, 5, 0, 1, 2, 3]


@pytest.mark.parametrize("edges,n,order,rounds", [
    # a path peels from both ends inward, two vertices per sub-round
    ([(i, i + 1) for i in range(6)], 7, [0, 6, 1, 5, 2, 4, 3], 4),
    # a star's leaves go first; the centre follows in the next sub-round
    # although its id is the smallest
    ([(0, i) for i in range(1, 6)], 6, [1, 2, 3, 4, 5, 0], 2),
    # every vertex of a cycle or a clique leaves in the first sub-round
    ([(i, (i + 1) % 8) for i in range(8)], 8, list(range(8)), 1),
    ([(i, j) for i in range(5) for j in range(i + 1, 5)], 5, list(range(5)), 1),
])
def test_peel_order_closed_forms(edges, n, order, rounds):
    # Sec. II-C's peel, level-synchronous: a sub-round removes every vertex
    # whose remaining degree is at most k, in ascending id
    g = gen.from_edges(n, edges)
    core, rank, got, got_rounds = oracle.peel(g.row_ptr, g.col)
    assert got.tolist() == order
    assert got_rounds == rounds
    assert np.array_equal(rank[got], np.arange(n))


# ----------------------------------------------------------------- validation

@pytest.mark.parametrize("bad", ["unsorted", "asym", "loop", "dup", "range", "rowptr"])
def test_validate_rejects(bad):
    g = gen.gnp(30, 0.3, 1)
    rp, col = g.row_ptr.copy(), g.col.copy()
    v = int(np.argmax(np.diff(rp) >= 2))
    a, b = rp[v], rp[v + 1]
    if bad == "unsorted":
        col[a], col[a + 1] = col[a + 1], col[a]
    elif bad == "asym":
        col = col.copy()
        col[a] = [x for x in range(30) if x != v and x not in set(col[a:b])][0]
        col[a:b] = np.sort(col[a:b])
    elif bad == "loop":
        col[a] = v
        col[a:b] = np.sort(col[a:b])
    elif bad == "dup":
        col[a + 1] = col[a]
    elif bad == "range":
        col[b - 1] = 30
    elif bad == "rowptr":
        rp[5] = rp[6] + 1
    assert oracle.validate(g.row_ptr, g.col)
    assert not oracle.validate(rp, col)


# ------------------------------------------------ work-estimator references

def test_features_complete_graph_closed_form():
    from oracle.features import root_features
    n = 9
    g = gen.complete(n)
    f = root_features(g.row_ptr, g.col)
    for r in range(n):  # K_n: one peel round, rank = id; P0 = later ids, X0 = earlier ids
        k, x = n - 1 - r, r
        pairs = k * (k - 1) // 2
        want = [n - 1, n - 1, k, x, pairs + k * x, pairs, k * x, 65536 if k >= 2 else 0,
                (n - 1) * (n - 1), k - 1 if k else 0, k - 1 if k else 0, k, n - 1 if k else 0,
                (n - 1) * k, k if x else 0, 0]
        assert f[r].tolist() == want, r


def test_features_star_and_path():
    from oracle.features import root_features
    g = gen.from_edges(6, [(0, i) for i in range(1, 6)])  # star: leaves peel first, centre last
    f = root_features(g.row_ptr, g.col)
    assert f[0].tolist()[:4] == [5, 1, 0, 5] and f[0, 8] == 5
    for leaf in range(1, 6):
        assert f[leaf].tolist()[:4] == [1, 1, 1, 0] and f[leaf, 8] == 5 and f[leaf, 15] == 0


def hub_graph():
    """Hub 0 with a K_5 on 1..5 and 300 leaves 6..305. Leaves 6 (-> 1),
    7 (-> 1, 2), 304 (-> 4) and 305 (-> 1, 2, 3) also touch the clique. The
    peel removes the plain leaves (k = 1), 6 and 304 (k = 2), 7 (k = 3), 305
    (k = 4), then 0..5 together (k = 5, ascending id): the hub's P0 is the
    K_5 and its X0 all 300 leaves, of which X0' holds ids 6..261."""
    edges = [(0, c) for c in range(1, 6)] + [(a, b) for a in range(1, 6) for b in range(a + 1, 6)]
    edges += [(0, x) for x in range(6, 306)]
    edges += [(6, 1), (7, 1), (7, 2), (304, 4), (305, 1), (305, 2), (305, 3)]
    return gen.from_edges(306, edges)


def test_features_hub_with_more_than_256_excluded():
    # features 4, 6 and 14 look at X0' = the 256 smallest ids of X0 only: of
    # the leaves touching P0, 6 and 7 are in X0', 304 and 305 are not
    from oracle.features import root_features
    g = hub_graph()
    f = root_features(g.row_ptr, g.col)
    want = [305, 5, 5, 300,
            10 + 3,      # e(P0) + e(P0, X0'): 6 -> {1}, 7 -> {1, 2}
            10, 3,
            65536,       # e(P0) / C(5, 2) = 1
            296 * 1 + 2 + 3 + 2 + 4 + (8 + 7 + 6 + 6 + 5),  # degrees of the leaves, then of 1..5
            4, 4, 5, 5, 25,
            2,           # leaf 7; leaf 305 (3) is outside X0'
            0]
    assert f[0].tolist() == want
    # a leaf: P0 = {0} (the hub is later), X0 empty
    assert f[100].tolist() == [1, 1, 1, 0, 0, 0, 0, 0, 305, 0, 0, 1, 5, 5, 0, 0]


def test_features_joined_cliques_with_pendant():
    # K4 on 0..3 and K5 on 4..8 joined by 0-4; vertex 9 adjacent to 3, 8 and
    # 10. Peel: 10 (k = 1), 9 (k = 2), then 1, 2, 3 and 0 (k = 3), then 4..8
    # (k = 4): cores 1 / 2 / 3 / 4, so P0 sets span different cores.
    from oracle.features import root_features
    edges = [(a, b) for a in range(4) for b in range(a + 1, 4)] + [(a, b) for a in range(4, 9) for b in range(a + 1, 9)]
    edges += [(0, 4), (3, 9), (8, 9), (9, 10)]
    g = gen.from_edges(11, edges)
    f = root_features(g.row_ptr, g.col)
    # root 9: P0 = {3 (core 3), 8 (core 4)}, not adjacent; X0 = {10}
    assert f[9].tolist() == [3, 2, 2, 1, 0, 0, 0, 0, 4 + 5 + 1, 0, 0, 0, 4, 7, 0, 1]
    # root 0: P0 = {4}, X0 = {1, 2, 3}
    assert f[0].tolist() == [4, 3, 1, 3, 0, 0, 0, 0, 3 + 3 + 4 + 5, 0, 0, 1, 4, 4, 0, 0]
    # root 3: 9 is earlier (rank 1), so P0 = {0} and X0 = {1, 2, 9}; 1 and 2
    # are adjacent to 0, 9 is not
    assert f[3].tolist() == [4, 3, 1, 3, 0 + 2, 0, 2, 0, 4 + 3 + 3 + 3, 0, 0, 1, 3, 3, 1, 0]


def test_adam_reference_closed_forms():
    from oracle import mlp
    rs = np.random.default_rng(5)
    p0 = rs.normal(0, 0.5, mlp.NPARAMS)
    g = rs.normal(0, 1e-2, mlp.NPARAMS)
    g[:5] = [0.0, 1e-3, -2.0, 1e-9, -1e-9]
    lr = 1e-3
    z = np.zeros(mlp.OMEAN)
    step = -lr * g[:mlp.OMEAN] / (np.abs(g[:mlp.OMEAN]) + mlp.ADAM_EPS)
    # the same gradient every step: m_hat = g and v_hat = g^2 at every t
    p, m, v = p0, z, z
    for t in range(1, 6):
        p, m, v = mlp.adam_step(p, g, m, v, t, lr)
        assert np.allclose(p[:mlp.OMEAN] - p0[:mlp.OMEAN], t * step, rtol=1e-12, atol=1e-15)
    assert np.array_equal(p[mlp.OMEAN:], p0[mlp.OMEAN:])  # mean and std are not trained
    # g then -g: m_hat_2 = -(1 - b1) / (1 + b1) g and v_hat_2 = g^2
    p1, m1, v1 = mlp.adam_step(p0, g, z, z, 1, lr)
    p2, _, _ = mlp.adam_step(p1, -g, m1, v1, 2, lr)
    b1 = mlp.ADAM_B1
    want = -lr * (-(1 - b1) / (1 + b1) * g[:mlp.OMEAN]) / (np.abs(g[:mlp.OMEAN]) + mlp.ADAM_EPS)
    assert np.allclose(p2[:mlp.OMEAN] - p1[:mlp.OMEAN], want, rtol=1e-12, atol=1e-15)
    assert p2[0] == p0[0]  # a zero gradient never moves its entry


def test_capped_walk_keeps_finished_roots_exact():
    # a root over the cap is abandoned and marked; every other root's count,
    # hash and node count equal the uncapped walk's, and the cap splits the
    # roots exactly by their node counts
    g = gen.chung_lu(3000, 12.0, 2.1, 300.0, 3, 10, 20, 4)
    r = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, per_root=True)
    c, h, nd = oracle.capped(g.row_ptr, g.col, np.arange(g.n, dtype=np.int32), 50)
    ok = nd != np.iinfo(np.uint64).max
    assert 0 < (~ok).sum() < g.n
    assert np.array_equal(c[ok], r.root_count[ok]) and np.array_equal(h[ok], r.root_hash[ok])
    assert np.array_equal(nd[ok], r.root_nodes[ok])
    assert np.all(r.root_nodes[ok] <= 50) and np.all(r.root_nodes[~ok] > 50)
    assert not c[~ok].any() and not h[~ok].any()


def test_tree_estimate_exact_on_regular_trees():
    # Moon-Moser and complete graphs: every node at a given depth of a root's
    # subtree has the same number of children, so every random path gives the
    # exact node count (zero variance), which the branching recurrence fixes:
    # the first root of K_{3xk} has T(k) = 1 + 3 T(k - 1), T(0) = 1 nodes,
    # and the first root of K_n is a chain of n nodes.
    for k in (3, 5, 7):
        g = gen.moon_moser(k)
        mean, var = oracle.tree_estimate(g.row_ptr, g.col, np.arange(g.n, dtype=np.int32), probes=5, seed=3)
        rn, _ = oracle.work(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
        assert np.array_equal(mean, rn.astype(np.float64)) and np.all(var == 0)
        t = 1
        for _ in range(k - 1):
            t = 1 + 3 * t
        assert mean[0] == t
    # K_n: under the partial rule (pivot from P u X_P) root r walks a chain of
    # n - r nodes; under full Tomita an earlier vertex covers P, so every root
    # after the first has one node
    g = gen.complete(10)
    ids = np.arange(10, dtype=np.int32)
    mean, var = oracle.tree_estimate(g.row_ptr, g.col, ids, probes=3, mode=oracle.PIVOT_IP)
    assert mean.tolist() == [10 - r for r in range(10)] and np.all(var == 0)
    mean, var = oracle.tree_estimate(g.row_ptr, g.col, ids, probes=3, mode=oracle.PIVOT_FULL)
    assert mean[0] == 10 and np.all(mean[1:] == 1) and np.all(var == 0)


@pytest.mark.parametrize("mode", [oracle.PIVOT_IP, oracle.PIVOT_FULL])
def test_tree_estimate_is_unbiased_on_irregular_graphs(mode):
    # Knuth's estimate is unbiased: the mean of many random paths sits within a
    # few standard errors of the exact node count, root by root and in total
    g = gen.chung_lu(3000, 12.0, 2.1, 300.0, 3, 10, 20, 4)
    roots = np.arange(g.n, dtype=np.int32)
    probes = 2000
    mean, var = oracle.tree_estimate(g.row_ptr, g.col, roots, probes=probes, seed=7, mode=mode)
    exact, _ = oracle.work(g.row_ptr, g.col, mode=mode)
    exact = exact.astype(np.float64)
    se = np.sqrt(var / probes)
    assert np.all(mean[var == 0] == exact[var == 0])
    z = np.abs(mean - exact)[var > 0] / se[var > 0]
    assert z.max() < 6.0
    assert abs(mean.sum() - exact.sum()) < 5.0 * np.sqrt((var / probes).sum())
    # and the path choice matters: a different seed changes some estimates
    mean2, _ = oracle.tree_estimate(g.row_ptr, g.col, roots, probes=probes, seed=8, mode=mode)
    assert np.any(mean2[var > 0] != mean[var > 0])


def test_mlp_reference_gradient_matches_finite_differences():
    from oracle import mlp
    rs = np.random.default_rng(0)
    p = rs.normal(0, 0.3, mlp.NPARAMS)
    p[mlp.OSTD:] = rs.uniform(0.5, 2.0, 16)
    x = rs.normal(1.0, 1.0, (7, 16))
    t = rs.normal(3.0, 1.0, 7)
    loss, g = mlp.loss_and_grad(p, x, t, rounded=False)
    eps = 1e-6
    for i in list(range(0, mlp.OMEAN, 97)) + [mlp.OB3, mlp.OW3 + 5, mlp.OB1 + 3]:
        q = p.copy()
        q[i] += eps
        lp = mlp.loss_and_grad(q, x, t, rounded=False)[0]
        q[i] -= 2 * eps
        lm = mlp.loss_and_grad(q, x, t, rounded=False)[0]
        assert abs((lp - lm) / (2 * eps) - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i
    assert np.all(g[mlp.OMEAN:] == 0)


def test_bf16_rounding_reference():
    from oracle.mlp import bf16_round
    # exactly representable values stay; halfway cases go to the even neighbour
    assert bf16_round(np.float32(1.0)) == 1.0
    assert bf16_round(np.float32(1.0 + 2 ** -8)) == 1.0                  # halfway, even is 1.0
    assert bf16_round(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6    # halfway, even is up
    assert bf16_round(np.float32(-2.5)) == -2.5
    assert bf16_round(np.float32(1.0 + 2 ** -7 + 2 ** -9)) == 1.0 + 2 ** -7


@pytest.mark.parametrize("k,size,first", [(1, 3, 0), (4, 3, 7), (6, 3, 100), (5, 2, 3), (3, 4, 11)])
def test_multipartite_enumeration(k, size, first):
    # transversal enumeration = Bron-Kerbosch on the same graph (ids offset by `first`)
    g = gen.multipartite(k, size)
    src = np.repeat(np.arange(g.n), g.degrees())
    e = np.stack([src, g.col], 1) + first
    shifted = gen.from_edges(first + g.n, e.tolist())
    r = oracle.mce(shifted.row_ptr, shifted.col, roots=np.arange(first, first + g.n, dtype=np.int32))
    c, h = oracle.multipartite(first, k, size)
    assert c == size ** k == r.count and h == r.hash


def peel_stage_passes(g):
    """The GPU peel's stage at every level-start pass of g, from the oracle.

    A level start of the GPU peel narrows the grid to 16 blocks when the live
    degree sum is at most 2^22, the live vertices at most 32,768 and its S at
    most 1,024 vertices; it goes to one block (checked first) at most 32,768,
    2,048 and 64. It guesses k + 1; when no live vertex has that degree, one
    more pass runs first, in the stage of the level before. At level k the
    live vertices are those of core number >= k, and S holds those with at
    most k live neighbours. Returns (stage of each level, stage of each extra
    pass); 0, 1, 2 = full grid, 16 blocks, one block.
    """
    core = oracle.peel(g.row_ptr, g.col)[0]
    src = np.repeat(np.arange(g.n), g.degrees())
    stage, levels, extra, prev = 0, [], [], -1
    for k in np.unique(core):
        live_v = core >= k
        both = live_v[src] & live_v[g.col]
        ldeg = np.bincount(src[both], minlength=g.n)
        live_sum, nlive = int(both.sum()), int(live_v.sum())
        s_size = int((live_v & (ldeg <= k)).sum())
        if k > prev + 1:
            extra.append(stage)
        if stage < 2 and live_sum <= 32768 and nlive <= 2048 and s_size <= 64:
            stage = 2
        elif stage == 0 and live_sum <= (1 << 22) and nlive <= 32768 and s_size <= 1024:
            stage = 1
        levels.append(stage)
        prev = int(k)
    return levels, extra


def test_peel_stages_graph_spans_every_stage():
    # gen.peel_stages() must run levels in all three stages of the GPU peel
    # and make the extra level-start pass in each
    g = gen.peel_stages()
    levels, extra = peel_stage_passes(g)
    assert set(levels) == {0, 1, 2}
    assert set(extra) == {0, 1, 2}
    assert int(g.degrees().min()) > 0


def test_peel_stage_model_on_small_graphs():
    # the grid narrows only once the live vertices bound every later S:
    # never on G(n, m), whose every level still holds most of its vertices
    levels, _ = peel_stage_passes(gen.er(200000, 1500000, 5))
    assert set(levels) == {0}
