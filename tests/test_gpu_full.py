"""Full-size workloads on the GPU, in the launch configuration bench.py uses.

* er_2000 and chunglu_1m: every result against the stored oracle values in
  tests/golden/ (written by tests/golden/make_golden.py, which calls only the
  oracle), after checking that the generator rebuilt the same graph.
* rmat_22 (R-MAT scale 22): too heavy for the oracle as a whole, so the peel
  (core numbers and ranks, unique by definition) is compared in full, and the
  first-level subtrees of seeded samples of roots are compared one by one
  (count, hash, tree nodes per root): roots of up to 4 words per row drawn
  here, and stored roots in every row-width band up to 16 words
  (tests/golden/rmat_22_roots.json, written by the oracle; from 17 words on
  no drawn root finishes within the oracle's cap of 4 million calls); and the
  whole subset of roots with at most 4 words per row, the bench's rmat_22_w4.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2212_01473_gb300 as mce  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fingerprint(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, np.int32).tobytes())
    h.update(np.ascontiguousarray(g.col, np.int32).tobytes())
    return {"n": g.n, "m": g.m, "sha256": h.hexdigest()}


@pytest.mark.parametrize("name", ["er_2000", "chunglu_1m"])
def test_workload_matches_stored_oracle(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        gold = json.load(f)
    g = gen.workload(name)
    assert fingerprint(g) == gold["fingerprint"], "generator produced a different graph"
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    h = mce.mce_create(rp, col)
    r = mce.mce_run(h, mce.mce_default_opts(pivot=mce.MCE_PIVOT_IP))  # the stored tree sizes are IP's
    auto = mce.mce_run(h)
    mce.mce_destroy(h)
    assert (auto.count, auto.hash, auto.max_size) == (gold["count"], int(gold["hash"], 16), gold["max_size"])
    assert auto.hist.tolist() == gold["hist"]
    assert r.count == gold["count"]
    assert "0x%016x" % r.hash == gold["hash"]
    assert r.max_size == gold["max_size"]
    assert r.hist.tolist() == gold["hist"]
    assert r.degeneracy == gold["degeneracy"]
    assert r.tree_nodes == gold["tree_nodes"]


@pytest.fixture(scope="module")
def rmat():
    g = gen.workload("rmat_22")
    core, rank, order, _ = oracle.peel(g.row_ptr, g.col)
    return g, core, rank


def test_rmat_22_peel(rmat):
    g, core_o, rank_o = rmat
    h = mce.mce_create(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    core, rank, outd = mce.mce_get_order(h)
    info = mce.mce_graph_info(h)
    mce.mce_destroy(h)
    assert np.array_equal(core, core_o)
    assert np.array_equal(rank, rank_o)
    assert info["degeneracy"] == int(core_o.max())
    assert int(outd.max()) <= info["degeneracy"]


def test_rmat_22_sampled_roots(rmat):
    g, core_o, rank_o = rmat
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    later = np.bincount(src[rank_o[g.col] > rank_o[src]], minlength=g.n)
    W = (later + 31) // 32
    rs = np.random.default_rng(2024)
    picks = []
    for lo, hi, k in ((0, 0, 100), (1, 1, 200), (2, 2, 150), (3, 4, 150)):
        cand = np.nonzero((W >= lo) & (W <= hi))[0]
        picks.append(rs.choice(cand, min(k, len(cand)), replace=False))
    roots = np.sort(np.concatenate(picks)).astype(np.int32)
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, roots=roots, per_root=True)
    r, (rc, rh, rn) = mce.enumerate_maximal_cliques(g.row_ptr, g.col, per_root=True, roots=roots,
                                                     pivot=mce.MCE_PIVOT_IP)
    assert r.count == o.count and r.hash == o.hash and r.max_size == o.max_size
    assert np.array_equal(r.hist, o.hist)
    assert np.array_equal(rc[roots], o.root_count[roots])
    assert np.array_equal(rh[roots], o.root_hash[roots])
    assert np.array_equal(rn[roots], o.root_nodes[roots])
    assert not rc[np.setdiff1d(np.arange(g.n), roots)].any()


def test_rmat_22_every_width_band(rmat):
    # the stored per-root oracle results of seeded roots in every band up to
    # W = 16 (roots the oracle finishes within its cap), through the launch
    # configuration of a whole run (all width classes, worker list on)
    g, core_o, rank_o = rmat
    with open(os.path.join(GOLDEN, "rmat_22_roots.json")) as f:
        gold = json.load(f)
    assert fingerprint(g) == gold["fingerprint"], "generator produced a different graph"
    roots = np.asarray(gold["roots"], np.int32)
    # every band up to W = 16; from W = 17 on no drawn root finished within the oracle's cap
    bands = [(1, 1), (2, 2), (3, 4), (5, 8), (9, 12), (13, 16)]
    assert all(any(lo <= w <= hi for w in gold["W"]) for lo, hi in bands)
    r, (rc, rh, rn) = mce.enumerate_maximal_cliques(g.row_ptr, g.col, per_root=True, roots=roots,
                                                     pivot=mce.MCE_PIVOT_IP)
    assert r.count == gold["count"] and "0x%016x" % r.hash == gold["hash"]
    assert rc[roots].tolist() == gold["root_count"]
    assert ["0x%016x" % int(x) for x in rh[roots]] == gold["root_hash"]
    assert rn[roots].tolist() == gold["root_nodes"]


def test_rmat_22_w4_subset_matches_stored_oracle(rmat):
    # the bench's rmat_22_w4 workload: every root with at most 4 words per
    # row (|P0| <= 128), isolated vertices included, enumerated whole, in the
    # launch configuration bench.py uses, against the stored oracle result
    g, core_o, rank_o = rmat
    with open(os.path.join(GOLDEN, "rmat_22_w4.json")) as f:
        gold = json.load(f)
    assert fingerprint(g) == gold["fingerprint"], "generator produced a different graph"
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    later = np.bincount(src[rank_o[g.col] > rank_o[src]], minlength=g.n)
    roots = np.nonzero((later + 31) // 32 <= 4)[0].astype(np.int32)
    assert len(roots) == gold["roots"]
    for pivot in (mce.MCE_PIVOT_IP, mce.MCE_PIVOT_AUTO):
        r = mce.enumerate_maximal_cliques(g.row_ptr, g.col, roots=roots, pivot=pivot)
        assert (r.count, "0x%016x" % r.hash, r.max_size) == (gold["count"], gold["hash"], gold["max_size"])
        assert r.hist.tolist() == gold["hist"]
        if pivot == mce.MCE_PIVOT_IP:
            assert r.tree_nodes == gold["tree_nodes"]
