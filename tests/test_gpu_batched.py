"""Batched graphs in one set of persistent launches, replayed from a CUDA
graph, with autotuned launch settings: every per-graph result equals the
oracle's (stored for the 4096-graph workload by tests/golden/make_golden.py,
which calls only the oracle)."""
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


def _same_batches(a, b):
    (pa, ha, ta), (pb, hb, tb) = a, b
    assert [(x.count, x.hash, x.max_size) for x in pa] == [(x.count, x.hash, x.max_size) for x in pb]
    assert np.array_equal(ha, hb)
    assert (ta.count, ta.hash, ta.tree_nodes) == (tb.count, tb.hash, tb.tree_nodes)


def test_prepared_replay_equals_direct_run():
    b = gen.batch(64, 11, nmin=20, nmax=600, dmin=4, dmax=40, mm_every=8)
    h = mce.mce_batch_create(b.graph_ptr, b.row_ptr, b.col)
    direct = mce.mce_run_batch(h)
    mce.mce_prepare(h)
    r1 = mce.mce_run_prepared(h)
    r2 = mce.mce_run_prepared(h)
    mce.mce_destroy(h)
    _same_batches(direct, r1)
    _same_batches(direct, r2)
    for i in range(64):
        a, z = int(b.graph_ptr[i]), int(b.graph_ptr[i + 1])
        o = oracle.mce(b.row_ptr, b.col, roots=np.arange(a, z, dtype=np.int32))
        assert (r1[0][i].count, r1[0][i].hash) == (o.count, o.hash)


def test_prepared_single_graph_and_per_root_buffers():
    g = gen.gnp(800, 0.04, 5)
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, per_root=True)
    h = mce.mce_create(g.row_ptr, g.col)
    nodes = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    opts = mce.mce_default_opts(pivot=mce.MCE_PIVOT_IP)  # the oracle's tree above is IP's
    opts.root_nodes = nodes.data_ptr()
    mce.mce_prepare(h, opts)
    for _ in range(2):
        per, hist, tot = mce.mce_run_prepared(h)
        torch.cuda.synchronize()
        assert (tot.count, tot.hash) == (o.count, o.hash)
        assert np.array_equal(nodes.cpu().numpy().view(np.uint64), o.root_nodes)
    mce.mce_destroy(h)


def test_autotune_changes_schedule_only():
    g = gen.chung_lu(30000, 14.0, 2.1, 1500.0, 4, 20, 32, 8)
    h = mce.mce_create(g.row_ptr, g.col)
    plain = mce.mce_run(h)
    t = mce.mce_autotune(h, budget_ms=2000.0)
    assert len(t["donate_min_p"]) == 9 and len(t["warps"]) == 9 and t["merge_wp"] in (1, 4, 12)
    tuned = mce.mce_run(h, mce.mce_default_opts(tuned=1))
    # every bitset width of the one-warp launch and every block size the tuner may pick
    others = [mce.mce_run(h, mce.mce_default_opts(merge_wp=mw, block_warps=bw))
              for mw in (1, 4, 12) for bw in (4, 8, 16, 24)]
    mce.mce_destroy(h)
    for r in [tuned] + others:
        assert (r.count, r.hash, r.tree_nodes) == (plain.count, plain.hash, plain.tree_nodes)
        assert np.array_equal(r.hist, plain.hist)


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLDEN, "batch_4096.json")), reason="no stored results")
def test_batch_4096_matches_stored_oracle():
    with open(os.path.join(GOLDEN, "batch_4096.json")) as f:
        gold = json.load(f)
    b = gen.workload("batch_4096")
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(b.row_ptr, np.int32).tobytes())
    h.update(np.ascontiguousarray(b.col, np.int32).tobytes())
    assert h.hexdigest() == gold["fingerprint"]["sha256"]
    hd = mce.mce_batch_create(torch.from_numpy(b.graph_ptr).cuda(), torch.from_numpy(b.row_ptr).cuda(),
                              torch.from_numpy(b.col).cuda())
    mce.mce_autotune(hd, budget_ms=8000.0)
    mce.mce_prepare(hd, mce.mce_default_opts(tuned=1))
    per, hist, tot = mce.mce_run_prepared(hd)
    mce.mce_destroy(hd)
    assert tot.count == gold["count"] and "0x%016x" % tot.hash == gold["hash"]
    for i, gg in enumerate(gold["graphs"]):
        assert per[i].count == gg["count"], i
        assert "0x%016x" % per[i].hash == gg["hash"], i
        assert per[i].max_size == gg["max_size"], i
        want = np.zeros(hist.shape[1], np.uint64)
        for k, v in gg["hist"].items():
            want[int(k)] = v
        assert np.array_equal(hist[i], want), i
