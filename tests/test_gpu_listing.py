"""Clique listing (mce_run_list) on the GPU.

A listed set is checked on its own terms, with no reference listing: every
record is a clique of the graph, maximal (no vertex outside it is adjacent
to all of it), and no record repeats. With the oracle's count and hash on
top, a set of distinct maximal cliques of the right size is M(G) itself.
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


def check_listing(g, cliques, o):
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    seen = set()
    total = 0
    for c in cliques:
        c = [int(x) for x in c]
        key = tuple(sorted(c))
        assert len(set(c)) == len(c) and key not in seen
        seen.add(key)
        for i, a in enumerate(c):
            for b in c[i + 1:]:
                assert b in adj[a]
        common = set.intersection(*(adj[a] for a in c)) if c else set()
        assert not (common - set(c)), "not maximal"
        total = (total + h_clique(c)) & M64
    assert len(cliques) == o.count
    assert total == o.hash


GRAPHS = [lambda: gen.worked_example(), lambda: gen.moon_moser(5), lambda: gen.gnp(300, 0.05, 3),
          lambda: gen.disjoint_union([gen.gnp(200, 0.08, 4), gen.complete(12), gen.moon_moser(7)]),
          lambda: gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5)]


@pytest.mark.parametrize("make", GRAPHS)
@pytest.mark.parametrize("pivot", [mce.MCE_PIVOT_IP, mce.MCE_PIVOT_IPX], ids=["IP", "IPX"])
def test_listing_is_the_set_of_maximal_cliques(make, pivot):
    g = make()
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    cl = mce.list_maximal_cliques(g.row_ptr, g.col, pivot=pivot)
    check_listing(g, cl, o)


def test_listing_under_many_donations():
    g = gen.disjoint_union([gen.chung_lu(3000, 12.0, 2.1, 400.0, 4, 12, 24, 5), gen.moon_moser(9)])
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    cl = mce.list_maximal_cliques(g.row_ptr, g.col, blocks=2, donate_min_p=3)
    check_listing(g, cl, o)


def test_listing_in_pieces_and_range_error():
    g = gen.gnp(400, 0.06, 9)
    o = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    h = mce.mce_create(g.row_ptr, g.col)
    try:
        r, need = mce.mce_run_list(h, None)
        assert r.count == o.count and r.hash == o.hash
        assert need == int(sum((k + 1) * int(c) for k, c in enumerate(o.hist)))
        small = torch.zeros(need // 2, dtype=torch.int32, device="cuda")
        with pytest.raises(mce.MCEError) as ei:
            mce.mce_run_list(h, small)
        assert ei.value.code == mce.MCE_ERANGE
        full = torch.zeros(need, dtype=torch.int32, device="cuda")
        r2, w2 = mce.mce_run_list(h, full)
        assert w2 == need and r2.count == o.count
    finally:
        mce.mce_destroy(h)
    # root subsets partition the cliques: a tiny limit forces many pieces
    cl = mce.list_maximal_cliques(g.row_ptr, g.col, max_words=need // 7)
    check_listing(g, cl, o)
