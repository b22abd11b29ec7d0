"""mce_peel_noalloc: the degeneracy peel for callers that cannot allocate
device memory (their memory is owned by a pool that reserves the GPU up
front, or they only get the buffers another framework hands them). Its
scratch is a static device array inside the library; its results must equal
the CPU oracle's peel and those of the allocating path (mce_create +
mce_get_order), call after call, since every call reuses the same array.

The file name keeps this module last in pytest's collection order, so a run
that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2212_01473_gb300 as mce  # noqa: E402


def reference_order(g):
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    h = mce.mce_create(rp, col)
    core, rank, _ = mce.mce_get_order(h)
    mce.mce_destroy(h)
    order = np.empty(g.n, np.int32)
    order[rank] = np.arange(g.n, dtype=np.int32)
    return core, rank, order


def noalloc_order(g):
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    outs = [torch.full((g.n,), -1, dtype=torch.int32, device="cuda") for _ in range(3)]
    mce.mce_peel_noalloc(rp, col, *outs)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in outs]


def oracle_order(g):
    core, rank, order, _ = oracle.peel(g.row_ptr, g.col)
    return core, rank, order


def test_noalloc_peel_equals_oracle_and_allocating_path_on_consecutive_calls():
    big = gen.workload("chunglu_200k")
    small = gen.workload("er_2000")
    ref_big, ref_small = oracle_order(big), oracle_order(small)
    for a, b in zip(reference_order(big), ref_big):
        assert np.array_equal(a, b)
    # two calls in a row on one graph, then another graph, then the first again:
    # whatever the previous call left in the shared array must not leak through
    for g, ref in ((big, ref_big), (big, ref_big), (small, ref_small), (big, ref_big)):
        got = noalloc_order(g)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_noalloc_peel_across_every_peel_stage():
    # full grid, 16 blocks and one block, with a k jump in each stage
    g = gen.peel_stages()
    ref = oracle_order(g)
    for a, b, c in zip(noalloc_order(g), reference_order(g), ref):
        assert np.array_equal(a, c) and np.array_equal(b, c)


def test_noalloc_peel_rejects_graphs_beyond_its_capacity():
    lib = mce.library()
    n = (1 << 20) + 1
    rc = lib.mce_peel_noalloc(None, None, n, 0, None, None, None, None)
    assert rc == mce.MCE_EUNSUPPORTED
    assert b"MCE_NOALLOC_MAX_VERTICES" in lib.mce_last_error()


def test_noalloc_peel_rejects_invalid_graph():
    g = gen.gnp(60, 0.2, 4)
    rp = torch.from_numpy(g.row_ptr).cuda()
    bad = g.col.copy()
    bad[0], bad[1] = bad[1], bad[0]
    col = torch.from_numpy(bad).cuda()
    outs = [torch.zeros(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
    with pytest.raises(mce.MCEError) as ei:
        mce.mce_peel_noalloc(rp, col, *outs)
    assert ei.value.code == mce.MCE_EINVAL
