"""Root sharding across ranks (paper_2212_01473_gb300/shard.py), checked on
CPU: two gloo ranks each enumerate their share of the first-level subtrees
(here with the CPU oracle standing in for one GPU each) and one all-reduce of
64-bit words must give the oracle's whole-graph count, hash and histogram."""
import os
import socket
import sys

import numpy as np
import pytest

import gen
import oracle
from paper_2212_01473_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def oracle_compute(row_ptr, col, roots, hist_len):
    r = oracle.mce(row_ptr, col, mode=oracle.PIVOT_IP, roots=roots, hist_len=hist_len)
    return r.count, r.hash, r.hist


def _rank(rank, world, port, mode, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = gen.chung_lu(3000, 12.0, 2.1, 300.0, 3, 10, 20, 4)
        c, h, hist, roots = shard.sharded_enumerate(g.row_ptr, g.col, dist, mode=mode, compute=oracle_compute)
        out[rank] = (c, h, hist.tolist(), roots.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["lpt", "round_robin"])
def test_two_ranks_sum_to_the_whole_graph(mode):
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, mode, out), nprocs=world, join=True)
        res = dict(out)
    g = gen.chung_lu(3000, 12.0, 2.1, 300.0, 3, 10, 20, 4)
    whole = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    roots = [set(res[r][3]) for r in range(world)]
    assert not (roots[0] & roots[1]) and roots[0] | roots[1] == set(range(g.n))
    for r in range(world):
        c, h, hist, _ = res[r]
        assert (c, h) == (whole.count, whole.hash)
        assert np.array_equal(np.asarray(hist, np.uint64)[:len(whole.hist)], whole.hist)
        assert not any(hist[len(whole.hist):])
    # the shares are real work on both ranks
    parts = [oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP, roots=np.array(sorted(x), np.int32)).count
             for x in roots]
    assert all(p > 0 for p in parts) and sum(parts) == whole.count


def test_hash_sum_wraps_modulo_2_64():
    # two halves whose hash sum overflows 64 bits reduce to the sum mod 2^64
    c, h, hist = shard.reduce_results(3, (1 << 64) - 5, [0, 1, 2])
    assert (c, h) == (3, (1 << 64) - 5) and hist.tolist() == [0, 1, 2]
    a = np.array([(1 << 64) - 5, 9], dtype=np.uint64)
    assert int((a.view(np.int64).sum()).astype(np.int64).view(np.uint64)) == 4


def test_lpt_partition_properties():
    rs = np.random.default_rng(0)
    w = rs.pareto(1.5, 1000) + 1.0
    for world in (1, 2, 3, 8):
        parts = shard.partition_roots(w, world, "lpt")
        ids = np.concatenate(parts)
        assert sorted(ids.tolist()) == list(range(len(w)))
        loads = [w[p].sum() for p in parts]
        # longest processing time first: no rank exceeds another by more than one job
        assert max(loads) - min(loads) <= w.max() + 1e-9
        # and the makespan is within Graham's 4/3 bound of the trivial lower bound
        assert max(loads) <= (4 / 3) * max(w.sum() / world, w.max()) + 1e-9
    rr = shard.partition_roots(w, 3, "round_robin")
    assert [p.tolist()[:3] for p in rr] == [[0, 3, 6], [1, 4, 7], [2, 5, 8]]
