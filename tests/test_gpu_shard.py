"""Sharded enumeration through the GPU engine: the root sets of three ranks,
run one after another on this GPU, sum to the whole graph's results (the
CPU oracle's), for both partitions of paper_2212_01473_gb300/shard.py."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2212_01473_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("mode", ["lpt", "round_robin"])
def test_three_shards_sum_to_oracle(mode):
    g = gen.chung_lu(20000, 16.0, 2.1, 1500.0, 4, 20, 30, 21)
    whole = oracle.mce(g.row_ptr, g.col, mode=oracle.PIVOT_IP)
    hist_len = int(np.diff(g.row_ptr).max()) + 2
    c, h, hist = 0, 0, np.zeros(hist_len, np.uint64)
    for roots in shard.partition_roots(np.diff(g.row_ptr), 3, mode):
        rc, rh, rhist = shard._engine_compute(g.row_ptr, g.col, roots, hist_len)
        c += rc
        h = (h + rh) & shard.M64
        hist[:len(rhist)] += np.asarray(rhist, np.uint64)
    assert (c, h) == (whole.count, whole.hash)
    assert np.array_equal(hist[:len(whole.hist)], whole.hist)
