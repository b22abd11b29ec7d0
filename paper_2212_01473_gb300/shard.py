"""Sharding the enumeration across ranks, one GPU per rank (Sec. IV-D).

First-level subtrees partition the maximal cliques: each clique is found in
the subtree of its earliest vertex in the degeneracy order (Algorithm 3).
So ranks that enumerate disjoint root sets need no exchange while they work,
and one sum at the end gives the whole result: the count and the histogram
add up, and the clique hash is a sum modulo 2^64, so adding the per-rank
values as wrapping 64-bit integers is exact.

The paper assigns roots to GPUs round robin. Here a root set can also be cut
by predicted work (longest processing time first): roots in descending order
of weight, each to the rank with the least work so far.
"""
import heapq
from typing import Callable, List, Optional, Tuple

import numpy as np

M64 = (1 << 64) - 1


def partition_roots(weights, world: int, mode: str = "lpt") -> List[np.ndarray]:
    """Split roots 0..len(weights)-1 into `world` disjoint sets (input vertex
    ids, ascending within a set). mode "round_robin": root i to rank
    i mod world (the paper's assignment); "lpt": by descending weight, each
    to the least-loaded rank (ties to the lower rank; equal weights by
    ascending id)."""
    w = np.asarray(weights, dtype=np.float64)
    n = len(w)
    if world < 1:
        raise ValueError("world must be >= 1")
    if mode == "round_robin":
        return [np.arange(r, n, world, dtype=np.int32) for r in range(world)]
    if mode != "lpt":
        raise ValueError("mode is 'lpt' or 'round_robin'")
    order = np.lexsort((np.arange(n), -w))  # descending weight, then ascending id
    heap = [(0.0, r) for r in range(world)]
    parts: List[list] = [[] for _ in range(world)]
    for v in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(v))
        heapq.heappush(heap, (load + float(w[v]), r))
    return [np.sort(np.asarray(p, dtype=np.int32)) for p in parts]


def reduce_results(count: int, hash_: int, hist, dist=None, device="cpu") -> Tuple[int, int, np.ndarray]:
    """Sum (count, hash, hist) over all ranks in one all-reduce of 64-bit
    words (wrapping: exact modulo 2^64). hist must have the same length on
    every rank."""
    h = np.asarray(hist, dtype=np.uint64)
    if dist is None:
        return int(count), int(hash_) & M64, h.copy()
    import torch
    words = np.concatenate([np.array([count & M64, hash_ & M64], dtype=np.uint64), h])
    t = torch.from_numpy(words.view(np.int64).copy()).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = t.cpu().numpy().view(np.uint64)
    return int(out[0]), int(out[1]), out[2:].copy()


def sharded_enumerate(row_ptr, col, dist=None, weights=None, mode: str = "lpt",
                      compute: Optional[Callable] = None, device="cpu"):
    """Every maximal clique of the graph, each rank enumerating its share of
    the first-level subtrees, then one reduction. weights: per-vertex work
    estimate (default: the degree); compute(row_ptr, col, roots, hist_len) ->
    (count, hash, hist) enumerates one root set (default: the GPU engine).
    Returns (count, hash, hist, this rank's roots)."""
    rank = dist.get_rank() if dist is not None else 0
    world = dist.get_world_size() if dist is not None else 1
    rp = np.asarray(row_ptr)
    deg = np.diff(rp)
    hist_len = int(deg.max()) + 2 if len(deg) else 2
    if weights is None:
        weights = deg
    roots = partition_roots(weights, world, mode)[rank]
    if compute is None:
        compute = _engine_compute
    c, h, hist = compute(row_ptr, col, roots, hist_len)
    hist = np.asarray(hist, dtype=np.uint64)
    full = np.zeros(hist_len, np.uint64)
    full[:min(len(hist), hist_len)] = hist[:hist_len]
    c, h, full = reduce_results(c, h, full, dist, device)
    return c, h, full, roots


def _engine_compute(row_ptr, col, roots, hist_len):
    from .engine import enumerate_maximal_cliques
    r = enumerate_maximal_cliques(row_ptr, col, roots=roots)
    return r.count, r.hash, r.hist
