"""Python front for the CPU oracle (oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg import this package. It shares nothing with the GPU engine.
"""
import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

PIVOT_FULL, PIVOT_IP, NO_PIVOT = 0, 1, 2
SECOND_LEVEL = 8  # or-ed into a mode: one subtree per edge (Algorithm 4)

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_validate.argtypes = [ctypes.c_int32, i32p, i32p]
        lib.oracle_peel.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p]
        lib.oracle_peel.restype = ctypes.c_int64
        lib.oracle_mce.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                   u64p, u64p, u64p, ctypes.c_int32, i32p, u64p, u64p, u64p]
        lib.oracle_mce_roots.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                         i32p, ctypes.c_int64, u64p, u64p, u64p, ctypes.c_int32,
                                         i32p, u64p, u64p, u64p]
        lib.oracle_mce_work.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                        i32p, ctypes.c_int64, u64p, u64p]
        lib.oracle_multipartite.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, u64p, u64p]
        lib.oracle_clique_hash.argtypes = [i32p, ctypes.c_int32]
        lib.oracle_clique_hash.restype = ctypes.c_uint64
        lib.oracle_default_threads.restype = ctypes.c_int32
        lib.oracle_mce_capped.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p,
                                          ctypes.c_int64, ctypes.c_uint64, u64p, u64p, u64p]
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_tree_estimate.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                             i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, dp, dp]
        _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _u64(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


@dataclass
class Result:
    count: int
    hash: int
    hist: np.ndarray          # hist[k] = number of maximal cliques of size k
    max_size: int
    root_count: Optional[np.ndarray] = None   # per input vertex id
    root_hash: Optional[np.ndarray] = None
    root_nodes: Optional[np.ndarray] = None


def validate(row_ptr, col) -> bool:
    rp, rpp = _i32(row_ptr)
    c, cp = _i32(col if len(col) else np.zeros(1, np.int32))
    return _load().oracle_validate(len(rp) - 1, rpp, cp) == 0


def peel(row_ptr, col):
    """(core, rank, order, sub_rounds) of the level-synchronous peel."""
    rp, rpp = _i32(row_ptr)
    c, cp = _i32(col if len(col) else np.zeros(1, np.int32))
    n = len(rp) - 1
    core = np.zeros(max(n, 1), np.int32)
    rank = np.zeros(max(n, 1), np.int32)
    order = np.zeros(max(n, 1), np.int32)
    P = ctypes.POINTER(ctypes.c_int32)
    rounds = _load().oracle_peel(n, rpp, cp, core.ctypes.data_as(P), rank.ctypes.data_as(P),
                                 order.ctypes.data_as(P))
    if rounds < 0:
        raise MemoryError("oracle_peel failed")
    return core[:n], rank[:n], order[:n], int(rounds)


def mce(row_ptr, col, mode: int = PIVOT_FULL, threads: int = 0, per_root: bool = False,
        roots=None, hist_len: int = 0, level: int = 1) -> Result:
    """All maximal cliques (or those of the listed roots' subtrees). level 2:
    one subtree per edge (Algorithm 4); per-root values sum a vertex's edges."""
    if level == 2:
        mode |= SECOND_LEVEL
    rp, rpp = _i32(row_ptr)
    c, cp = _i32(col if len(col) else np.zeros(1, np.int32))
    n = len(rp) - 1
    if hist_len <= 0:
        hist_len = int(np.diff(rp).max()) + 2 if n else 2
    hist = np.zeros(hist_len, np.uint64)
    cnt = ctypes.c_uint64()
    hsh = ctypes.c_uint64()
    mx = ctypes.c_int32()
    rc_arr = rh_arr = rn_arr = None
    if per_root:
        rc_arr = np.zeros(max(n, 1), np.uint64)
        rh_arr = np.zeros(max(n, 1), np.uint64)
        rn_arr = np.zeros(max(n, 1), np.uint64)
    lib = _load()
    if roots is None:
        rc = lib.oracle_mce(n, rpp, cp, mode, threads, ctypes.byref(cnt), ctypes.byref(hsh),
                            _u64(hist), hist_len, ctypes.byref(mx), _u64(rc_arr), _u64(rh_arr),
                            _u64(rn_arr))
    else:
        ro, rop = _i32(roots)
        rc = lib.oracle_mce_roots(n, rpp, cp, mode, threads, rop, len(ro), ctypes.byref(cnt),
                                  ctypes.byref(hsh), _u64(hist), hist_len, ctypes.byref(mx),
                                  _u64(rc_arr), _u64(rh_arr), _u64(rn_arr))
    if rc == 1:
        raise ValueError("oracle: invalid graph")
    if rc == 2:
        raise MemoryError("oracle: out of memory")
    if rc == 5:
        raise RuntimeError("oracle: hist_len too short")
    res = Result(int(cnt.value), int(hsh.value), hist[: mx.value + 1].copy(), int(mx.value))
    if per_root:
        res.root_count, res.root_hash, res.root_nodes = rc_arr[:n], rh_arr[:n], rn_arr[:n]
    return res


def work(row_ptr, col, mode: int = PIVOT_IP, threads: int = 0, roots=None):
    """(root_nodes, root_work) uint64 per input vertex id; see oracle_mce_work."""
    rp, rpp = _i32(row_ptr)
    c, cp = _i32(col if len(col) else np.zeros(1, np.int32))
    n = len(rp) - 1
    rn = np.zeros(max(n, 1), np.uint64)
    rw = np.zeros(max(n, 1), np.uint64)
    if roots is None:
        rop, nr = None, 0
    else:
        ro, rop = _i32(roots)
        nr = len(ro)
    rc = _load().oracle_mce_work(n, rpp, cp, mode, threads, rop, nr, _u64(rn), _u64(rw))
    if rc != 0:
        raise RuntimeError("oracle_mce_work failed: %d" % rc)
    return rn[:n], rw[:n]


def capped(row_ptr, col, roots, node_cap: int, mode: int = PIVOT_IP, threads: int = 0):
    """Per-root (count, hash, nodes) uint64 arrays by input id for the listed
    roots; a root needing more than node_cap calls is abandoned and gets
    nodes = 2^64 - 1 (count and hash 0)."""
    rp, rpp = _i32(row_ptr)
    c, cp = _i32(col if len(col) else np.zeros(1, np.int32))
    ro, rop = _i32(roots)
    n = len(rp) - 1
    rc_a, rh_a, rn_a = (np.zeros(max(n, 1), np.uint64) for _ in range(3))
    rc = _load().oracle_mce_capped(n, rpp, cp, mode, threads, rop, len(ro), ctypes.c_uint64(node_cap),
                                   _u64(rc_a), _u64(rh_a), _u64(rn_a))
    if rc == 1:
        raise ValueError("oracle: invalid graph or arguments")
    if rc != 0:
        raise MemoryError("oracle_mce_capped failed")
    return rc_a[:n], rh_a[:n], rn_a[:n]


def tree_estimate(row_ptr, col, roots, probes: int = 64, seed: int = 1, mode: int = PIVOT_IP, threads: int = 0):
    """Knuth's estimate of each root's first-level subtree size (tree nodes):
    (mean, variance of one path's estimate), float64 per listed root."""
    rp, rpp = _i32(row_ptr)
    c, cp = _i32(col if len(col) else np.zeros(1, np.int32))
    ro, rop = _i32(roots)
    mean = np.zeros(max(len(ro), 1), np.float64)
    var = np.zeros(max(len(ro), 1), np.float64)
    D = ctypes.POINTER(ctypes.c_double)
    rc = _load().oracle_tree_estimate(len(rp) - 1, rpp, cp, mode, threads, rop, len(ro), int(probes),
                                      ctypes.c_uint64(seed), mean.ctypes.data_as(D), var.ctypes.data_as(D))
    if rc == 1:
        raise ValueError("oracle: invalid graph or arguments")
    if rc != 0:
        raise MemoryError("oracle_tree_estimate failed")
    return mean[:len(ro)], var[:len(ro)]


def multipartite(first: int, parts: int, part_size: int):
    """(count, hash) of the maximal cliques of a complete multipartite graph."""
    c, h = ctypes.c_uint64(), ctypes.c_uint64()
    if _load().oracle_multipartite(first, parts, part_size, ctypes.byref(c), ctypes.byref(h)) != 0:
        raise ValueError("bad multipartite arguments")
    return int(c.value), int(h.value)


def clique_hash(ids) -> int:
    a, ap = _i32(ids)
    return int(_load().oracle_clique_hash(ap, len(a)))


def default_threads() -> int:
    return int(_load().oracle_default_threads())
