"""Seeded synthetic graph inputs shared by the GPU engine and the CPU oracle.

Nothing here computes cliques: these functions only produce canonical CSR
graphs (``row_ptr`` int32 [n+1], ``col`` int32 [row_ptr[n]], rows sorted,
symmetric, simple). The large families come from ``gen.c`` (compiled by
``gen/build.py``); the small closed-form families are plain numpy.

Named workloads (the shapes of the paper's evaluation graphs, Table I, which
range over |V| 1.6M-428M, mean degree 2-55, degeneracy 47-1,120 and
max-degree/degeneracy 12-3,814):

* ``er_2000``       G(n=2000, m=20000), seed 0
* ``chunglu_1m``    Chung-Lu n=1e6, mean degree 16, exponent 2.1, weight cap
                    20,000, 50 planted cliques of size U[20,40], seed 1
* ``chunglu_200k``  the same family at n=200,000, cap 4,000, 10 planted cliques
                    (a small case for kernel profiles), seed 1
* ``rmat_22``       R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), seed 2
* ``batch_4096``    4096 G(n,p) graphs, n power-law on [50,5000] (density
                    proportional to n^-2), mean degree U[5,60], one in eight
                    joined with a Moon-Moser K_{3,..,3} block on 15/30/45
                    vertices, seed 3
"""
import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        i32p = P(ctypes.c_int32)
        lib.gen_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, P(i32p), P(i32p)]
        lib.gen_chunglu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                    P(i32p), P(i32p)]
        lib.gen_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint64, P(i32p), P(i32p)]
        lib.gen_batch.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                  P(i32p), P(i32p), P(i32p), i32p]
        lib.gen_gnp.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P(i32p), P(i32p)]
        lib.gen_free.argtypes = [ctypes.c_void_p]
        lib.gen_log_for_test.argtypes = [ctypes.c_double]
        lib.gen_log_for_test.restype = ctypes.c_double
        lib.gen_exp_for_test.argtypes = [ctypes.c_double]
        lib.gen_exp_for_test.restype = ctypes.c_double
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Canonical CSR graph (int32). ``graph_ptr`` is set for batches."""
    row_ptr: np.ndarray
    col: np.ndarray
    name: str = ""
    graph_ptr: Optional[np.ndarray] = None
    mm_sizes: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def _take(rp, cp, n: int):
    lib = _load()
    nnz = int(rp[n]) if n >= 0 else 0
    row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(cp, shape=(max(nnz, 1),))[:nnz].copy() if nnz else np.zeros(0, np.int32)
    lib.gen_free(ctypes.cast(rp, ctypes.c_void_p))
    lib.gen_free(ctypes.cast(cp, ctypes.c_void_p))
    return row_ptr, col


def _ptrs():
    i32p = ctypes.POINTER(ctypes.c_int32)
    return i32p(), i32p()


def er(n: int, m: int, seed: int) -> Graph:
    rp, cp = _ptrs()
    if _load().gen_er(n, m, seed, ctypes.byref(rp), ctypes.byref(cp)) != 0:
        raise ValueError("gen_er failed")
    row_ptr, col = _take(rp, cp, n)
    return Graph(row_ptr, col, name="er_%d_%d_s%d" % (n, m, seed))


def chung_lu(n: int, mean_deg: float, gamma: float, wcap: float, n_planted: int, kmin: int,
             kmax: int, seed: int) -> Graph:
    rp, cp = _ptrs()
    if _load().gen_chunglu(n, mean_deg, gamma, wcap, n_planted, kmin, kmax, seed,
                           ctypes.byref(rp), ctypes.byref(cp)) != 0:
        raise ValueError("gen_chunglu failed")
    row_ptr, col = _take(rp, cp, n)
    return Graph(row_ptr, col, name="chunglu_%d_s%d" % (n, seed))


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int) -> Graph:
    rp, cp = _ptrs()
    if _load().gen_rmat(scale, edge_factor, a, b, c, seed, ctypes.byref(rp), ctypes.byref(cp)) != 0:
        raise ValueError("gen_rmat failed")
    row_ptr, col = _take(rp, cp, 1 << scale)
    return Graph(row_ptr, col, name="rmat_%d_%d_s%d" % (scale, edge_factor, seed))


def gnp(n: int, p: float, seed: int) -> Graph:
    rp, cp = _ptrs()
    if _load().gen_gnp(n, p, seed, ctypes.byref(rp), ctypes.byref(cp)) != 0:
        raise ValueError("gen_gnp failed")
    row_ptr, col = _take(rp, cp, n)
    return Graph(row_ptr, col, name="gnp_%d_%g_s%d" % (n, p, seed))


def batch(G: int, seed: int, nmin: float = 50, nmax: float = 5000, alpha: float = 2.0,
          dmin: float = 5, dmax: float = 60, mm_every: int = 8) -> Graph:
    lib = _load()
    i32p = ctypes.POINTER(ctypes.c_int32)
    gp, rp, cp = i32p(), i32p(), i32p()
    mm = np.zeros(G, np.int32)
    if lib.gen_batch(G, nmin, nmax, alpha, dmin, dmax, mm_every, seed, ctypes.byref(gp),
                     ctypes.byref(rp), ctypes.byref(cp),
                     mm.ctypes.data_as(i32p)) != 0:
        raise ValueError("gen_batch failed")
    graph_ptr = np.ctypeslib.as_array(gp, shape=(G + 1,)).copy()
    lib.gen_free(ctypes.cast(gp, ctypes.c_void_p))
    n = int(graph_ptr[-1])
    row_ptr, col = _take(rp, cp, n)
    return Graph(row_ptr, col, name="batch_%d_s%d" % (G, seed), graph_ptr=graph_ptr, mm_sizes=mm)


# ------------------------------------------------------------ named workloads

def workload(name: str, seed: Optional[int] = None) -> Graph:
    """The named synthetic workloads (see module docstring)."""
    if name == "er_2000":
        return er(2000, 20000, 0 if seed is None else seed)
    if name == "chunglu_1m":
        return chung_lu(1_000_000, 16.0, 2.1, 20000.0, 50, 20, 40, 1 if seed is None else seed)
    if name == "chunglu_200k":  # a small case of the same family, for profiling
        return chung_lu(200_000, 16.0, 2.1, 4000.0, 10, 20, 40, 1 if seed is None else seed)
    if name == "rmat_22":
        return rmat(22, 16, 0.57, 0.19, 0.19, 2 if seed is None else seed)
    if name == "batch_4096":
        return batch(4096, 3 if seed is None else seed)
    raise KeyError(name)


# ------------------------------------------------- small closed-form graphs

def from_edges(n: int, edges, name: str = "") -> Graph:
    """Canonical CSR from an iterable of undirected pairs (self-loops dropped,
    duplicates merged)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    if e.size:
        e = e[e[:, 0] != e[:, 1]]
        both = np.concatenate([e, e[:, ::-1]], axis=0)
        key = np.unique(both[:, 0] * (n + 1) + both[:, 1])
        src = key // (n + 1)
        dst = key % (n + 1)
    else:
        src = dst = np.zeros(0, np.int64)
    counts = np.bincount(src, minlength=n) if n else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(counts)
    return Graph(row_ptr.astype(np.int32), dst.astype(np.int32), name=name)


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], "K%d" % n)


def empty(n: int) -> Graph:
    return from_edges(n, [], "E%d" % n)


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], "C%d" % n)


def multipartite(parts: int, part_size: int) -> Graph:
    """Complete multipartite graph with `parts` parts of `part_size` vertices;
    vertex x is in part x // part_size. part_size 3 gives Moon-Moser graphs,
    part_size 2 cocktail-party graphs."""
    n = parts * part_size
    e = [(x, y) for x in range(n) for y in range(x + 1, n) if x // part_size != y // part_size]
    return from_edges(n, e, "K%dx%d" % (parts, part_size))


def moon_moser(k: int) -> Graph:
    return multipartite(k, 3)


def worked_example() -> Graph:
    """Six vertices A..F = 0..5: ABCD is a 4-clique, AEF a triangle."""
    A, B, C, D, E, F = range(6)
    e = [(A, B), (A, C), (A, D), (B, C), (B, D), (C, D), (A, E), (A, F), (E, F)]
    return from_edges(6, e, "worked_example")


def random_forest(n: int, seed: int, p_edge: float = 0.8) -> Graph:
    """Each vertex i > 0 attaches to a uniform earlier vertex with prob p_edge."""
    rs = np.random.default_rng(seed)
    e = [(i, int(rs.integers(0, i))) for i in range(1, n) if rs.random() < p_edge]
    return from_edges(n, e, "forest_%d_s%d" % (n, seed))


def small_gnp(n: int, p: float, seed: int) -> Graph:
    rs = np.random.default_rng(seed)
    e = [(i, j) for i in range(n) for j in range(i + 1, n) if rs.random() < p]
    return from_edges(n, e, "sgnp_%d_%g_s%d" % (n, p, seed))


def disjoint_union(graphs: List[Graph]) -> Graph:
    """Concatenate graphs; sets graph_ptr to the vertex offsets."""
    offs = [0]
    rps, cols = [], []
    eoff = 0
    for g in graphs:
        rps.append(g.row_ptr[:-1].astype(np.int64) + eoff)
        cols.append(g.col.astype(np.int64) + offs[-1])
        eoff += int(g.row_ptr[-1])
        offs.append(offs[-1] + g.n)
    row_ptr = np.concatenate(rps + [np.array([eoff])]).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return Graph(row_ptr, col, name="union", graph_ptr=np.array(offs, np.int32))


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Vertex v becomes perm[v]."""
    src = np.repeat(np.arange(g.n), g.degrees())
    e = np.stack([perm[src], perm[g.col]], axis=1)
    e = e[e[:, 0] < e[:, 1]]
    return from_edges(g.n, e.tolist(), g.name + "_perm")


def stats(g: Graph) -> dict:
    deg = g.degrees()
    return {"n": g.n, "m": g.m, "max_deg": int(deg.max()) if g.n else 0,
            "isolated": int((deg == 0).sum()), "mean_deg": float(deg.mean()) if g.n else 0.0}


def peel_stages(seed: int = 21) -> Graph:
    """G(n, m) with n = 300,000 and m = 2.2M, plus K_30, K_50, K_60 and K_170.

    Once G(n, m) is peeled, 410 vertices remain, with live degree sums
    35,590, 34,720, 32,270 and 28,730 at the cliques' levels. The smallest
    live degree jumps past k + 1 at the first level and at each clique.
    """
    return disjoint_union([er(300000, 2200000, seed), complete(30), complete(50), complete(60), complete(170)])
