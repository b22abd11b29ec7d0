"""Per-root features of the work estimator, from their definitions --
TEST INFRASTRUCTURE ONLY (plain Python sets; small graphs).

For a root v with P0 = later and X0 = earlier neighbours in the oracle's
degeneracy order (oracle_peel), the 16 int32 features listed in
include/mce.h, saturating at 2^31 - 1 (features 4, 6 and 14 use X0', the
256 smallest input ids of X0).
"""
import numpy as np

from . import peel

I32 = 2 ** 31 - 1
XCAP = 256  # features 4, 6 and 14 look at X0' = the XCAP smallest input ids of X0


def root_features(row_ptr, col):
    core, rank, order, _ = peel(row_ptr, col)
    n = len(row_ptr) - 1
    nb = [set(col[row_ptr[v]:row_ptr[v + 1]].tolist()) for v in range(n)]
    deg = [len(s) for s in nb]
    out = np.zeros((n, 16), np.int64)
    for v in range(n):
        P0 = [u for u in nb[v] if rank[u] > rank[v]]
        X0 = [u for u in nb[v] if rank[u] < rank[v]]
        Ps = set(P0)
        dP = {u: len(nb[u] & Ps) for u in P0}
        eP = sum(dP.values()) // 2
        X0c = sorted(X0)[:XCAP]  # X0': the smallest input ids of X0
        xc = [len(nb[x] & Ps) for x in X0c]
        eX = sum(xc)
        k = len(P0)
        pairs = k * (k - 1) // 2
        f = [deg[v], int(core[v]), k, len(X0), eP + eX, eP, eX,
             (eP * 65536) // pairs if pairs else 0,
             sum(deg[u] for u in nb[v]),
             max(dP.values()) if k else 0, min(dP.values()) if k else 0,
             sum(1 for u in P0 if dP[u] == k - 1),
             max((int(core[u]) for u in P0), default=0), sum(int(core[u]) for u in P0),
             max(xc, default=0), pairs - eP]
        out[v] = [min(x, I32) for x in f]
    return out
