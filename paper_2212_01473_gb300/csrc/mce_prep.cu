// Pre-processing on the GPU: CSR validation, degeneracy ordering by
// level-synchronous peeling (Sec. II-C "Degeneracy Ordering"; the paper
// times this step with the enumeration, Sec. IV-A), and orientation of each
// vertex's neighbours into later (root P, Algorithm 3) and earlier (root X)
// lists in rank space.
#include <climits>

#include <cooperative_groups.h>

#include "mce_prep.cuh"

namespace mce {

// ------------------------------------------------------------ validation

__global__ void k_check_rowptr(int n, const int32_t *rp, int64_t m2, int *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    bool bad = false;
    if (i == 0 && rp[0] != 0) bad = true;
    if (i < n && rp[i] > rp[i + 1]) bad = true;
    if (i == n && (int64_t)rp[n] != m2) bad = true;
    if (bad) atomicOr(status, ST_BADGRAPH);
}

// one warp per row: ids in range, no self-loop, strictly ascending, symmetric
__global__ void k_check_cols(int n, const int32_t *rp, const int32_t *col, int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < n; v += nw) {
        const int b = rp[v], e = rp[v + 1];
        bool bad = false;
        for (int j = b + lane; j < e; j += 32) {
            const int32_t u = col[j];
            if (u < 0 || u >= n || u == (int32_t)v) { bad = true; continue; }
            if (j + 1 < e && col[j + 1] <= u) bad = true;
            // symmetric: v in row u
            int lo = rp[u], hi = rp[u + 1];
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (col[mid] < (int32_t)v) lo = mid + 1; else hi = mid;
            }
            if (lo >= rp[u + 1] || col[lo] != (int32_t)v) bad = true;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BADGRAPH);
    }
}

// -------------------------------------------------------------- helpers

__device__ __forceinline__ int warp_push(int *counter, bool pred) {
    // warp-aggregated slot reservation; returns the slot for pred lanes
    const unsigned act = __activemask();
    const unsigned b = __ballot_sync(act, pred);
    const int lane = threadIdx.x & 31;
    int base = 0;
    const int leader = __ffs(act) - 1;
    if (lane == leader && b) base = atomicAdd(counter, __popc(b));
    base = __shfl_sync(act, base, leader);
    return base + __popc(b & ((1u << lane) - 1u));
}

template <int NT>
__device__ __forceinline__ int block_reduce_min(int x, int *sh) {
    for (int o = 16; o; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        x = lane < NT / 32 ? sh[lane] : INT_MAX;
        for (int o = 16; o; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0) sh[0] = x;
    }
    __syncthreads();
    int r = sh[0];
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ int block_reduce_sum(int x, int *sh) {
    x = __reduce_add_sync(0xffffffffu, x);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = x;
    __syncthreads();
    int t = 0;
    for (int i = 0; i < NT / 32; i++) t += sh[i];
    __syncthreads();
    return t;
}

// exclusive block scan; returns prefix, *total = block sum
template <int NT>
__device__ __forceinline__ int block_scan_excl(int x, int *sh, int *total) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    int off = 0, tot = 0;
    for (int i = 0; i < NT / 32; i++) {
        int c = sh[i];
        if (i < w) off += c;
        tot += c;
    }
    __syncthreads();
    *total = tot;
    return off + inc - x;
}

// ---------------------------------------------------------------- peel

constexpr int kPeelThreads = 1024;  // one block per SM: fewer arrivals per grid barrier
constexpr int kRankThreads = 512;
constexpr int kSmallSort = 4096;

__device__ __forceinline__ int vload(const int *p) { return *(volatile const int *)p; }

// bitonic sort of a[0..len) ascending in shared memory by the whole block
__device__ void block_bitonic(int *a, int len) {
    int m = 1;
    while (m < len) m <<= 1;
    for (int i = len + threadIdx.x; i < m; i += blockDim.x) a[i] = INT_MAX;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    int x = a[i], y = a[p];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[p] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// Level-synchronous peel (Sec. II-C). At a level start k = max(k, smallest
// remaining degree) and S = every remaining vertex of degree <= k; each
// sub-round removes S (core number k) and the next S is the set of vertices
// whose degree fell to k while it was removed. Ranks follow the removal
// sub-round, then ascending vertex id inside a sub-round.
//
// One grid barrier per sub-round: a vertex is marked removed (rank = 0, core
// = k) and appended to the next sub-round's segment of `order` by the thread
// whose decrement took its degree from k + 1 to k, so nothing needs a second
// pass. Decrements are unconditional: a removed vertex already has degree
// <= k and never reaches k + 1 again. The three counters of S sizes form a
// ring that every pass and sub-round advances: a phase fills one slot while
// the size filled by the phase before is still being read, and resets the
// third, whose readers all passed the last barrier.
// Segments longer than kSmallSort are put in id order here through a bitmap;
// shorter ones, and all final ranks, are done by k_peel_rank afterwards.
//
// As the remaining graph shrinks, fewer blocks go on. A level start may narrow
// the grid when the live degree sum, the live vertices and the level's S are
// all small: at most kNarrowDegrees, kNarrowLive and kNarrowS. The full grid
// then hands the rest to one cluster of kNarrowBlocks CTAs (k_peel<true>,
// below) whose barriers stay inside the cluster, or, where such a cluster
// cannot be placed, blocks kNarrowBlocks and up return and the rest meet at
// grid barriers among fewer blocks (the dense core's many short sub-rounds are
// barrier-bound). Within kSoloDegrees, kSoloLive and kSoloS, block 0 finishes
// alone with block barriers. A warp removes one vertex at a time, so the stage
// must not start while S sets of thousands of vertices can still come: the
// live vertices bound every later S. Removal order and core numbers are the
// same either way.
constexpr long long kNarrowDegrees = 1ll << 22;
constexpr int kNarrowBlocks = 16;
constexpr int kNarrowLive = 2 * kNarrowBlocks * kPeelThreads;
constexpr int kNarrowS = 2 * kNarrowBlocks * (kPeelThreads / 32);
constexpr long long kSoloDegrees = 32768;
constexpr int kSoloLive = 2 * kPeelThreads;
constexpr int kSoloS = 2 * (kPeelThreads / 32);
// adjacency lists longer than this are removed by a whole block: the warp
// that meets such a vertex queues it for its own block (up to kHeavyCap a
// sub-round; past that, the warp removes it alone)
constexpr int kHeavyDeg = 64;
constexpr int kHeavyCap = 1024;

// ------------------------------------------------ narrow stage as a cluster
// The narrow stage's kNarrowBlocks blocks can run as one thread-block
// cluster, whose barrier needs no round trip to L2: every CTA holds one
// mbarrier expecting one arrival from each CTA; at a barrier, thread t <
// kNarrowBlocks of every CTA arrives (release, cluster scope) on CTA t's
// mbarrier, and thread 0 waits on its own (acquire, cluster scope), with the
// grid barrier's bound and status checks. No CTA may leave the kernel while
// another can still arrive on its mbarrier, so every exit of the cluster
// kernel passes one hardware cluster barrier; every wait before it is
// bounded, so every CTA gets there.
__device__ __forceinline__ void mbar_init(unsigned mb, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool cluster_barrier(unsigned mb, unsigned &phase, int *status, uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x < (unsigned)kNarrowBlocks) {
        unsigned remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(mb), "r"((unsigned)threadIdx.x));
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
    }
    if (threadIdx.x == 0) {
        int ok = 1;
        uint64_t t0 = globaltimer_ns();
        for (unsigned spins = 1;; spins++) {
            unsigned done;
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
                "selp.u32 %0, 1, 0, p; }"
                : "=r"(done)
                : "r"(mb), "r"(phase)
                : "memory");
            if (done) break;
            if ((spins & 63u) == 0) {
                if (ld_relaxed(status) & ST_TIMEOUT) { ok = 0; break; }
                const uint64_t now = globaltimer_ns();
                if (now < t0) {
                    t0 = now;
                } else if (now - t0 > timeout_ns) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    phase ^= 1u;
    return s_ok != 0;
}

// CL = false: the full grid, launched cooperatively; with handoff set, it
// stops where the narrow stage would begin and leaves the state in ctl->rs_*.
// CL = true: one cluster of kNarrowBlocks CTAs that goes on from there (it
// returns at once when the full grid finished alone).
template <bool CL>
__global__ void __launch_bounds__(kPeelThreads) k_peel(int n, const int32_t *rp, const int32_t *col,
                                                       int32_t *deg, int32_t *rank, int32_t *core,
                                                       int32_t *order, int32_t *remA, int32_t *remB,
                                                       int32_t *segstart, unsigned *bitmap, int *blocksums,
                                                       PeelCtl *ctl, int *status, uint64_t timeout_ns,
                                                       int handoff) {
    __shared__ int sh[64];
    __shared__ long long shl[32];
    __shared__ __align__(8) unsigned long long cl_mbar;
    __shared__ int hv_cnt;             // this block's queued heavy vertices in the current sub-round
    __shared__ int32_t hv_beg[kHeavyCap], hv_end[kHeavyCap];  // the queued vertices' adjacency ranges
    if (CL && vload(&ctl->rs_active) == 0) return;  // the full grid finished alone
    // The rings of stage counters (S sizes, remaining-list sizes, level minima
    // and degree sums): in global memory on the full grid; in the cluster, in
    // CTA 0's shared memory, which every CTA reaches through distributed
    // shared memory (no L2 round trip for a push or for reading a size).
    __shared__ int cl_cnt[3], cl_nrem2[3], cl_minval[3];
    __shared__ unsigned long long cl_sumdeg[3];
    int *c_cnt = ctl->cnt, *c_nrem2 = ctl->nrem2, *c_minval = ctl->minval;
    unsigned long long *c_sumdeg = ctl->sumdeg;
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&cl_mbar);
    unsigned mb_phase = 0;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    int64_t nwarps = nth >> 5;
    int nblocks = gridDim.x, bid = blockIdx.x;
    bool solo = false;
    unsigned nbar = gridDim.x;  // blocks meeting at grid barriers
    GridBar *gbar = &ctl->bar;
    unsigned bar_target = 0, bar_gen = 0;  // running copies, the same in every block
    auto barrier = [&]() -> bool {
        if (solo) {
            __syncthreads();
            return true;
        }
        if (CL) return cluster_barrier(mb, mb_phase, status, timeout_ns);
        return grid_barrier(gbar, status, timeout_ns, nbar, bar_target, bar_gen);
    };

    // every block keeps the same copies of these
    // t counts sub-rounds (segments of `order`), r every pass and sub-round,
    // L every level-start pass
    int k = 0, next = 0, nrem = n, t = 0, r = 0, L = 0, ns = 0;
    bool remsel = false;
    // A level start is one pass and one barrier. The pass builds S for a
    // guessed k while it reduces the smallest live degree and the live degree
    // sum. After a level at k every live degree is above k, so the guess k + 1
    // is right whenever a live vertex has degree k + 1. Otherwise S comes out
    // empty, the pass has only compacted the remaining list, and the next pass
    // takes the reduced minimum. The first level guesses 0.
    int guess = 0;
    // the cluster kernel starts at the first sub-round of the level where the
    // full grid stopped
    bool resume = CL;
    if (threadIdx.x == 0) hv_cnt = 0;  // published by the first barrier's block barrier
    if (CL) {
        if (threadIdx.x == 0) mbar_init(mb, kNarrowBlocks);
        if (blockIdx.x == 0 && threadIdx.x == 0)
            for (int i = 0; i < 3; i++) {
                cl_cnt[i] = ctl->cnt[i];
                cl_nrem2[i] = ctl->nrem2[i];
                cl_minval[i] = ctl->minval[i];
                cl_sumdeg[i] = ctl->sumdeg[i];
            }
        // every mbarrier and CTA 0's counters are ready before the first use
        cooperative_groups::this_cluster().sync();
        {
            cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
            c_cnt = cl.map_shared_rank(cl_cnt, 0);
            c_nrem2 = cl.map_shared_rank(cl_nrem2, 0);
            c_minval = cl.map_shared_rank(cl_minval, 0);
            c_sumdeg = cl.map_shared_rank(cl_sumdeg, 0);
        }
        k = ctl->rs_k;
        guess = ctl->rs_guess;
        next = ctl->rs_next;
        nrem = ctl->rs_nrem;
        t = ctl->rs_t;
        r = ctl->rs_r;
        L = ctl->rs_L;
        remsel = ctl->rs_remsel != 0;
        ns = ctl->rs_ns;
        nbar = kNarrowBlocks;
    } else {
        if (tid == 0) ctl->t_start = globaltimer_ns();
        for (int64_t v = tid; v < n; v += nth) {
            deg[v] = rp[v + 1] - rp[v];
            rank[v] = -1;
            remA[v] = (int32_t)v;
        }
        if (!barrier()) goto done;
    }
    while (next < n) {
        if (!resume) {
            const int32_t *rem = remsel ? remB : remA;
            int32_t *rem2 = remsel ? remA : remB;
            const int ls = L % 3;  // this level's slot of nrem2, minval and sumdeg
            int lmin = INT_MAX;
            long long lsum = 0;
            {
                // S of the level into order[next..), the rest into the next remaining list
                int *cnt = &c_cnt[r % 3];
                const int64_t lim = (nrem + 31) / 32 * 32;
                for (int64_t i = tid; i < lim; i += nth) {
                    bool live = false, inS = false;
                    int v = 0;
                    if (i < nrem) {
                        v = rem[i];
                        live = rank[v] < 0;
                        if (live) {
                            const int d = deg[v];
                            lmin = min(lmin, d);
                            lsum += d;
                            inS = d <= guess;
                        }
                    }
                    const int ps = warp_push(cnt, inS);
                    if (inS) {
                        rank[v] = 0;
                        core[v] = guess;
                        order[next + ps] = v;
                    }
                    const int pk = warp_push(&c_nrem2[ls], live && !inS);
                    if (live && !inS) rem2[pk] = v;
                }
            }
            lmin = block_reduce_min<kPeelThreads>(lmin, sh);
            for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if (lane == 0) shl[threadIdx.x >> 5] = lsum;
            __syncthreads();
            if (threadIdx.x == 0) {
                long long bs = 0;
                for (int w = 0; w < kPeelThreads / 32; w++) bs += shl[w];
                if (lmin != INT_MAX) atomicMin(&c_minval[ls], lmin);
                if (bs) atomicAdd(&c_sumdeg[ls], (unsigned long long)bs);
                // slot (L + 1) % 3 was last read after level L - 2's barrier, and
                // every block has since passed level L - 1's
                if (bid == 0) {
                    const int lz = (L + 1) % 3;
                    c_minval[lz] = INT_MAX;
                    c_sumdeg[lz] = 0ull;
                    c_nrem2[lz] = 0;
                    c_cnt[(r + 1) % 3] = 0;
                }
            }
            if (!barrier()) goto done;
            nrem = vload(&c_nrem2[ls]);
            remsel = !remsel;
            L++;
            ns = vload(&c_cnt[r % 3]);
            r++;
            if (ns == 0) {
                // no live vertex has degree `guess`: the level is at the smallest live degree
                guess = vload(&c_minval[ls]);
                continue;
            }
            k = guess;
            guess = k + 1;
            // every block reads the same sum after the barrier and decides alike
            const long long live = (long long)*(volatile unsigned long long *)&c_sumdeg[ls];
            const int nlive = nrem + ns;
            const bool to_solo = !solo && live <= kSoloDegrees && nlive <= kSoloLive && ns <= kSoloS;
            if (!solo && !to_solo && nbar > (unsigned)kNarrowBlocks && live <= kNarrowDegrees && nlive <= kNarrowLive &&
                ns <= kNarrowS) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    ctl->t_narrow = globaltimer_ns();
                    ctl->r_narrow = t;
                }
                if (handoff) {
                    // the cluster kernel goes on from the first sub-round at level k
                    if (blockIdx.x == 0 && threadIdx.x == 0) {
                        ctl->rs_k = k;
                        ctl->rs_guess = guess;
                        ctl->rs_next = next;
                        ctl->rs_nrem = nrem;
                        ctl->rs_t = t;
                        ctl->rs_r = r;
                        ctl->rs_L = L;
                        ctl->rs_remsel = remsel ? 1 : 0;
                        ctl->rs_ns = ns;
                        ctl->rs_active = 1;
                    }
                    goto done;
                }
                if (blockIdx.x >= kNarrowBlocks) goto done;
                nbar = kNarrowBlocks;
                nblocks = kNarrowBlocks;
                tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
                nth = (int64_t)kNarrowBlocks * blockDim.x;
                nwarps = nth >> 5;
            }
            if (to_solo) {
                if (blockIdx.x != 0) goto done;
                if (threadIdx.x == 0) {
                    ctl->t_solo = globaltimer_ns();
                    ctl->r_solo = t;
                }
                solo = true;
                tid = threadIdx.x;
                nth = blockDim.x;
                nwarps = nth >> 5;
                nblocks = 1;
                bid = 0;
            }
        }
        resume = false;

        // sub-rounds at level k
        for (;;) {
            if (bid == 0 && threadIdx.x == 0) {
                // cnt[(r+1)%3] held the size read two phases ago, by every block
                // before the last barrier
                c_cnt[(r + 1) % 3] = 0;
                segstart[t] = next;
            }
            int32_t *S = order + next;
            if (ns > kSmallSort) {
                // ascending id through a bitmap: mark, count per block chunk, compact
                for (int64_t i = tid; i < ns; i += nth) {
                    const int v = S[i];
                    atomicOr(&bitmap[v >> 5], 1u << (v & 31));
                }
                if (!barrier()) goto done;
                const int nw = (n + 31) >> 5;
                const int chunk = (nw + nblocks - 1) / nblocks;
                const int w_lo = min(nw, bid * chunk), w_hi = min(nw, w_lo + chunk);
                int c = 0;
                for (int w = w_lo + threadIdx.x; w < w_hi; w += blockDim.x) c += __popc(bitmap[w]);
                c = block_reduce_sum<kPeelThreads>(c, sh);
                if (threadIdx.x == 0) blocksums[bid] = c;
                if (!barrier()) goto done;
                int off = 0;
                for (int b = threadIdx.x; b < bid; b += blockDim.x) off += blocksums[b];
                off = block_reduce_sum<kPeelThreads>(off, sh);
                for (int t0 = w_lo; t0 < w_hi; t0 += blockDim.x) {
                    const int w = t0 + threadIdx.x;
                    unsigned bits = (w < w_hi) ? bitmap[w] : 0u;
                    int tot;
                    const int pre = block_scan_excl<kPeelThreads>(__popc(bits), sh, &tot);
                    int pos = off + pre;
                    while (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        S[pos++] = w * 32 + b;
                    }
                    if (w < w_hi) bitmap[w] = 0u;
                    off += tot;
                }
                if (!barrier()) goto done;
            }
            // remove S: the vertices whose degree falls to k form the next sub-round.
            // A vertex of degree <= kHeavyDeg is one warp's work (two 32-edge
            // chunks in flight); a longer adjacency list is strided over the
            // block whose warp met it, so no block walks all of S.
            int *cn = &c_cnt[r % 3];
            int32_t *S2 = S + ns;
            auto remove_edge = [&](bool valid, int j) {
                bool push = false;
                int u = 0;
                if (valid) {
                    u = col[j];
                    push = atomicSub(&deg[u], 1) == k + 1;
                }
                const int p = warp_push(cn, push);
                if (push) {
                    rank[u] = 0;
                    core[u] = k;
                    S2[p] = u;
                }
            };
            // warps numbered block-interleaved: vertex i goes to block
            // i % nblocks, so the few hubs of a short sub-round land in
            // different blocks
            const int64_t iw = (int64_t)(threadIdx.x >> 5) * nblocks + bid;
            for (int64_t i = iw; i < ns; i += nwarps) {
                const int v = S[i];
                const int b = rp[v], e = rp[v + 1];
                if (e - b > kHeavyDeg) {
                    int q = 0;
                    if (lane == 0) q = atomicAdd(&hv_cnt, 1);
                    q = __shfl_sync(0xffffffffu, q, 0);
                    if (q < kHeavyCap) {
                        if (lane == 0) {
                            hv_beg[q] = b;
                            hv_end[q] = e;
                        }
                    } else {
                        for (int j0 = b; j0 < e; j0 += 32) remove_edge(j0 + lane < e, j0 + lane);
                    }
                    continue;
                }
                for (int j0 = b; j0 < e; j0 += 64) {
                    const int ja = j0 + lane, jb = ja + 32;
                    const bool va = ja < e, vb = jb < e;
                    int ua = 0, ub = 0;
                    if (va) ua = col[ja];
                    if (vb) ub = col[jb];
                    const bool pa = va && atomicSub(&deg[ua], 1) == k + 1;
                    const bool pb = vb && atomicSub(&deg[ub], 1) == k + 1;
                    const int qa = warp_push(cn, pa);
                    if (pa) {
                        rank[ua] = 0;
                        core[ua] = k;
                        S2[qa] = ua;
                    }
                    const int qb = warp_push(cn, pb);
                    if (pb) {
                        rank[ub] = 0;
                        core[ub] = k;
                        S2[qb] = ub;
                    }
                }
            }
            // the heavy vertices this block's warps queued, each strided over the block
            __syncthreads();
            const int nh = min(hv_cnt, kHeavyCap);
            for (int h = 0; h < nh; h++) {
                const int b = hv_beg[h], e = hv_end[h];
                for (int j0 = b; j0 < e; j0 += blockDim.x) remove_edge(j0 + (int)threadIdx.x < e, j0 + threadIdx.x);
            }
            __syncthreads();
            if (threadIdx.x == 0) hv_cnt = 0;
            if (!barrier()) goto done;
            next += ns;
            t++;
            ns = vload(&c_cnt[r % 3]);
            r++;
            if (ns == 0) break;
        }
    }
    if (bid == 0 && threadIdx.x == 0) {
        ctl->next = next;
        ctl->rounds = t;
        ctl->k = k;
        ctl->t_end = globaltimer_ns();
    }
done:
    // no CTA of the cluster leaves while another can still arrive on its mbarrier
    if (CL) cooperative_groups::this_cluster().sync();
}

// Final ranks: sort each short sub-round segment of `order` by vertex id (the
// long ones are sorted already), then rank[order[i]] = i.
__global__ void __launch_bounds__(kRankThreads) k_peel_rank(int n, const int32_t *segstart, const PeelCtl *ctl,
                                                            int32_t *order, int32_t *rank) {
    __shared__ int ssort[kSmallSort];
    const int rounds = ctl->rounds;
    for (int r = blockIdx.x; r < rounds; r += gridDim.x) {
        const int a = segstart[r], b = r + 1 < rounds ? segstart[r + 1] : n;
        const int len = b - a;
        if (len > 1 && len <= kSmallSort) {
            for (int i = threadIdx.x; i < len; i += blockDim.x) ssort[i] = order[a + i];
            block_bitonic(ssort, len);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                order[a + i] = ssort[i];
                rank[ssort[i]] = a + i;
            }
            __syncthreads();
        } else {
            for (int i = a + threadIdx.x; i < b; i += blockDim.x) rank[order[i]] = i;
        }
    }
}

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_tiles(const int32_t *in, int32_t *out, int32_t *tile_sums, int64_t n) {
    __shared__ int sh[32];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = (t0 + i < n) ? in[t0 + i] : 0;
        s += v[i];
    }
    int tot;
    int pre = block_scan_excl<kScanThreads>(s, sh, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (t0 + i < n) out[t0 + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int32_t *out, const int32_t *tile_off, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    const int add = tile_off[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        int64_t j = i + (int64_t)k * kScanThreads;
        if (j < n) out[j] += add;
    }
}

__global__ void k_set_total(int32_t *out, int64_t n, const int32_t *in) {
    // out[n] = out[n-1] + in[n-1]
    if (n > 0) out[n] = out[n - 1] + in[n - 1];
    else out[0] = 0;
}

// exclusive scan of in[0..n) into out[0..n], out[n] = total; tmp >= scan_tmp_words(n)
cudaError_t exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s) {
    if (n <= 0) {
        k_set_total<<<1, 1, 0, s>>>(out, 0, in);
        count_launch();
        return cudaGetLastError();
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    int32_t *sums = tmp;
    int32_t *offs = tmp + tiles;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, sums, n);
    count_launch();
    if (tiles > 1) {
        cudaError_t e = exclusive_scan(sums, offs, tiles, tmp + 2 * tiles + 1, s);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, offs, n);
        count_launch();
    }
    k_set_total<<<1, 1, 0, s>>>(out, n, in);
    count_launch();
    return cudaGetLastError();
}

int64_t scan_tmp_words(int64_t n) {
    int64_t w = 0;
    while (n > 1) {
        int64_t tiles = (n + kScanTile - 1) / kScanTile;
        w += 2 * tiles + 1;
        n = tiles;
    }
    return w + 4;
}

// ----------------------------------------------------------- orientation

__global__ void k_count_split(int n, const int32_t *rp, const int32_t *col, const int32_t *order,
                              const int32_t *rank, int32_t *outdeg, int32_t *indeg) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw) {
        const int v = order[r];
        const int b = rp[v], e = rp[v + 1];
        int c = 0;
        for (int j = b + lane; j < e; j += 32) c += rank[col[j]] > (int32_t)r;
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) {
            outdeg[r] = c;
            indeg[r] = (e - b) - c;
        }
    }
}

__global__ void k_fill_split(int n, const int32_t *rp, const int32_t *col, const int32_t *order,
                             const int32_t *rank, const int32_t *out_ptr, int32_t *out_col,
                             const int32_t *in_ptr, int32_t *in_col) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw) {
        const int v = order[r];
        const int b = rp[v], e = rp[v + 1];
        int oc = out_ptr[r], ic = in_ptr[r];
        for (int j0 = b; j0 < e; j0 += 32) {
            int j = j0 + lane;
            int ru = 0;
            bool valid = j < e, later = false;
            if (valid) {
                ru = rank[col[j]];
                later = ru > (int32_t)r;
            }
            unsigned bl = __ballot_sync(0xffffffffu, valid && later);
            unsigned be = __ballot_sync(0xffffffffu, valid && !later);
            unsigned lt = (1u << lane) - 1u;
            if (valid && later) out_col[oc + __popc(bl & lt)] = ru;
            if (valid && !later) in_col[ic + __popc(be & lt)] = ru;
            oc += __popc(bl);
            ic += __popc(be);
        }
    }
}

constexpr int kRowSortWarpCap = 1024;
constexpr int kRowSortBlockCap = 4096;

// rows of length <= kRowSortWarpCap: one warp per row, bitonic in shared
// memory; longer rows are listed for k_sort_rows_block
__global__ void __launch_bounds__(256) k_sort_rows_warp(int n, const int32_t *ptr, int32_t *colv, int *long_rows) {
    __shared__ int buf[8][kRowSortWarpCap];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *a = buf[wib];
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw) {
        const int b = ptr[r], len = ptr[r + 1] - b;
        if (len > kRowSortWarpCap) {
            if (lane == 0) long_rows[1 + atomicAdd(&long_rows[0], 1)] = (int)r;
            continue;
        }
        if (len <= 1) continue;
        int m = 1;
        while (m < len) m <<= 1;
        for (int i = lane; i < m; i += 32) a[i] = i < len ? colv[b + i] : INT_MAX;
        __syncwarp();
        for (int k = 2; k <= m; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < m; i += 32) {
                    int p = i ^ j;
                    if (p > i) {
                        int x = a[i], y = a[p];
                        bool up = (i & k) == 0;
                        if ((x > y) == up) { a[i] = y; a[p] = x; }
                    }
                }
                __syncwarp();
            }
        for (int i = lane; i < len; i += 32) colv[b + i] = a[i];
        __syncwarp();
    }
}

// the listed rows longer than kRowSortWarpCap (at most the degeneracy): one block per row
__global__ void __launch_bounds__(1024) k_sort_rows_block(const int *long_rows, const int32_t *ptr, int32_t *colv) {
    __shared__ int a[kRowSortBlockCap];
    const int cnt = long_rows[0];
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        const int r = long_rows[1 + i];
        const int b = ptr[r], len = ptr[r + 1] - b;
        if (len > kRowSortBlockCap) continue;
        for (int i = threadIdx.x; i < len; i += blockDim.x) a[i] = colv[b + i];
        __syncthreads();
        block_bitonic(a, len);
        for (int i = threadIdx.x; i < len; i += blockDim.x) colv[b + i] = a[i];
        __syncthreads();
    }
}

__global__ void k_mix_gid(int n, const int32_t *order, uint64_t *mixid, int32_t *gid,
                          const int32_t *graph_ptr, int G) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int v = order[r];
        mixid[r] = mix64((uint64_t)(int64_t)v + 1ull);
        if (gid) {
            int lo = 0, hi = G;  // largest g with graph_ptr[g] <= v
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (graph_ptr[mid] <= v) lo = mid; else hi = mid;
            }
            gid[r] = lo;
        }
    }
}

// class statistics and per-class flags
__global__ void k_class_stats(int n, const int32_t *outdeg, const int32_t *indeg, int *cls_rows,
                              int *cls_x, int *cls_count) {
    __shared__ int srows[kNumClasses + 1], sx[kNumClasses + 1], scnt[kNumClasses + 1];
    if (threadIdx.x <= kNumClasses) {
        srows[threadIdx.x] = 0;
        sx[threadIdx.x] = 0;
        scnt[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int n0 = outdeg[r];
        const int c = n0 == 0 ? kNumClasses : class_of(n0);
        if (c < 0) continue;
        atomicMax(&srows[c], n0);
        atomicMax(&sx[c], indeg[r]);
        atomicAdd(&scnt[c], 1);
    }
    __syncthreads();
    if (threadIdx.x <= kNumClasses && scnt[threadIdx.x]) {
        atomicMax(&cls_rows[threadIdx.x], srows[threadIdx.x]);
        atomicMax(&cls_x[threadIdx.x], sx[threadIdx.x]);
        atomicAdd(&cls_count[threadIdx.x], scnt[threadIdx.x]);
    }
}

__global__ void k_class_flags(int n, const int32_t *outdeg, int c, int32_t *flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int n0 = outdeg[r];
        const int cr = n0 == 0 ? kNumClasses : class_of(n0);
        flags[r] = cr == c;
    }
}

// the flagged ranks in descending order (pos[n] = their number)
__global__ void k_scatter_flagged_desc(int n, const int32_t *flags, const int32_t *pos, int32_t *out) {
    const int32_t total = pos[n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        if (flags[r]) out[total - 1 - pos[r]] = (int32_t)r;
}

__global__ void k_mark_roots(const int32_t *ids, int64_t k, const int32_t *rank, int n, int32_t *mask,
                             int *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ids[i];
        if (v < 0 || v >= n) {
            atomicOr(status, ST_BADGRAPH);
            continue;
        }
        mask[rank[v]] = 1;
    }
}

__global__ void k_subset_flags(const int32_t *list, int cnt, const int32_t *mask, int32_t *flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = mask[list[i]] != 0;
}

__global__ void k_gather_flagged(const int32_t *list, int cnt, const int32_t *flags, const int32_t *pos,
                                 int32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i]) out[pos[i]] = list[i];
}

// -------------------------------------------------- priority order (buckets)

constexpr int kPrioBuckets = 256;

__device__ __forceinline__ int prio_bucket(float p) {
    // descending priority first; quarter-unit buckets (priorities are log2 work)
    if (!(p > 0.f)) p = 0.f;  // NaN and negatives land in the last bucket
    int b = (int)(p * 4.f);
    b = b > kPrioBuckets - 1 ? kPrioBuckets - 1 : b;
    return kPrioBuckets - 1 - b;
}

// Roots with a priority below 0 (or NaN) are unscored: they keep the list's
// own (plain) order behind all scored roots, placed by a prefix sum of the
// unscored flags, so neither their order nor one crowded bucket depends on
// atomics. unscored[0..cnt] gets the flags (unscored[cnt] = 0).
__global__ void k_prio_hist(const int32_t *list, int cnt, const int32_t *order, const float *prio, int *hist,
                            int32_t *unscored) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= cnt; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == cnt) {
            unscored[cnt] = 0;
            continue;
        }
        const float p = prio[order[list[i]]];
        const bool u = !(p >= 0.f);
        unscored[i] = u ? 1 : 0;
        if (!u) atomicAdd(&hist[prio_bucket(p)], 1);
    }
}

__global__ void k_prio_offsets(int *hist) {
    // exclusive scan of kPrioBuckets counts in place (one block of kPrioBuckets threads)
    __shared__ int sh[32];
    int tot;
    const int x = hist[threadIdx.x];
    const int pre = block_scan_excl<kPrioBuckets>(x, sh, &tot);
    hist[threadIdx.x] = pre;
}

// upos = exclusive prefix of the unscored flags (upos[cnt] = their number)
__global__ void k_prio_scatter(const int32_t *list, int cnt, const int32_t *order, const float *prio, int *cursor,
                               const int32_t *upos, int32_t *out) {
    const int scored = cnt - upos[cnt];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = list[i];
        const float p = prio[order[r]];
        if (p >= 0.f) out[atomicAdd(&cursor[prio_bucket(p)], 1)] = r;
        else out[scored + upos[i]] = r;
    }
}

// ------------------------------------------------------------ host side

static unsigned grid_for(int64_t work, int per_block, int cap = 1 << 20) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

cudaError_t launch_validate(int n, const int32_t *rp, const int32_t *col, int64_t m2, int *status,
                            cudaStream_t s, bool cols) {
    if (!cols) {
        k_check_rowptr<<<grid_for((int64_t)n + 1, 256), 256, 0, s>>>(n, rp, m2, status);
        count_launch();
    } else if (n > 0) {
        k_check_cols<<<grid_for((int64_t)n * 32, 256, 65536), 256, 0, s>>>(n, rp, col, status);
        count_launch();
    }
    return cudaGetLastError();
}

// The narrow stage runs as one cluster of kNarrowBlocks CTAs when this
// device can hold one (checked once per device: the non-portable cluster size
// must be allowed and the occupancy query must find room for a cluster).
static cudaLaunchConfig_t narrow_cluster_config(cudaStream_t s, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kNarrowBlocks);
    cfg.blockDim = dim3(kPeelThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kNarrowBlocks;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

static bool narrow_cluster_ok(cudaStream_t s) {
    static int ok[64];  // per device: 0 unknown, 1 yes, 2 no
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (ok[dev] == 0) {
        bool yes = cudaFuncSetAttribute(k_peel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
        if (yes) {
            cudaLaunchAttribute at[1];
            cudaLaunchConfig_t cfg = narrow_cluster_config(s, at);
            int clusters = 0;
            yes = cudaOccupancyMaxActiveClusters(&clusters, k_peel<true>, &cfg) == cudaSuccess && clusters >= 1;
        }
        (void)cudaGetLastError();  // a refusal above is an answer, not an error of the caller's
        ok[dev] = yes ? 1 : 2;
    }
    return ok[dev] == 1;
}

cudaError_t launch_peel(int n, const int32_t *rp, const int32_t *col, PeelBufs &b, int sm_count,
                        uint64_t timeout_ns, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel<false>, kPeelThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int blocks = sm_count;  // per_sm >= 1 checked above
    if (blocks > b.max_blocks) blocks = b.max_blocks;
    int32_t *segstart = b.SA;
    int handoff = (blocks > kNarrowBlocks && narrow_cluster_ok(s)) ? 1 : 0;
    void *args[] = {(void *)&n,        (void *)&rp,      (void *)&col,         (void *)&b.deg,
                    (void *)&b.rank,   (void *)&b.core,  (void *)&b.order,     (void *)&b.remA,
                    (void *)&b.remB,   (void *)&segstart, (void *)&b.bitmap,   (void *)&b.blocksums,
                    (void *)&b.ctl,    (void *)&b.status, (void *)&timeout_ns, (void *)&handoff};
    count_launch();
    e = cudaLaunchCooperativeKernel((void *)k_peel<false>, dim3(blocks), dim3(kPeelThreads), args, 0, s);
    if (e != cudaSuccess) return e;
    if (handoff) {
        // the narrow stage, if the full grid stopped there (the kernel returns
        // at once otherwise)
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = narrow_cluster_config(s, at);
        count_launch();
        e = cudaLaunchKernelEx(&cfg, k_peel<true>, n, rp, col, b.deg, b.rank, b.core, b.order, b.remA, b.remB,
                               segstart, b.bitmap, b.blocksums, b.ctl, b.status, timeout_ns, 0);
        if (e != cudaSuccess) return e;
    }
    k_peel_rank<<<2 * sm_count, kRankThreads, 0, s>>>(n, segstart, b.ctl, b.order, b.rank);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_peel_init(PeelCtl *ctl, int n) {
    ctl->k = 0;
    ctl->next = 0;
    ctl->rounds = 0;
    for (int i = 0; i < 3; i++) ctl->cnt[i] = 0;
    for (int i = 0; i < 3; i++) {
        ctl->nrem2[i] = 0;
        ctl->minval[i] = INT_MAX;
        ctl->sumdeg[i] = 0ull;
    }
    ctl->bar.count = 0;
    ctl->bar.gen = 0;
    ctl->t_start = ctl->t_narrow = ctl->t_solo = ctl->t_end = 0ull;
    ctl->r_narrow = ctl->r_solo = -1;
    ctl->rs_active = 0;
}

cudaError_t launch_peel_init(PeelCtl *ctl, int n, cudaStream_t s) {
    k_peel_init<<<1, 1, 0, s>>>(ctl, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_orient(int n, const int32_t *rp, const int32_t *col, const int32_t *order,
                          const int32_t *rank, int32_t *outdeg, int32_t *indeg, int32_t *out_ptr,
                          int32_t *out_col, int32_t *in_ptr, int32_t *in_col, int32_t *scan_tmp,
                          int *long_rows, cudaStream_t s) {
    if (n == 0) {
        cudaError_t e = exclusive_scan(outdeg, out_ptr, 0, scan_tmp, s);
        if (e != cudaSuccess) return e;
        return exclusive_scan(indeg, in_ptr, 0, scan_tmp, s);
    }
    const unsigned gw = grid_for((int64_t)n * 32, 256, 65536);
    k_count_split<<<gw, 256, 0, s>>>(n, rp, col, order, rank, outdeg, indeg);
    count_launch();
    cudaError_t e = exclusive_scan(outdeg, out_ptr, n, scan_tmp, s);
    if (e != cudaSuccess) return e;
    e = exclusive_scan(indeg, in_ptr, n, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_fill_split<<<gw, 256, 0, s>>>(n, rp, col, order, rank, out_ptr, out_col, in_ptr, in_col);
    count_launch();
    // long_rows[0] = count, then the rows longer than a warp sorts
    e = cudaMemsetAsync(long_rows, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_sort_rows_warp<<<gw, 256, 0, s>>>(n, out_ptr, out_col, long_rows);
    count_launch();
    k_sort_rows_block<<<152, 1024, 0, s>>>(long_rows, out_ptr, out_col);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_gather_outdeg(const int32_t *roots, int64_t k, const int32_t *outdeg, int32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = outdeg[roots[i]];
}

cudaError_t launch_gather_outdeg(const int32_t *roots, int64_t k, const int32_t *outdeg, int32_t *out,
                                 cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    k_gather_outdeg<<<grid_for(k, 256, 65536), 256, 0, s>>>(roots, k, outdeg, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mix_gid(int n, const int32_t *order, uint64_t *mixid, int32_t *gid,
                           const int32_t *graph_ptr, int G, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_mix_gid<<<grid_for(n, 256, 65536), 256, 0, s>>>(n, order, mixid, gid, graph_ptr, G);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_classify(int n, const int32_t *outdeg, const int32_t *indeg, int *cls_rows,
                            int *cls_x, int *cls_count, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_class_stats<<<grid_for(n, 256, 65536), 256, 0, s>>>(n, outdeg, indeg, cls_rows, cls_x, cls_count);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mark_roots(const int32_t *ids, int64_t k, const int32_t *rank, int n, int32_t *mask,
                              int *status, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    k_mark_roots<<<grid_for(k, 256, 65536), 256, 0, s>>>(ids, k, rank, n, mask, status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_subset(const int32_t *list, int cnt, const int32_t *mask, int32_t *flags, int32_t *pos,
                          int32_t *scan_tmp, int32_t *out, cudaStream_t s) {
    if (cnt <= 0) return cudaSuccess;
    k_subset_flags<<<grid_for(cnt, 256, 65536), 256, 0, s>>>(list, cnt, mask, flags);
    count_launch();
    cudaError_t e = exclusive_scan(flags, pos, cnt, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_gather_flagged<<<grid_for(cnt, 256, 65536), 256, 0, s>>>(list, cnt, flags, pos, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_priority_order(const int32_t *list, int cnt, const int32_t *order, const float *prio,
                                  int *hist, int32_t *flags, int32_t *pos, int32_t *scan_tmp, int32_t *out,
                                  cudaStream_t s) {
    if (cnt <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(hist, 0, kPrioBuckets * sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_prio_hist<<<grid_for(cnt + 1, 256, 65536), 256, 0, s>>>(list, cnt, order, prio, hist, flags);
    count_launch();
    if ((e = exclusive_scan(flags, pos, (int64_t)cnt + 1, scan_tmp, s)) != cudaSuccess) return e;
    k_prio_offsets<<<1, kPrioBuckets, 0, s>>>(hist);
    count_launch();
    k_prio_scatter<<<grid_for(cnt, 256, 65536), 256, 0, s>>>(list, cnt, order, prio, hist, pos, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_class_list(int n, const int32_t *outdeg, int c, int32_t *flags, int32_t *pos,
                              int32_t *scan_tmp, int32_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_class_flags<<<grid_for(n, 256, 65536), 256, 0, s>>>(n, outdeg, c, flags);
    count_launch();
    cudaError_t e = exclusive_scan(flags, pos, n, scan_tmp, s);
    if (e != cudaSuccess) return e;
    // Descending rank: later vertices of the degeneracy order sit in denser
    // cores and tend to carry the heavier subtrees, so they start first.
    k_scatter_flagged_desc<<<grid_for(n, 256, 65536), 256, 0, s>>>(n, flags, pos, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mce
