// Persistent depth-first Bron-Kerbosch traversal (Algorithm 2 with Tomita
// pivoting) of independent first-level subtrees (Algorithm 3), one subtree
// per cooperating group of GW warps, with the worker list of Sec. III-C.
//
// Per root vertex r (rank order = degeneracy order, Sec. II-C):
//   P0 = later neighbours of r (sorted ranks), local index i <-> P0[i];
//   A[i] = bitset over P0 of N(P0[i]) n P0     -- partial induced subgraph
//          (Sec. III-D, binary encoded, rows padded to WP words);
//   X_X  = earlier neighbours x of r that have a neighbour in P0, each held
//          as a bitset row N(x) n P0 in the group's global arena, and listed
//          in one index array shared by all levels, each level's set being
//          a prefix [0, lpX[level]) of it (compact X, Sec. III-E);
//   X_P  = excluded vertices that came from P0: one bitset per level.
// A node is (P, X_P, X_X prefix). Pivot: u in P u X_P maximising
// |P n N(u)| (Sec. III-E restricts the pivot to X_P u P for partial induced
// subgraphs; with IPX, Sec. IV-E, X_X rows are candidates too), ties to the
// smallest rank. Branches: P - N(u) in ascending rank. R is maximal when P,
// X_P and X_X are all empty.
//
// The pivot scan visits candidates in ascending index, 32*GW at a time, and
// stops after the first chunk whose best score equals the largest score any
// candidate can have (|P| if X_P is non-empty, else |P| - 1): the smallest
// index reaching it is then the argmax, so the pivot is the same as a full scan.
//
// Two walks share the kernel. The wide walk above keeps a node's sets one word
// per thread over P0. Once a node has |P| + |X_P| <= 32 (and at roots with
// |P0| <= 32) its whole subtree runs in compact mode: one-word sets over that
// node's P u X_P, with one- and two-vertex children resolved in closed form.
// Both walk Algorithm 2's tree node for node, so tree-node counts, cliques and
// hashes do not depend on where the switch happens. Idle groups take subtrees
// of either kind from busy ones (the worker list, Sec. III-C).
//
// Template parameters: WP padded words per row, GW warps per group, AG true
// when A lives in the global arena, LIST true when cliques are listed, L2
// true when tasks are edges.
#pragma once
#include "mce_internal.cuh"

namespace mce {

// Level record in the DFS stack (words).
template <int WP>
struct Lvl {
    static constexpr int P = 0, XP = WP, B = 2 * WP, LPX = 3 * WP, NPEND = 3 * WP + 1,
                         VSEL = 3 * WP + 2, SLO = 3 * WP + 4, SHI = 3 * WP + 5, SIZE = 3 * WP + 6;
};

template <int GW>
struct Grp {
    int gl;    // thread index in group
    int warp;  // warp index in group
    int lane;
    int gib;   // group index in block
    __device__ __forceinline__ void sync() const {
        if (GW == 1) {
            __syncwarp();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(gib + 1), "n"(32 * GW) : "memory");
        }
    }
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// rounded to 4 words so whatever follows the stack stays 16-byte aligned
__host__ __device__ inline size_t stack_words(int wp, int rows) {
    return ((size_t)(rows + 2) * (3 * wp + 6) + 3) / 4 * 4;
}

// Shared-memory layout: one block region, then one region per group
// (offsets in bytes; group offsets relative to the group's base).
struct GrpSmem {
    size_t block_hist, group0;                               // block region
    size_t a, cur, p0, cand, red, misc, stack, hist, total;  // per group
};

// rows = max |P0| handled; block_hist: one clique-size histogram per block
// (single graph) instead of one per group (batched graphs)
__host__ __device__ inline GrpSmem grp_smem_layout(int wp, int gw, int rows, bool a_global, bool stack_smem,
                                                   bool block_hist) {
    GrpSmem L;
    size_t off = 0;
    L.block_hist = 0;
    if (block_hist) off += (size_t)(rows + 2) * 8;
    L.group0 = align_up(off, 16);
    off = 0;
    L.a = off;
    if (!a_global) off += (size_t)rows * wp * 4;
    off = align_up(off, 16);
    L.cur = off;
    off += (size_t)wp * 2 * 4;  // P, then P u X_P, of the node being entered
    off = align_up(off, 16);
    L.p0 = off;
    off += (size_t)rows * 4;
    L.cand = off;
    off += (size_t)rows * 4;
    off = align_up(off, 16);  // holds 64-bit reduction words
    L.red = off;
    off += (size_t)gw * 4 * 4;
    L.misc = off;
    off += 16 * 4;
    off = align_up(off, 16);
    L.stack = off;
    if (stack_smem) off += stack_words(wp, rows) * 4;
    off = align_up(off, 16);
    L.hist = off;
    if (!block_hist) off += (size_t)(rows + 2) * 8;
    L.total = align_up(off, 16);
    return L;
}

__host__ __device__ inline size_t smem_bytes(const GrpSmem &L, int groups_per_block) {
    return L.group0 + (size_t)groups_per_block * L.total;
}

// Arena words per group: [stack if global][A rows][X rows][xidx][xscr][xrank]
// [xcomp][R ids: the current clique's input ids, when cliques are listed].
// The A region holds A itself when it lives in global memory, else it is the
// landing area where a donor writes A for this group when it is a receiver.
__host__ __device__ inline size_t arena_words(int wp, int rows, int xcap, bool a_global, bool stack_smem) {
    size_t w = 0;
    if (!stack_smem) w += stack_words(wp, rows);
    w += (size_t)rows * wp;
    w += (size_t)xcap * wp + 4 * (size_t)xcap;
    w += (size_t)rows + 2;
    (void)a_global;
    return align_up(w, 4);
}

struct ArenaPtrs {
    uint32_t *stk, *A, *xrows, *xidx, *xscr;
    uint32_t *xrank;  // xrank[slot]: degeneracy rank of that X_X row's vertex
    uint32_t *xcomp;  // xcomp[slot]: that row over a compact subtree's index space
    uint32_t *rid;    // rid[i]: input id of the i-th vertex of the current R (listing)
};

__device__ __forceinline__ ArenaPtrs arena_at(uint32_t *base, int wp, int rows, int xcap, bool stack_smem) {
    ArenaPtrs a;
    uint32_t *q = base;
    a.stk = q;
    if (!stack_smem) q += stack_words(wp, rows);
    a.A = q;
    q += (size_t)rows * wp;
    a.xrows = q;
    a.xidx = q + (size_t)xcap * wp;
    a.xscr = a.xidx + xcap;
    a.xrank = a.xscr + xcap;
    a.xcomp = a.xrank + xcap;
    a.rid = a.xcomp + xcap;
    return a;
}

// Edge tasks (Algorithm 4) claimed per atomic.
constexpr int kEdgeChunk = 16;

// Warps per traversal block, at most and by default. The traversal is bound
// by dependent latency (shuffle and reduction chains, L1/L2 round trips), so
// resident warps are what hides it: 24 warps at 80 registers a thread beat 16
// at 128 (chunglu_1m 54.5 -> 46.6 ms) despite a few spilled registers.
constexpr int kTravMaxWarps = 24;

__device__ __forceinline__ int find_in(const int32_t *a, int lo, int hi, int32_t key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;  // first index with a[idx] >= key
}

template <int GW>
__device__ __forceinline__ int grp_sum(const Grp<GW> &g, int *red, int x) {
    int s = __reduce_add_sync(0xffffffffu, x);
    if (GW == 1) return s;
    if (g.lane == 0) red[g.warp] = s;
    g.sync();
    int t = 0;
#pragma unroll
    for (int i = 0; i < GW; i++) t += red[i];
    g.sync();
    return t;
}

template <int GW>
__device__ __forceinline__ unsigned grp_max(const Grp<GW> &g, int *red, unsigned x) {
    unsigned s = __reduce_max_sync(0xffffffffu, x);
    if (GW == 1) return s;
    if (g.lane == 0) red[g.warp] = (int)s;
    g.sync();
    unsigned t = 0;
#pragma unroll
    for (int i = 0; i < GW; i++) t = max(t, (unsigned)red[i]);
    g.sync();
    return t;
}

template <int GW>
__device__ __forceinline__ int grp_or(const Grp<GW> &g, int *red, int x) {
    int s = __any_sync(0xffffffffu, x) ? 1 : 0;
    if (GW == 1) return s;
    if (g.lane == 0) red[g.warp] = s;
    g.sync();
    int t = 0;
#pragma unroll
    for (int i = 0; i < GW; i++) t |= red[i];
    g.sync();
    return t;
}

template <int GW>
__device__ __forceinline__ unsigned long long grp_max64(const Grp<GW> &g, unsigned long long *red64,
                                                         unsigned long long x) {
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    if (GW == 1) return x;
    if (g.lane == 0) red64[g.warp] = x;
    g.sync();
    unsigned long long t = 0;
#pragma unroll
    for (int i = 0; i < GW; i++) t = red64[i] > t ? red64[i] : t;
    g.sync();
    return t;
}

// exclusive prefix of pred over the group; *total receives the count
template <int GW>
__device__ __forceinline__ int grp_prefix(const Grp<GW> &g, int *red, bool pred, int *total) {
    unsigned b = __ballot_sync(0xffffffffu, pred);
    int in_warp = __popc(b & ((1u << g.lane) - 1u));
    if (GW == 1) {
        *total = __popc(b);
        return in_warp;
    }
    if (g.lane == 0) red[g.warp] = __popc(b);
    g.sync();
    int off = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < GW; i++) {
        int c = red[i];
        if (i < g.warp) off += c;
        tot += c;
    }
    g.sync();
    *total = tot;
    return off + in_warp;
}

// Writes the set bits of a bitset held one word per thread (thread gl owns
// word gl < WP) to list[] as indices in ascending order and returns their
// number. Each owner writes its word's bits at its exclusive prefix of the
// popcounts; the list is complete for the whole group on return.
template <int WP, int GW>
__device__ __forceinline__ int grp_bits_to_list(const Grp<GW> &g, int *red, uint32_t word, int32_t *list) {
    const int c = __popc(word);
    int inc = c;
    constexpr int span = GW == 1 ? WP : 32;
#pragma unroll
    for (int o = 1; o < span; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (g.lane >= o) inc += y;
    }
    int pre, tot;
    if (GW == 1) {
        tot = __shfl_sync(0xffffffffu, inc, WP - 1);
        pre = inc - c;
    } else {
        if (g.lane == 31) red[g.warp] = inc;
        g.sync();
        int off = 0;
        tot = 0;
#pragma unroll
        for (int i = 0; i < GW; i++) {
            const int t = red[i];
            if (i < g.warp) off += t;
            tot += t;
        }
        g.sync();
        pre = off + inc - c;
    }
    uint32_t bits = word;
    while (bits) {
        list[pre++] = g.gl * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
    }
    g.sync();
    return tot;
}

// Position of the t-th (from 0) set bit of m; t < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int t) {
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const int c = __popc(m & ((1u << sh) - 1u));
        if (c <= t) {
            t -= c;
            m >>= sh;
            pos += sh;
        }
    }
    return pos;
}

// Copies the rows listed in rows[0..nrows) of a WP-word bit matrix.
template <int WP, int GW>
__device__ __forceinline__ void grp_copy_rows(const Grp<GW> &g, const int32_t *rows, int nrows, const uint32_t *src,
                                              uint32_t *dst) {
    constexpr int GT = 32 * GW;
    if constexpr (WP % 4 == 0) {
        constexpr int Q = WP / 4;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (int i = g.gl; i < nrows * Q; i += GT) {
            const int j = i / Q, q = i - j * Q;
            const size_t at = (size_t)rows[j] * Q + q;
            d4[at] = s4[at];
        }
    } else {
        for (int i = g.gl; i < nrows * WP; i += GT) {
            const int j = i / WP, w = i - j * WP;
            const size_t at = (size_t)rows[j] * WP + w;
            dst[at] = src[at];
        }
    }
}

// Optional per-phase cycle counters (runtime switch; thread 0 of each group).
struct PhaseClock {
    bool on;
    long long t0;
    unsigned long long cyc[kNumPhases], cnt[kNumPhases];
    __device__ __forceinline__ void start() {
        if (on) t0 = clock64();
    }
    __device__ __forceinline__ void stop(int k) {
        if (on) {
            long long t = clock64();
            cyc[k] += (unsigned long long)(t - t0);
            t0 = t;
        }
    }
    __device__ __forceinline__ void count(int k, unsigned long long c) {
        if (on) cnt[k] += c;
    }
};

// LIST: the variant that also writes each clique's members (mce_run_list);
// L2: the variant whose tasks are edges (Algorithm 4); ST: the counting
// variant that also keeps per-phase cycle counters (opts.stats). The plain
// counting variant carries none of that code. PV: the pivot rule, fixed at
// compile time in the counting variants (0 = IP, 1 = IPX), so each carries
// the code of one rule only; 2 = read from the launch (C.pivot_ipx).
template <int WP, int GW, bool AG, bool LIST, bool L2, bool ST = false, int PV = 2>
__global__ void __launch_bounds__(32 * kTravMaxWarps) k_traverse(DevGraph G, DevOut O, ClassArgs C, int rows_cap, int stack_smem) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int GT = 32 * GW;
    constexpr int LS = Lvl<WP>::SIZE;
    const int warps_pb = blockDim.x >> 5;
    const int gpb = warps_pb / GW;
    const int wib = threadIdx.x >> 5;
    Grp<GW> g;
    g.gib = wib / GW;
    g.warp = wib % GW;
    g.lane = threadIdx.x & 31;
    g.gl = g.warp * 32 + g.lane;
    // one clique-size histogram per block (single graph, multi-warp groups) or
    // per group: one-warp groups record cliques too often to share one through
    // shared-memory atomics, and batched runs flush per graph
    const bool block_hist = G.gid == nullptr && GW > 1;
    const GrpSmem L = grp_smem_layout(WP, GW, rows_cap, AG, stack_smem != 0, block_hist);
    unsigned long long *bhist = (unsigned long long *)(smem_raw + L.block_hist);
    if (block_hist) {
        for (int i = threadIdx.x; i < rows_cap + 2; i += blockDim.x) bhist[i] = 0ull;
        __syncthreads();
    }
    const bool in_group = g.gib < gpb;
    const int gg = blockIdx.x * gpb + g.gib;  // global group id
    const int ngroups = gridDim.x * gpb;

    unsigned char *base = smem_raw + L.group0 + (size_t)g.gib * L.total;
    unsigned long long *hist = block_hist ? bhist : (unsigned long long *)(base + L.hist);
    int32_t *p0 = (int32_t *)(base + L.p0);
    int32_t *cand = (int32_t *)(base + L.cand);
    uint32_t *cur = (uint32_t *)(base + L.cur);
    int *red = (int *)(base + L.red);
    int *misc = (int *)(base + L.misc);

    const ArenaPtrs ar = arena_at(C.arena + (size_t)(in_group ? gg : 0) * C.arena_words_per_group, WP,
                                  rows_cap, C.x_cap, stack_smem != 0);
    uint32_t *stk = stack_smem ? (uint32_t *)(base + L.stack) : ar.stk;
    uint32_t *Arow = AG ? ar.A : (uint32_t *)(base + L.a);
    uint32_t *xrows = ar.xrows;
    uint32_t *xidx = ar.xidx;
    uint32_t *xscr = ar.xscr;
    uint32_t *xrank = ar.xrank;
    uint32_t *xcomp = ar.xcomp;
    uint32_t *rid = ar.rid;
    constexpr bool listing = LIST;

    // Only waits are timed (idle_wait); busy groups post a heartbeat for them
    // at most every timeout/8. Work itself is bounded only by the optional run
    // budget, checked with the heartbeat every 1024 loop iterations.
    unsigned long long *const beat = reinterpret_cast<unsigned long long *>(C.ctl + CTL_BEAT);
    const uint64_t beat_every = C.timeout_ns / 8 > 100000ull ? C.timeout_ns / 8 : 100000ull;
    const uint64_t budget_end = C.budget_ns ? *O.t0 + C.budget_ns : ~0ull;
    uint64_t last_beat = 0;
    // thread 0 of a group: post the heartbeat when due; true past the budget
    auto tick = [&]() -> bool {
        const uint64_t now = globaltimer_ns();
        if (now - last_beat > beat_every) {
            st_relaxed_u64(beat, now);
            last_beat = now;
        }
        return now > budget_end;
    };
    PhaseClock pc{};
    pc.on = ST && g.gl == 0;
    // IPX: X_X rows are pivot candidates too (Sec. IV-E)
    const bool ipx_rule = PV == 2 ? C.pivot_ipx != 0 : PV == 1;

    // per-group accumulators (meaningful in thread 0 of the group)
    unsigned long long acc_cnt = 0, acc_hash = 0, acc_nodes = 0, acc_don = 0;
    int acc_gid = -1, acc_maxsz = 0;
    unsigned iters = 0;

    auto flush = [&](void) {
        // add the group's count and hash (and, batched, histogram) to graph acc_gid
        if (acc_gid >= 0) {
            if (g.gl == 0) {
                if (acc_cnt) atomicAdd(&O.count[acc_gid], acc_cnt);
                if (acc_hash) atomicAdd(&O.hash[acc_gid], acc_hash);
            }
            if (!block_hist) {
                for (int s = g.gl; s < rows_cap + 2; s += GT) {
                    unsigned long long c = hist[s];
                    if (c) {
                        if (s < O.hist_len) atomicAdd(&O.hist[(size_t)acc_gid * O.hist_len + s], c);
                        hist[s] = 0;
                    }
                }
            }
        }
        acc_cnt = 0;
        acc_hash = 0;
        g.sync();
    };

    if (in_group) {
        if (!block_hist)
            for (int i = g.gl; i < rows_cap + 2; i += GT) hist[i] = 0;
        g.sync();
        int cached_r = -1, cached_nx = 0;  // level 2: the root whose P0, A and X rows are loaded
        int ch_i = 0, ch_j = 0, ch_left = 0;  // level 2, thread 0: the claimed run of edges
        for (;;) {
            // --------------------------------------------------- get a task
            if (g.gl == 0) {
                int r = -1, mail = 0, ej = -1;
                bool have = false;
                if (L2) {
                    // edges are claimed kEdgeChunk at a time, consecutive edges of a
                    // root staying with one group so that its A is built once
                    if (ch_left == 0) {
                        const int idx = atomicAdd(&C.ctl[CTL_NEXT_ROOT], kEdgeChunk);
                        if (idx < C.n_tasks) {
                            // root i is the last with eoff[i] <= idx
                            int lo = 0, hi = C.n_roots - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (C.eoff[mid] <= idx) lo = mid;
                                else hi = mid - 1;
                            }
                            ch_i = lo;
                            ch_j = idx - C.eoff[lo];
                            ch_left = (int)min((int64_t)kEdgeChunk, C.n_tasks - idx);
                        }
                    }
                    if (ch_left > 0) {
                        r = C.roots[ch_i];
                        ej = ch_j;
                        have = true;
                        ch_left--;
                        if (++ch_j == C.eoff[ch_i + 1] - C.eoff[ch_i]) {
                            ch_i++;
                            ch_j = 0;
                        }
                    }
                } else {
                    const int idx = atomicAdd(&C.ctl[CTL_NEXT_ROOT], 1);
                    if (idx < C.n_tasks) {
                        r = C.roots[idx];
                        have = true;
                    }
                }
                if (!have && C.worker_list) {
                    // join the worker list and wait for a donated subtree (Sec. III-C)
                    pc.start();
                    atomicOr(&C.idle_bits[gg >> 5], 1u << (gg & 31));
                    atomicAdd(&C.ctl[CTL_IDLE], 1);
                    __threadfence();
                    atomicSub(&C.ctl[CTL_ACTIVE], 1);
                    int *const flag = &C.mail_flag[(size_t)gg * kMailFlagStride];
                    if (idle_wait(flag, &C.ctl[CTL_ACTIVE], O.status, beat, C.timeout_ns, budget_end) > 0) {
                        mail = 1;
                        r = (int)C.mail[(size_t)gg * C.mail_words + 0];
                    }
                    pc.stop(PH_IDLE);
                    pc.count(PH_IDLE, mail);
                }
                misc[0] = r;
                misc[1] = mail;
                misc[5] = ej;
            }
            g.sync();
            const int r = misc[0];
            const bool have_mail = misc[1] != 0;
            const int ej = misc[5];  // level 2: the edge's later end, as a local index of P0
            g.sync();
            if (r < 0) break;

            const int gid = G.gid ? G.gid[r] : 0;
            if (gid != acc_gid) {
                flush();
                acc_gid = gid;
            }
            const int n0 = G.out_ptr[r + 1] - G.out_ptr[r];
            const int W = (n0 + 31) >> 5;
            const int x0 = G.in_ptr[r + 1] - G.in_ptr[r];
            const int32_t *prow = G.out_col + G.out_ptr[r];
            const int32_t *xrow = G.in_col + G.in_ptr[r];
            if (n0 > rows_cap || x0 > C.x_cap || W > WP) {
                if (g.gl == 0) atomicOr(O.status, ST_OVERFLOW);
                break;
            }
            unsigned long long t_nodes = 0, t_cnt = 0, t_hash = 0;
            pc.start();
            pc.count(PH_SETUP, 1);

            // layout of a donated subtree's mail: [0] root, [1] level (|R| - 1),
            // [2] number of X_X rows the donor wrote into this group's arena,
            // [3] kind. Kind 0 (wide): [4..4+WP) R' (path below the root), then
            // P', then X_P'. Kind 1 (compact, one-warp groups): [4..36) the rows
            // over the index space, [36..68) its local indices, [68] P, [69] X_P,
            // [70..72) the hash sum of R; its X_X rows are in the arena's xcomp
            // (by position), their ranks in xscr.
            const uint32_t *mb = C.mail + (size_t)gg * C.mail_words;
            const bool edge = L2 && !have_mail;  // a task of one edge {r, P0[ej]}
            const int l0 = have_mail ? (int)mb[1] : (edge ? 1 : 0);
            const bool cmail = GW == 1 && have_mail && mb[3] != 0u;
            // consecutive edge tasks of one root reuse its P0, A and X rows (an
            // edge task changes none of them; a received subtree does)
            const bool reuse = edge && r == cached_r;
            if (!reuse)
                for (int i = g.gl; i < n0; i += GT) p0[i] = prow[i];
            int nx = 0;
            // A root with |P0| <= 32 in a one-warp group (not an edge task, not
            // received): its whole subtree runs in compact mode over L = P0, so
            // its rows are built straight into registers: A in shared memory
            // (cand[0, n0)), the X_X rows as one word each, packed by position
            // into lane registers (rows 32 and on, and their ranks, in the arena's
            // xcomp and xscr). No A or X_X rows go to the global arena.
            const bool fast = GW == 1 && !have_mail && !L2 && n0 <= 32;
            uint32_t f_row = 0u, f_xr = 0u, f_xk = 0u;
            if (fast) {
                constexpr unsigned FULL = 0xffffffffu;
                uint32_t *frow = reinterpret_cast<uint32_t *>(cand);
                if (g.lane < n0) frow[g.lane] = 0u;
                __syncwarp();
                int rb = 0, re = 0;
                if (g.lane < n0) {
                    const int32_t u = p0[g.lane];
                    rb = G.out_ptr[u];
                    re = G.out_ptr[u + 1];
                }
                const int npairs = n0 * (n0 - 1) / 2;
                for (int q0 = 0; q0 < npairs; q0 += 32) {
                    const int q = q0 + g.lane;
                    // row i of pair q: the largest i with i (2 n0 - i - 1) / 2 <= q
                    int i = 0;
                    if (q < npairs) {
                        int lo = 0, hi = n0 - 2;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (mid * (2 * n0 - mid - 1) / 2 <= q) lo = mid;
                            else hi = mid - 1;
                        }
                        i = lo;
                    }
                    const int lo0 = __shfl_sync(FULL, rb, i), hi0 = __shfl_sync(FULL, re, i);
                    if (q < npairs) {
                        const int k = i + 1 + (q - i * (2 * n0 - i - 1) / 2);
                        const int32_t w = p0[k];
                        int lo = lo0, hi = hi0;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (G.out_col[mid] < w) lo = mid + 1;
                            else hi = mid;
                        }
                        if (lo < hi0 && G.out_col[lo] == w) {
                            atomicOr(&frow[i], 1u << k);
                            atomicOr(&frow[k], 1u << i);
                        }
                    }
                }
                __syncwarp();
                f_row = g.lane < n0 ? frow[g.lane] : 0u;
                for (int it = 0; it < x0; it += 32) {
                    const int idx = it + g.lane;
                    uint32_t w = 0u;
                    int32_t x = 0;
                    if (idx < x0) {
                        x = xrow[idx];
                        const int32_t *nr = G.out_col + G.out_ptr[x];
                        const int len = G.out_ptr[x + 1] - G.out_ptr[x];
                        int lo = 0;
                        for (int j = find_in(nr, 0, len, r + 1); j < len && lo < n0; j++) {
                            const int k = find_in(p0, lo, n0, nr[j]);
                            if (k < n0 && p0[k] == nr[j]) {
                                w |= 1u << k;
                                lo = k + 1;
                            } else {
                                lo = k;
                            }
                        }
                    }
                    const unsigned hm = __ballot_sync(FULL, w != 0u);
                    const int tot = __popc(hm);
                    // lane j takes the (j - nx)-th row found in this chunk
                    const int t = g.lane - nx;
                    const int src = (t >= 0 && t < tot) ? nth_set_bit(hm, t) : 0;
                    const uint32_t wv = __shfl_sync(FULL, w, src);
                    const uint32_t xv = (uint32_t)__shfl_sync(FULL, x, src);
                    if (t >= 0 && t < tot) {
                        f_xr = wv;
                        f_xk = xv;
                    }
                    if (w != 0u) {
                        const int k = nx + __popc(hm & ((1u << g.lane) - 1u));
                        if (k >= 32) {
                            xcomp[k] = w;
                            xscr[k] = (uint32_t)x;
                        }
                    }
                    nx += tot;
                }
                __syncwarp();
            } else if (reuse) {
                nx = cached_nx;
            } else if (have_mail) {
                // the donor wrote the A rows of P' u X_P' into the arena's A region
                // and the surviving X_X rows into the arena's X rows: nothing to
                // rebuild. Every row the subtree reads (candidates, branches) is
                // one of those; the other rows are never read.
                if (!AG && !cmail) {
                    const uint32_t want = g.gl < WP ? (mb[4 + WP + g.gl] | mb[4 + 2 * WP + g.gl]) : 0u;
                    const int nrows = grp_bits_to_list<WP, GW>(g, red, want, cand);
                    grp_copy_rows<WP, GW>(g, cand, nrows, ar.A, Arow);
                }
                nx = (int)mb[2];
                g.sync();
            } else {
                // ----------------------------------- induced subgraph (Sec. III-D)
                for (int i = g.gl; i < n0 * WP; i += GT) Arow[i] = 0u;
                g.sync();
                if (GW == 1 && n0 <= 32) {
                    // Few rows whose out-lists are long (a small root's later
                    // neighbours sit deeper in the order): test each pair i < k
                    // by a binary search for P0[k] in the out-list of P0[i], all
                    // pairs of the root spread over the lanes.
                    int rb = 0, re = 0;
                    if (g.lane < n0) {
                        const int32_t u = p0[g.lane];
                        rb = G.out_ptr[u];
                        re = G.out_ptr[u + 1];
                    }
                    const int npairs = n0 * (n0 - 1) / 2;
                    for (int q0 = 0; q0 < npairs; q0 += 32) {
                        const int q = q0 + g.lane;
                        // row i of pair q: the largest i with i (2 n0 - i - 1) / 2 <= q
                        int i = 0;
                        if (q < npairs) {
                            int lo = 0, hi = n0 - 2;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (mid * (2 * n0 - mid - 1) / 2 <= q) lo = mid;
                                else hi = mid - 1;
                            }
                            i = lo;
                        }
                        const int lo0 = __shfl_sync(0xffffffffu, rb, i), hi0 = __shfl_sync(0xffffffffu, re, i);
                        if (q < npairs) {
                            const int k = i + 1 + (q - i * (2 * n0 - i - 1) / 2);
                            const int32_t w = p0[k];
                            int lo = lo0, hi = hi0;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (G.out_col[mid] < w) lo = mid + 1;
                                else hi = mid;
                            }
                            if (lo < hi0 && G.out_col[lo] == w) {
                                atomicOr(&Arow[(size_t)i * WP + (k >> 5)], 1u << (k & 31));
                                atomicOr(&Arow[(size_t)k * WP + (i >> 5)], 1u << (i & 31));
                            }
                        }
                    }
                } else if (GW == 1) {
                    // 32 rows at a time: the part of each later neighbour's
                    // out-list up to the last rank of P0 (all of it lies after that
                    // neighbour), walked by the whole warp
                    const int32_t maxp = p0[n0 - 1];
                    for (int i0 = 0; i0 < n0; i0 += 32) {
                        const int i = i0 + g.lane;
                        int jb = 0, cnt = 0;
                        if (i < n0) {
                            const int32_t u = p0[i];
                            jb = G.out_ptr[u];
                            const int len = G.out_ptr[u + 1] - jb;
                            cnt = (len == 0 || G.out_col[jb + len - 1] <= maxp) ? len
                                                                                 : find_in(G.out_col + jb, 0, len, maxp + 1);
                        }
                        warp_walk_lists<4>(G.out_col, jb, cnt, g.lane, p0, n0, [&](int l, int k) {
                            const int ii = i0 + l;
                            atomicOr(&Arow[(size_t)ii * WP + (k >> 5)], 1u << (k & 31));
                            atomicOr(&Arow[(size_t)k * WP + (ii >> 5)], 1u << (ii & 31));
                        });
                    }
                } else {
                    for (int i = g.warp; i < n0; i += GW) {
                        const int32_t u = p0[i];
                        const int32_t *nr = G.out_col + G.out_ptr[u];
                        const int len = G.out_ptr[u + 1] - G.out_ptr[u];
                        for (int j = g.lane; j < len; j += 32) {
                            int32_t w = nr[j];
                            int k = find_in(p0, i + 1, n0, w);
                            if (k < n0 && p0[k] == w) {
                                atomicOr(&Arow[(size_t)i * WP + (k >> 5)], 1u << (k & 31));
                                atomicOr(&Arow[(size_t)k * WP + (i >> 5)], 1u << (i & 31));
                            }
                        }
                    }
                }
                if (AG) __threadfence_block();
                g.sync();

                // ----------------------------------- X_X rows (Sec. III-E)
                if (GW == 1) {
                    // The row of X0[i] goes to slot i. Clear the words a row can
                    // use, walk the later lists of X0 between r and the last rank
                    // of P0 with the whole warp, then list the slots whose row
                    // holds a bit.
                    constexpr unsigned FULL = 0xffffffffu;
                    const int32_t maxp = n0 > 0 ? p0[n0 - 1] : -1;
                    for (int i = g.lane; i < x0; i += 32) {
                        xrank[i] = (uint32_t)xrow[i];
                        for (int w = 0; w < W; w++) xrows[(size_t)i * WP + w] = 0u;
                    }
                    __syncwarp();
                    for (int i0 = 0; i0 < x0; i0 += 32) {
                        const int i = i0 + g.lane;
                        int jb = 0, cnt = 0;
                        if (i < x0) {
                            const int32_t x = xrow[i];
                            const int b0 = G.out_ptr[x], len = G.out_ptr[x + 1] - b0;
                            const int32_t *nr = G.out_col + b0;
                            const int j0 = find_in(nr, 0, len, r + 1);  // only later vertices can be in P0
                            const int j1 = (j0 == len || nr[len - 1] <= maxp) ? len : find_in(nr, j0, len, maxp + 1);
                            jb = b0 + j0;
                            cnt = j1 - j0;
                        }
                        warp_walk_lists<4>(G.out_col, jb, cnt, g.lane, p0, n0, [&](int l, int k) {
                            atomicOr(&xrows[(size_t)(i0 + l) * WP + (k >> 5)], 1u << (k & 31));
                        });
                    }
                    __threadfence_block();
                    __syncwarp();
                    int nl = 0;
                    for (int i0 = 0; i0 < x0; i0 += 32) {
                        const int i = i0 + g.lane;
                        bool ne = false;
                        if (i < x0)
                            for (int w = 0; w < W; w++) ne |= __ldcg(&xrows[(size_t)i * WP + w]) != 0u;
                        const unsigned bm = __ballot_sync(FULL, ne);
                        if (ne) xidx[nl + __popc(bm & ((1u << g.lane) - 1u))] = (uint32_t)i;
                        nl += __popc(bm);
                    }
                    nx = nl;
                } else {
                    int base_slot = 0;
                    for (int it = 0; it < x0; it += GT) {
                        int idx = it + g.gl;
                        int hits = 0;
                        const int32_t *nr = nullptr;
                        int len = 0, j0 = 0;
                        int32_t x = 0;
                        if (idx < x0) {
                            x = xrow[idx];
                            nr = G.out_col + G.out_ptr[x];
                            len = G.out_ptr[x + 1] - G.out_ptr[x];
                            j0 = find_in(nr, 0, len, r + 1);  // only later vertices can be in P0
                            int lo = 0;
                            for (int j = j0; j < len && lo < n0; j++) {
                                int32_t w = nr[j];
                                int k = find_in(p0, lo, n0, w);
                                if (k < n0 && p0[k] == w) { hits++; lo = k + 1; }
                                else lo = k;
                            }
                        }
                        int tot;
                        int pos = grp_prefix(g, red, hits > 0, &tot);
                        if (hits > 0) {
                            int slot = base_slot + pos;
                            uint32_t *row = xrows + (size_t)slot * WP;
                            int cw = 0;
                            uint32_t accw = 0;
                            int lo = 0;
                            for (int j = j0; j < len && lo < n0; j++) {
                                int32_t w = nr[j];
                                int k = find_in(p0, lo, n0, w);
                                if (k < n0 && p0[k] == w) {
                                    int wi = k >> 5;
                                    while (cw < wi) { row[cw++] = accw; accw = 0; }
                                    accw |= 1u << (k & 31);
                                    lo = k + 1;
                                } else {
                                    lo = k;
                                }
                            }
                            while (cw < WP) { row[cw++] = accw; accw = 0; }
                            xidx[slot] = (uint32_t)slot;
                            xrank[slot] = (uint32_t)x;
                        }
                        base_slot += tot;
                    }
                    nx = base_slot;
                }
            }
            if (edge) {
                cached_r = r;
                cached_nx = nx;
            } else {
                cached_r = -1;
            }
            __threadfence_block();
            g.sync();

            // -------------------------------------------- initial node
            // The current node's P, X_P and branch set live in registers, one
            // 32-bit word per thread (thread gl owns word gl < WP); the stack
            // holds the ancestors (pushed on descent, reloaded on backtrack).
            const bool own = g.gl < WP;
            // the words of the root's rows that can hold bits (W <= WP): the
            // stack keeps only these; the node's other words stay 0
            const bool ownw = g.gl < W;
            uint32_t p = 0u, xp = 0u, b = 0u;
            int lpx = nx, npend = 0;
            uint64_t S = G.mixid[r];
            if (!have_mail) {
                if (own) {
                    const int lo = g.gl * 32;
                    if (lo < n0) p = (n0 - lo >= 32) ? 0xffffffffu : ((1u << (n0 - lo)) - 1u);
                }
                if (listing && g.gl == 0) rid[0] = (uint32_t)G.order[r];
            } else if (!cmail) {
                // P', X_P' and the path R' below the root come from the mail; the
                // X_X rows in the arena are exactly the donor's survivors
                const uint32_t *mR = mb + 4, *mP = mb + 4 + WP, *mX = mb + 4 + 2 * WP;
                if (own) {
                    p = mP[g.gl];
                    xp = mX[g.gl];
                }
                int lv = 0;
                for (int w = 0; w < W; w++) {
                    uint32_t bits = mR[w];
                    while (bits) {
                        const int bb = __ffs(bits) - 1;
                        bits &= bits - 1;
                        S += G.mixid[p0[w * 32 + bb]];
                        // the path, so that deeper donations can rebuild R
                        if (g.gl == 0) stk[(size_t)lv * LS + Lvl<WP>::VSEL] = (uint32_t)(w * 32 + bb);
                        lv++;
                    }
                }
            }
            __threadfence_block();
            g.sync();
            pc.stop(PH_SETUP);

            // ------------------------------------------------- DFS (Algorithm 2)
            uint32_t *curP = cur;
            int l = l0;
            bool enter = true;
            bool over_budget = false;
            // one maximal clique of sz vertices: R's first sz - nx ids (rid) and up
            // to three more (x1..x3); sum = the sum of its members' hash ids
            auto record = [&](int sz, uint64_t sum, int nx, int32_t x1, int32_t x2, int32_t x3) {
                if (g.gl == 0) {
                    t_cnt++;
                    t_hash += mix64(sum + (uint64_t)sz * kPhi);
                    if (block_hist) atomicAdd(&hist[sz], 1ull);
                    else hist[sz] += 1ull;
                    acc_maxsz = max(acc_maxsz, sz);
                    if (listing) {
                        // the cursor counts every record; only those that fit are written
                        const unsigned long long pos = atomicAdd(O.list_used, (unsigned long long)sz + 1ull);
                        if (pos + (unsigned long long)sz + 1ull <= O.list_cap) {
                            int32_t *dst = O.list + pos;
                            const int nr = sz - nx;
                            dst[0] = sz;
                            for (int i = 0; i < nr; i++) dst[1 + i] = (int32_t)rid[i];
                            if (nx > 0) dst[1 + nr] = x1;
                            if (nx > 1) dst[2 + nr] = x2;
                            if (nx > 2) dst[3 + nr] = x3;
                        }
                    }
                }
            };
            // move the X_X rows e of xidx[0, n_in) with holds(e) to the front; returns their number
            auto partition = [&](int n_in, auto holds) -> int {
                int out = 0, nout = 0;
                for (int it = 0; it < n_in; it += GT) {
                    const int idx = it + g.gl;
                    const bool valid = idx < n_in;
                    const uint32_t e = valid ? xidx[idx] : 0u;
                    const bool surv = valid && holds(e);
                    int ts, tn;
                    const int ps = grp_prefix(g, red, surv, &ts);
                    const int pn = grp_prefix(g, red, valid && !surv, &tn);
                    if (surv) xidx[out + ps] = e;
                    else if (valid) xscr[nout + pn] = e;
                    out += ts;
                    nout += tn;
                }
                if (nout > 0) {
                    g.sync();
                    for (int j = g.gl; j < nout; j += GT) xidx[out + j] = xscr[j];
                }
                g.sync();
                return out;
            };
            // claim an idle group for a donation (-1: none): the lanes read 32 words
            // of the idle bitmap at a time, and the first lane holding a set bit
            // tries to take one with atomicAnd (another donor may win the race)
            auto claim_idle = [&]() -> int {
                if (g.warp == 0) {
                    int claimed = -1;
                    const bool any_idle =
                        __shfl_sync(0xffffffffu, g.lane == 0 ? ld_relaxed(&C.ctl[CTL_IDLE]) > 0 : false, 0);
                    if (any_idle) {
                        const int nwords = (ngroups + 31) >> 5;
                        for (int q0 = 0; q0 < nwords && claimed < 0; q0 += 32) {
                            const int qd = q0 + g.lane;
                            const int wi = (gg / 32 + 1 + qd) % nwords;
                            const unsigned bits = qd < nwords ? *((volatile unsigned *)&C.idle_bits[wi]) : 0u;
                            unsigned nz = __ballot_sync(0xffffffffu, bits != 0u);
                            while (nz && claimed < 0) {
                                const int src = __ffs(nz) - 1;
                                nz &= nz - 1;
                                int got = -1;
                                if (g.lane == src) {
                                    unsigned left = bits;
                                    while (left) {
                                        const int bb = __ffs(left) - 1;
                                        const unsigned old = atomicAnd(&C.idle_bits[wi], ~(1u << bb));
                                        if (old & (1u << bb)) {
                                            got = wi * 32 + bb;
                                            break;
                                        }
                                        left = old & ~(1u << bb) & ~((2u << bb) - 1u);
                                    }
                                }
                                claimed = __shfl_sync(0xffffffffu, got, src);
                            }
                        }
                        if (claimed >= 0 && g.lane == 0) {
                            atomicSub(&C.ctl[CTL_IDLE], 1);
                            atomicAdd(&C.ctl[CTL_ACTIVE], 1);
                        }
                    }
                    if (g.lane == 0) misc[4] = claimed;
                }
                g.sync();
                const int recv = misc[4];
                g.sync();
                return recv;
            };

            // Compact mode (one-warp groups). A node with |P| + |X_P| <= 32 and
            // its whole subtree run on one-word sets over the index space
            // L = P u X_P of that node, in ascending local index so ties still go
            // to the smaller rank. Lane i holds L[i]'s adjacency row over L (kRow),
            // its local index (kL) and clique-hash id (kmj), and the saved state
            // of compact depth i (ks*); X_X rows are re-encoded over L once. Entered from a wide descent, at a root with |P0| <= 32, or
            // from a donated compact subtree; when the subtree is done the wide
            // loop backtracks as from any child.
            bool kstart = false;
            bool kmode = false, kcentr = false, kpend = false;
            // In compact mode the node's P, X_P, branch set, X_X end and hash sum
            // reuse the wide registers: the wide node is on the stack meanwhile.
            uint32_t &kP = p, &kX = xp, &kB = b;
            uint64_t &kS = S;
            uint32_t kRow = 0u;
            // X_X rows at compact entry (lane i keeps row i, and its rank, in kxr
            // and kxk; rows 32 and on in xcomp[i], ranks in xscr[i]); kRc = the
            // compact part of R as bits over L
            int kclx = 0;
            uint32_t kxr = 0u, kxk = 0u, kRc = 0u;
            int kL = 0, kd = 0, kbase = 0;
            if (edge) {
                // Algorithm 4: R = {r, v_j}; P = the common neighbours after v_j,
                // X = those before it: X_P from P0, X_X = the rows holding j
                const int j = ej, jw = j >> 5;
                const uint32_t jb = 1u << (j & 31);
                const uint32_t aj = own ? Arow[(size_t)j * WP + g.gl] : 0u;
                const uint32_t above = g.gl > jw ? 0xffffffffu : (g.gl == jw ? ~((jb << 1) - 1u) : 0u);
                p = aj & above;
                xp = aj & ~above;
                if (lpx > 0) lpx = partition(lpx, [&](uint32_t e) { return (xrows[(size_t)e * WP + jw] & jb) != 0u; });
                S += G.mixid[p0[j]];
                if (g.gl == 0) stk[Lvl<WP>::VSEL] = (uint32_t)j;  // level 0's branch, for donated paths
                if (listing && g.gl == 0) rid[1] = (uint32_t)G.order[p0[j]];
                const int np_e = grp_sum(g, red, __popc(p));
                if (np_e == 0) {
                    // a leaf: {r, v_j} is maximal iff X is empty
                    t_nodes++;
                    if (!grp_or(g, red, xp != 0u) && lpx == 0 && g.gl == 0) record(2, S, 0, 0, 0, 0);
                    b = 0u;
                    enter = false;
                } else if (GW == 1 && np_e + grp_sum(g, red, __popc(xp)) <= 32) {
                    kstart = true;
                }
            }
            if (fast) {
                // the root itself, in compact mode over L = P0 (local index = lane)
                kRow = f_row;
                kL = g.lane < n0 ? g.lane : 0;
                kP = n0 == 32 ? 0xffffffffu : (1u << n0) - 1u;
                kX = 0u;
                kclx = nx;
                kxr = f_xr;
                kxk = ipx_rule ? f_xk : 0u;
                kRc = 0u;
                kbase = 1;
                kd = 0;
                kcentr = true;
                kpend = false;
                kmode = true;
                t_nodes++;  // the root node
                enter = false;
            }
            if (cmail) {
                kRow = mb[4 + g.lane];
                kL = (int)mb[36 + g.lane];
                kP = mb[68];
                kX = mb[69];
                kS = (uint64_t)mb[70] | ((uint64_t)mb[71] << 32);
                // the donor wrote the surviving X_X rows to xcomp, their ranks to xscr
                kclx = (int)mb[2];
                kxr = g.lane < kclx ? xcomp[g.lane] : 0u;
                kxk = (ipx_rule && g.lane < kclx) ? xscr[g.lane] : 0u;
                kRc = 0u;
                kbase = l0 + 1;
                kd = 0;
                kcentr = true;
                kmode = true;
                t_nodes++;  // the donated node
                enter = false;
            }
            while (true) {
                if ((++iters & 1023u) == 0) {
                    // group-uniform decision (every thread must leave together)
                    if (grp_or(g, red, g.gl == 0 && tick())) {
                        over_budget = true;
                        break;
                    }
                }
                if (GW == 1 && kstart) {
                    // enter compact mode at the current node (P = p, X_P = xp, X_X =
                    // xidx[0, lpx), hash sum S, level l)
                    constexpr unsigned FULL = 0xffffffffu;
                    kstart = false;
                    t_nodes++;  // the node itself
                    const int c = grp_bits_to_list<WP, GW>(g, red, own ? (p | xp) : 0u, cand);
                    if (own) curP[g.gl] = p;
                    __syncwarp();
                    const bool inl = g.lane < c;
                    kL = inl ? cand[g.lane] : 0;
                    const bool inP = inl && ((curP[kL >> 5] >> (kL & 31)) & 1u) != 0u;
                    kP = __ballot_sync(FULL, inP);
                    kX = __ballot_sync(FULL, inl && !inP);
                    // At a root L is P0 itself (local indices 0 .. c-1): rows and
                    // X_X rows are their first words. Elsewhere each lane gathers
                    // the bits of L from its row (lane i: A row of L[i]; lane k:
                    // X_X row k).
                    const bool ident = l == 0;
                    const uint32_t cmask = c == 32 ? FULL : (1u << c) - 1u;
                    kRow = 0u;
                    if (ident) {
                        if (inl) kRow = Arow[(size_t)kL * WP] & cmask;
                    } else {
                        const uint32_t *ar_ = Arow + (size_t)kL * WP;
#pragma unroll 4
                        for (int j = 0; j < c; j++) {
                            const int lj = __shfl_sync(FULL, kL, j);
                            kRow |= ((ar_[lj >> 5] >> (lj & 31)) & 1u) << j;
                        }
                        if (!inl) kRow = 0u;
                    }
                    // the X_X rows over L, by position: lane i keeps row i (and
                    // its rank) in registers, rows 32 and on go to xcomp[i] and
                    // their ranks to xscr[i]
                    kclx = lpx;
                    for (int i0 = 0; i0 < kclx; i0 += 32) {
                        const int i = i0 + g.lane;
                        const uint32_t e = i < kclx ? xidx[i] : 0u;
                        const uint32_t *xr = xrows + (size_t)e * WP;
                        uint32_t w = 0u;
                        if (ident) {
                            w = xr[0] & cmask;
                        } else {
#pragma unroll 4
                            for (int j = 0; j < c; j++) {
                                const int lj = __shfl_sync(FULL, kL, j);
                                w |= ((xr[lj >> 5] >> (lj & 31)) & 1u) << j;
                            }
                        }
                        const uint32_t rk = (ipx_rule && i < kclx) ? xrank[e] : 0u;
                        if (i0 == 0) {
                            kxr = i < kclx ? w : 0u;
                            kxk = rk;
                        } else if (i < kclx) {
                            xcomp[i] = w;
                            xscr[i] = rk;
                        }
                    }
                    __syncwarp();
                    kRc = 0u;
                    kbase = l + 1;
                    kd = 0;
                    kcentr = true;
                    kpend = npend > 0;
                    kmode = true;
                    enter = false;
                    pc.stop(PH_CENTRY);
                    pc.count(PH_CENTRY, (unsigned long long)kclx);
                }
                if (GW == 1 && kmode) {
                    constexpr unsigned FULL = 0xffffffffu;
                    const bool ipx = ipx_rule;
                    // lane i: clique-hash id of L[i] (lanes past |L| hold a harmless
                    // copy of P0[0]'s), and the saved state of compact depth i
                    const uint64_t kmj = G.mixid[p0[kL]];
                    const int32_t kid = listing ? G.order[p0[kL]] : 0;  // input id of L[i]
                    uint32_t ksP = 0u, ksX = 0u, ksB = 0u, ksR = 0u;
                    uint64_t ksS = 0ull;
                    // The X_X of a compact node is the entry rows that hold all of
                    // R's compact part Rc (each branch keeps the rows adjacent to
                    // its vertex), so no list is partitioned on the way down.
                    // row_at: X_X row i (and its rank) of the lane's entry in the
                    // chunk starting at i0
                    auto row_at = [&](int i0, int i) -> uint32_t { return i0 == 0 ? kxr : (i < kclx ? xcomp[i] : 0u); };
                    auto rank_at = [&](int i0, int i) -> uint32_t { return i0 == 0 ? kxk : (i < kclx ? xscr[i] : 0u); };
                    // any X_X row holding all of `need` (Rc plus the branch) with f(row)
                    auto xx_any = [&](uint32_t need, auto f) -> bool {
                        bool found = false;
                        for (int i0 = 0; i0 < kclx && !found; i0 += 32) {
                            const int i = i0 + g.lane;
                            const uint32_t xc = row_at(i0, i);
                            found = __any_sync(FULL, i < kclx && (xc & need) == need && f(xc)) != 0;
                        }
                        return found;
                    };
                    for (;;) {
                        if (kcentr) {
                            kcentr = false;
                            // pivot over P u X_P: lane u scores |P n N(u)|, ties to the
                            // smaller index; IPX also scores the X_X rows, which win ties
                            const bool isc = (((kP | kX) >> g.lane) & 1u) != 0u;
                            const unsigned key =
                                isc ? (((unsigned)__popc(kRow & kP) + 1u) << 8) | (unsigned)(31 - g.lane) : 0u;
                            const unsigned best = __reduce_max_sync(FULL, key);
                            const int bsc = (int)(best >> 8) - 1;
                            uint32_t prow = __shfl_sync(FULL, kRow, 31 - (int)(best & 255u));
                            // An X_P candidate adjacent to all of P leaves no branch, and
                            // so would any X_X row that beat it: skip the X_X scan then
                            if (ipx && kclx > 0 && bsc < __popc(kP)) {
                                // the best X_X row: largest score, then smallest rank
                                int xs = 0;
                                uint32_t xk = 0u, xrow = 0u;
                                for (int i0 = 0; i0 < kclx; i0 += 32) {
                                    const int i = i0 + g.lane;
                                    const uint32_t xc = row_at(i0, i);
                                    const bool cur = i < kclx && (xc & kRc) == kRc;
                                    const int s = cur ? __popc(xc & kP) + 1 : 0;
                                    const int sm = (int)__reduce_max_sync(FULL, (unsigned)s);
                                    if (sm == 0 || sm < xs) continue;
                                    const uint32_t rk = rank_at(i0, i);
                                    const uint32_t inv = s == sm ? 0xffffffffu - rk : 0u;
                                    const uint32_t bi = __reduce_max_sync(FULL, inv);
                                    if (sm > xs || 0xffffffffu - bi < xk) {
                                        const unsigned hm = __ballot_sync(FULL, s == sm && inv == bi);
                                        xrow = __shfl_sync(FULL, xc, __ffs(hm) - 1);
                                        xk = 0xffffffffu - bi;
                                        xs = sm;
                                    }
                                }
                                if (xs - 1 >= bsc && xs > 0) prow = xrow;
                            }
                            kB = kP & ~prow;
                            pc.stop(PH_PIVOT);
                            pc.count(PH_PIVOT, (unsigned long long)__popc(kP | kX));
                        }
                        if (kB == 0u) {
                            if (kd == 0) break;  // the compact subtree is done
                            kd--;
                            kP = __shfl_sync(FULL, ksP, kd);
                            kX = __shfl_sync(FULL, ksX, kd);
                            kB = __shfl_sync(FULL, ksB, kd);
                            kRc = __shfl_sync(FULL, ksR, kd);
                            kS = __shfl_sync(FULL, ksS, kd);
                            pc.stop(PH_POP);
                            pc.count(PH_POP, 1);
                            continue;
                        }
                        const int u = __ffs(kB) - 1;
                        const uint32_t ubit = 1u << u;
                        const uint32_t ru = __shfl_sync(FULL, kRow, u);
                        const uint32_t q = kP & ru, qx = kX & ru;  // the child's P and X_P
                        kB &= ~ubit;
                        kP &= ~ubit;
                        kX |= ubit;
                        const int qn = __popc(q);
                        const uint64_t mu = __shfl_sync(FULL, kmj, u);
                        const int32_t idu = __shfl_sync(FULL, kid, u);
                        const int szc = kbase + kd + 1;  // |R u {u}|
                        const uint32_t need = kRc | ubit;  // the child's Rc
                        pc.stop(PH_BRANCH);
                        if (qn <= 2) {
                            t_nodes++;
                            // the child's X_X rows are the rows holding `need`
                            if (qn == 0) {
                                if (qx == 0u && !xx_any(need, [](uint32_t) { return true; }))
                                    record(szc, kS + mu, 1, idu, 0, 0);
                            } else if (qn == 1) {
                                // as for a one-vertex P' in the wide walk
                                const int w = __ffs(q) - 1;
                                const uint32_t rw = __shfl_sync(FULL, kRow, w);
                                if ((qx & rw) == 0u) {
                                    const uint32_t both = ubit | (1u << w);
                                    const bool found = xx_any(need, [&](uint32_t xc) { return (xc & both) == both; });
                                    if (!found || !ipx) t_nodes++;
                                    const int32_t idw = __shfl_sync(FULL, kid, w);
                                    if (!found) record(szc + 1, kS + mu + __shfl_sync(FULL, kmj, w), 2, idu, idw, 0);
                                }
                            } else {
                                // as for a two-vertex P' in the wide walk
                                const int w1 = __ffs(q) - 1, w2 = 31 - __clz(q);
                                const uint32_t a1 = __shfl_sync(FULL, kRow, w1), a2 = __shfl_sync(FULL, kRow, w2);
                                const uint64_t m1 = __shfl_sync(FULL, kmj, w1), m2 = __shfl_sync(FULL, kmj, w2);
                                const int32_t id1 = __shfl_sync(FULL, kid, w1), id2 = __shfl_sync(FULL, kid, w2);
                                const bool e12 = ((a1 >> w2) & 1u) != 0u;
                                const bool s2p = (qx & a1 & a2) != 0u;
                                const uint32_t one = qx & (a1 ^ a2);
                                bool s2x = false, x1 = false, x2 = false;
                                unsigned firstx = 0u;
                                for (int i0 = 0; i0 < kclx; i0 += 32) {
                                    const int i = i0 + g.lane;
                                    bool h1 = false, h2 = false;
                                    unsigned k1 = 0u;
                                    const uint32_t xc = row_at(i0, i);
                                    if (i < kclx && (xc & need) == need) {
                                        h1 = ((xc >> w1) & 1u) != 0u;
                                        h2 = ((xc >> w2) & 1u) != 0u;
                                        if (ipx && h1 != h2) k1 = ((0x7fffffffu - rank_at(i0, i)) << 1) | (h1 ? 1u : 0u);
                                    }
                                    s2x |= __any_sync(FULL, h1 && h2) != 0;
                                    x1 |= __any_sync(FULL, h1) != 0;
                                    x2 |= __any_sync(FULL, h2) != 0;
                                    if (ipx) firstx = max(firstx, __reduce_max_sync(FULL, k1));
                                }
                                const bool s2 = s2p || (ipx && s2x);
                                if (e12) {
                                    if (!s2) {
                                        t_nodes += 2;
                                        if (!s2x) record(szc + 2, kS + mu + m1 + m2, 3, idu, id1, id2);
                                    }
                                } else if (!s2) {
                                    int touch = 0;
                                    if (firstx) touch = (firstx & 1u) ? 1 : 2;
                                    else if (one) touch = ((a1 >> (__ffs(one) - 1)) & 1u) ? 1 : 2;
                                    if (touch) {
                                        t_nodes++;
                                        const uint32_t aj = touch == 1 ? a2 : a1;
                                        const bool xj = touch == 1 ? x2 : x1;
                                        if (!xj && (qx & aj) == 0u)
                                            record(szc + 1, kS + mu + (touch == 1 ? m2 : m1), 2, idu, touch == 1 ? id2 : id1, 0);
                                    } else {
                                        t_nodes += 2;
                                        if (!x1) record(szc + 1, kS + mu + m1, 2, idu, id1, 0);
                                        if (!x2) record(szc + 1, kS + mu + m2, 2, idu, id2, 0);
                                    }
                                }
                            }
                            pc.stop(PH_LEAF);
                            continue;
                        }
                        // donation of the child as a compact subtree (Sec. III-C): the
                        // receiver gets the rows over L, the child's sets and its X_X rows
                        if (C.worker_list && qn >= C.donate_min_p) {
                            const bool above = kpend || __ballot_sync(FULL, g.lane < kd && ksB != 0u) != 0u;
                            const bool may = C.donate_policy == MCE_DONATE_ANY ||
                                             (C.donate_policy == MCE_DONATE_EITHER ? (kB != 0u || above)
                                                                                   : (kB != 0u && above));
                            if (may) {
                                const int recv = claim_idle();
                                if (recv >= 0) {
                                    const ArenaPtrs ra = arena_at(C.arena + (size_t)recv * C.arena_words_per_group, WP,
                                                                  rows_cap, C.x_cap, stack_smem != 0);
                                    int out = 0;
                                    for (int i0 = 0; i0 < kclx; i0 += 32) {
                                        const int i = i0 + g.lane;
                                        const uint32_t xc = row_at(i0, i);
                                        const bool surv = i < kclx && (xc & need) == need;
                                        const unsigned bm = __ballot_sync(FULL, surv);
                                        if (surv) {
                                            const int k = out + __popc(bm & ((1u << g.lane) - 1u));
                                            ra.xcomp[k] = xc;
                                            ra.xscr[k] = rank_at(i0, i);
                                        }
                                        out += __popc(bm);
                                    }
                                    uint32_t *m = C.mail + (size_t)recv * C.mail_words;
                                    m[4 + g.lane] = kRow;
                                    m[36 + g.lane] = (uint32_t)kL;
                                    if (g.lane == 0) {
                                        const uint64_t s2 = kS + mu;
                                        m[0] = (uint32_t)r;
                                        m[1] = (uint32_t)(szc - 1);
                                        m[2] = (uint32_t)out;
                                        m[3] = 1u;
                                        m[68] = q;
                                        m[69] = qx;
                                        if (listing) {
                                            for (int qd = 0; qd < szc - 1; qd++) ra.rid[qd] = rid[qd];
                                            ra.rid[szc - 1] = (uint32_t)idu;
                                        }
                                        m[70] = (uint32_t)s2;
                                        m[71] = (uint32_t)(s2 >> 32);
                                    }
                                    __threadfence();
                                    __syncwarp();
                                    if (g.lane == 0) {
                                        st_release(&C.mail_flag[(size_t)recv * kMailFlagStride], 1);
                                        acc_don++;
                                    }
                                    __syncwarp();
                                    pc.stop(PH_DONATE);
                                    pc.count(PH_DONATE, 1);
                                    continue;
                                }
                            }
                            pc.stop(PH_DONATE);
                        }
                        // descend: this node's state goes to lane kd
                        if (g.lane == kd) {
                            ksP = kP;
                            ksX = kX;
                            ksB = kB;
                            ksR = kRc;
                            ksS = kS;
                        }
                        if (listing && g.lane == 0) rid[kbase + kd] = (uint32_t)idu;
                        kRc = need;
                        kP = q;
                        kX = qx;
                        kS += mu;
                        kd++;
                        kcentr = true;
                        t_nodes++;
                        pc.stop(PH_PARTITION);
                        // the budget and heartbeat check, on descents only: between two
                        // descents a compact walk takes at most about 33 steps
                        if ((++iters & 255u) == 0 && __any_sync(FULL, g.lane == 0 && tick())) {
                            over_budget = true;
                            break;
                        }
                        continue;
                    }
                    // the compact subtree is done; the wide loop backtracks (the
                    // branch set is empty, and words no thread owns are 0)
                    kmode = false;
                    if (over_budget) break;
                    if (!ownw) {
                        p = 0u;
                        xp = 0u;
                    }
                    continue;
                }
                if (enter) {
                    t_nodes++;
                    if (own) curP[g.gl] = p;
                    const int np = grp_sum(g, red, __popc(p));
                    const int xany = grp_or(g, red, xp != 0u);
                    // candidate list P u X_P in ascending index
                    const int nc = grp_bits_to_list<WP, GW>(g, red, own ? (p | xp) : 0u, cand);
                    // Pivot: the candidate with the largest |P n N(u)|, ties to the
                    // smaller degeneracy rank. P u X_P candidates are keyed
                    // score << 16 | (0xffff - local index) (local index order is rank
                    // order). X_X candidates (IPX) all rank below every P0 vertex and
                    // compare among themselves by score << 32 | ~rank.
                    int best_x_score = -1;  // best X_X score, -1 if none scanned
                    int piv_x = -1;         // X_X slot of the best X_X candidate
                    int scanned = 0;
                    if (ipx_rule && lpx > 0) {
                        unsigned long long bx = 0;
                        for (int j0 = 0; j0 < lpx; j0 += GT) {
                            const int j = j0 + g.gl;
                            unsigned long long key = 0;
                            if (j < lpx) {
                                const uint32_t e = xidx[j];
                                const uint32_t *xr = xrows + (size_t)e * WP;
                                int sc = 0;
                                for (int w = 0; w < W; w++) sc += __popc(xr[w] & curP[w]);
                                key = ((unsigned long long)(sc + 1) << 32) | (unsigned long long)(0xffffffffu - xrank[e]);
                            }
                            const unsigned long long m = grp_max64(g, (unsigned long long *)red, key);
                            bx = m > bx ? m : bx;
                        }
                        scanned += lpx;
                        best_x_score = (int)(bx >> 32) - 1;
                        // the slot of the winning X_X vertex (ranks are unique)
                        const uint32_t want_rank = 0xffffffffu - (uint32_t)(bx & 0xffffffffull);
                        int found = -1;
                        for (int j0 = 0; j0 < lpx && found < 0; j0 += GT) {
                            const int j = j0 + g.gl;
                            const int hit = (j < lpx && xrank[xidx[j]] == want_rank) ? j : -1;
                            found = (int)grp_max(g, red, (unsigned)(hit + 1)) - 1;
                        }
                        if (found >= 0) piv_x = (int)xidx[found];
                        else best_x_score = -1;  // cannot happen (the max key came from a slot)
                    }
                    int piv = -1;  // P0 local index of the pivot when it is not an X_X vertex
                    if (best_x_score < np) {
                        // best score a P u X_P candidate can reach: |P| in X_P, |P|-1 in P
                        const unsigned bound = (unsigned)(xany ? np : np - 1);
                        unsigned best = 0;
                        for (int j0 = 0; j0 < nc; j0 += GT) {
                            const int j = j0 + g.gl;
                            unsigned key = 0;
                            if (j < nc) {
                                const int c = cand[j];
                                const uint32_t *arow = Arow + (size_t)c * WP;
                                int sc = 0;
                                if (WP % 4 == 0) {
                                    const uint4 *a4 = reinterpret_cast<const uint4 *>(arow);
                                    const uint4 *p4 = reinterpret_cast<const uint4 *>(curP);
                                    for (int qq = 0; qq < (W + 3) / 4; qq++) {
                                        const uint4 a = a4[qq], pw = p4[qq];
                                        sc += __popc(a.x & pw.x) + __popc(a.y & pw.y) + __popc(a.z & pw.z) +
                                              __popc(a.w & pw.w);
                                    }
                                } else {
                                    for (int w = 0; w < W; w++) sc += __popc(arow[w] & curP[w]);
                                }
                                key = ((unsigned)sc << 16) | (unsigned)(0xffff - c);
                            }
                            best = max(best, grp_max(g, red, key));
                            scanned += min(nc - j0, GT);
                            if ((best >> 16) >= bound) break;
                        }
                        // an X_X vertex wins ties (smaller rank)
                        if ((int)(best >> 16) > best_x_score) piv = 0xffff - (int)(best & 0xffffu);
                    }
                    if (piv >= 0) {
                        b = own ? (p & ~Arow[(size_t)piv * WP + g.gl]) : 0u;
                    } else {
                        b = own ? (p & ~xrows[(size_t)piv_x * WP + g.gl]) : 0u;
                    }
                    enter = false;
                    pc.stop(PH_PIVOT);
                    pc.count(PH_PIVOT, (unsigned long long)scanned);
                }
                // --------------------------------------- next branch: lowest bit of B
                const unsigned bkey = b ? ~(unsigned)(g.gl * 32 + __ffs(b) - 1) : 0u;
                const unsigned bsel = grp_max(g, red, bkey);
                if (bsel == 0u) {
                    // all branches done: backtrack
                    pc.stop(PH_BRANCH);
                    if (l == l0) break;
                    l--;
                    const uint32_t *lv = stk + (size_t)l * LS;
                    if (ownw) {
                        p = lv[Lvl<WP>::P + g.gl];
                        xp = lv[Lvl<WP>::XP + g.gl];
                        b = lv[Lvl<WP>::B + g.gl];
                    }
                    lpx = (int)lv[Lvl<WP>::LPX];
                    npend = (int)lv[Lvl<WP>::NPEND];
                    S = (uint64_t)lv[Lvl<WP>::SLO] | ((uint64_t)lv[Lvl<WP>::SHI] << 32);
                    if (pc.on) {
                        // wait for the reloads so that their latency lands in this phase
                        const uint32_t used = p ^ xp ^ b ^ (uint32_t)lpx ^ (uint32_t)npend ^ (uint32_t)S;
                        asm volatile("" ::"r"(used));
                        pc.stop(PH_POP);
                        pc.count(PH_POP, 1);
                    }
                    continue;
                }
                const int v = (int)(~bsel);
                const int vw = v >> 5;
                const uint32_t vb = 1u << (v & 31);
                // child sets P n N(v), X_P n N(v); then P -= v, X_P += v, B -= v
                const uint32_t av = own ? Arow[(size_t)v * WP + g.gl] : 0u;
                const uint32_t cp = p & av, cx = xp & av;
                if (g.gl == vw) {
                    b &= ~vb;
                    p &= ~vb;
                    xp |= vb;
                }
                const int pcnt = grp_sum(g, red, __popc(cp));
                const int xa = grp_or(g, red, cx != 0u);
                pc.stop(PH_BRANCH);
                if (pcnt == 0) {
                    // the child is a leaf: R u {v} is maximal iff X_P' and X_X' are empty
                    t_nodes++;
                    if (!xa) {
                        int found = 0, it = 0;
                        for (; it < lpx && !found; it += GT) {
                            const int idx = it + g.gl;
                            int hit = 0;
                            if (idx < lpx) hit = (xrows[(size_t)xidx[idx] * WP + vw] & vb) != 0u;
                            found = grp_or(g, red, hit);
                        }
                        pc.count(PH_LEAF, (unsigned long long)min(it, lpx));
                        if (!found && g.gl == 0)
                            record(l + 2, S + G.mixid[p0[v]], 1, listing ? G.order[p0[v]] : 0, 0, 0);
                    }
                    pc.stop(PH_LEAF);
                    continue;
                }
                const int others_here = grp_or(g, red, b != 0u);
                // ------------------------------ donation (Sec. III-C)
                const bool may_donate = C.donate_policy == MCE_DONATE_ANY ||
                                        (C.donate_policy == MCE_DONATE_EITHER ? (others_here || npend >= 1)
                                                                              : (others_here && npend >= 1));
                if (C.worker_list && pcnt >= C.donate_min_p && may_donate) {
                    const int recv = claim_idle();
                    if (recv >= 0) {
                        // X_X of the child = rows of this level's prefix with bit v
                        int out = 0;
                        for (int it = 0; it < lpx; it += GT) {
                            const int idx = it + g.gl;
                            const bool valid = idx < lpx;
                            const uint32_t e = valid ? xidx[idx] : 0u;
                            const bool surv = valid && (xrows[(size_t)e * WP + vw] & vb) != 0u;
                            int ts;
                            const int ps = grp_prefix(g, red, surv, &ts);
                            if (surv) xscr[out + ps] = e;
                            out += ts;
                        }
                        __threadfence_block();
                        g.sync();
                        // push A and the surviving rows into the receiver's arena
                        const ArenaPtrs ra = arena_at(C.arena + (size_t)recv * C.arena_words_per_group, WP,
                                                      rows_cap, C.x_cap, stack_smem != 0);
                        {
                            // only the rows of the child's P' u X_P'
                            const int nrows = grp_bits_to_list<WP, GW>(g, red, own ? (cp | cx) : 0u, cand);
                            grp_copy_rows<WP, GW>(g, cand, nrows, Arow, ra.A);
                        }
                        for (int i = g.gl; i < out * WP; i += GT) {
                            const int k = i / WP, w = i - k * WP;
                            ra.xrows[i] = xrows[(size_t)xscr[k] * WP + w];
                        }
                        for (int k = g.gl; k < out; k += GT) {
                            ra.xidx[k] = (uint32_t)k;
                            ra.xrank[k] = xrank[xscr[k]];
                        }
                        uint32_t *m = C.mail + (size_t)recv * C.mail_words;
                        if (own) {
                            m[4 + g.gl] = 0u;
                            m[4 + WP + g.gl] = cp;
                            m[4 + 2 * WP + g.gl] = cx;
                        }
                        g.sync();
                        if (g.gl == 0) {
                            // R' = the path below the root at levels [0, l), plus v
                            for (int qd = 0; qd < l; qd++) {
                                const int u = (int)stk[(size_t)qd * LS + Lvl<WP>::VSEL];
                                m[4 + (u >> 5)] |= 1u << (u & 31);
                            }
                            m[4 + vw] |= vb;
                            m[0] = (uint32_t)r;
                            m[1] = (uint32_t)(l + 1);
                            m[2] = (uint32_t)out;
                            m[3] = 0u;
                            if (listing) {
                                for (int qd = 0; qd <= l; qd++) ra.rid[qd] = rid[qd];
                                ra.rid[l + 1] = (uint32_t)G.order[p0[v]];
                            }
                        }
                        __threadfence();
                        g.sync();
                        if (g.gl == 0) {
                            st_release(&C.mail_flag[(size_t)recv * kMailFlagStride], 1);
                            acc_don++;
                        }
                        g.sync();
                        pc.stop(PH_DONATE);
                        pc.count(PH_DONATE, 1);
                        continue;
                    }
                    pc.stop(PH_DONATE);
                }
                // A child with |P'| + |X_P'| <= 32 runs in compact mode (below) after
                // the usual push of this level and partition of X_X.
                bool to_compact = false;
                if (GW == 1 && WP > 1 && pcnt <= 32) to_compact = pcnt + grp_sum(g, red, __popc(cx)) <= 32;
                // ------------------------------ descend: push this level, partition X_X by v
                {
                    uint32_t *lv = stk + (size_t)l * LS;
                    if (ownw) {
                        lv[Lvl<WP>::P + g.gl] = p;
                        lv[Lvl<WP>::XP + g.gl] = xp;
                        lv[Lvl<WP>::B + g.gl] = b;
                    }
                    if (g.gl == 0) {
                        lv[Lvl<WP>::LPX] = (uint32_t)lpx;
                        lv[Lvl<WP>::NPEND] = (uint32_t)npend;
                        lv[Lvl<WP>::VSEL] = (uint32_t)v;
                        lv[Lvl<WP>::SLO] = (uint32_t)S;
                        lv[Lvl<WP>::SHI] = (uint32_t)(S >> 32);
                    }
                    int out = 0;
                    if (lpx > 0) out = partition(lpx, [&](uint32_t e) { return (xrows[(size_t)e * WP + vw] & vb) != 0u; });
                    pc.stop(PH_PARTITION);
                    pc.count(PH_PARTITION, (unsigned long long)lpx);
                    p = cp;
                    xp = cx;
                    lpx = out;
                    npend += others_here ? 1 : 0;
                    S += G.mixid[p0[v]];
                    if (listing && g.gl == 0) rid[l + 1] = (uint32_t)G.order[p0[v]];
                }
                l++;
                enter = true;
                if (l > rows_cap) {
                    if (g.gl == 0) atomicOr(O.status, ST_OVERFLOW);
                    break;
                }
                if (GW == 1 && to_compact) {
                    kstart = true;
                    enter = false;
                }
            }
            if (over_budget && g.gl == 0) atomicOr(O.status, ST_BUDGET);
            g.sync();
            if (ld_relaxed(O.status) & (ST_TIMEOUT | ST_OVERFLOW | ST_BUDGET)) break;
            // --------------------------------------------------- task done
            if (g.gl == 0) {
                acc_nodes += t_nodes;
                acc_cnt += t_cnt;
                acc_hash += t_hash;
                pc.count(PH_BRANCH, t_nodes);
                const int id = G.order[r];
                if (O.root_nodes) atomicAdd(&O.root_nodes[id], t_nodes);
                if (O.root_count && t_cnt) atomicAdd(&O.root_count[id], t_cnt);
                if (O.root_hash && t_hash) atomicAdd(&O.root_hash[id], t_hash);
            }
            g.sync();
        }
        // group end: flush the group's results
        flush();
        if (g.gl == 0) {
            if (acc_nodes) atomicAdd(O.nodes, acc_nodes);
            if (acc_don) atomicAdd(O.donations, acc_don);
            if (acc_maxsz) atomicMax(O.max_size, acc_maxsz);
            if (pc.on) {
                for (int k = 0; k < kNumPhases; k++) {
                    if (pc.cyc[k]) atomicAdd(&O.phase_cycles[k], pc.cyc[k]);
                    if (pc.cnt[k]) atomicAdd(&O.phase_counts[k], pc.cnt[k]);
                }
            }
        }
    }
    if (block_hist) {
        // every warp of the block reaches this barrier exactly once
        __syncthreads();
        for (int s = threadIdx.x; s < rows_cap + 2; s += blockDim.x) {
            unsigned long long c = bhist[s];
            if (c && s < O.hist_len) atomicAdd(&O.hist[s], c);
        }
    }
}

}  // namespace mce
