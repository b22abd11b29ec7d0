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
// subgraphs), ties to the smallest local index = smallest rank. Branches:
// P - N(u) in ascending rank. R is maximal when P, X_P and X_X are all empty.
//
// Template parameters: WP padded words per row, GW warps per group, AG true
// when A lives in the global arena (rows too wide for shared memory).
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

// rounded to 4 words so whatever follows the stack stays 16-byte aligned
__host__ __device__ inline size_t stack_words(int wp, int rows) {
    return ((size_t)(rows + 2) * (3 * wp + 6) + 3) / 4 * 4;
}

// Shared-memory layout of one group (offsets in bytes from the group base).
struct GrpSmem {
    size_t a, p0, p0mix, cand, hist, cur, red, misc, stack, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// rows = max |P0| handled; stack_smem: DFS stack in shared memory
__host__ __device__ inline GrpSmem grp_smem_layout(int wp, int gw, int rows, bool a_global, bool stack_smem) {
    GrpSmem L;
    size_t off = 0;
    L.p0mix = off;
    off += (size_t)rows * 8;
    L.hist = off;
    off += (size_t)(rows + 2) * 8;
    off = align_up(off, 16);
    L.a = off;
    if (!a_global) off += (size_t)rows * wp * 4;
    off = align_up(off, 16);
    L.cur = off;
    off += (size_t)wp * 4;
    off = align_up(off, 16);
    L.p0 = off;
    off += (size_t)rows * 4;
    L.cand = off;
    off += (size_t)rows * 4;
    L.red = off;
    off += (size_t)gw * 4 * 4;
    L.misc = off;
    off += 16 * 4;
    off = align_up(off, 16);
    L.stack = off;
    if (stack_smem) off += stack_words(wp, rows) * 4;
    off = align_up(off, 16);
    L.total = off;
    return L;
}

// Arena words per group: [stack if global][A if global][X rows][xidx][xscr]
__host__ __device__ inline size_t arena_words(int wp, int rows, int xcap, bool a_global, bool stack_smem) {
    size_t w = 0;
    if (!stack_smem) w += stack_words(wp, rows);
    if (a_global) w += (size_t)rows * wp;
    w += (size_t)xcap * wp + 2 * (size_t)xcap;
    return align_up(w, 4);
}

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

template <int WP, int GW, bool AG>
__global__ void __launch_bounds__(256) k_traverse(DevGraph G, DevOut O, ClassArgs C, int rows_cap, int stack_smem) {
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
    if (g.gib >= gpb) return;
    const int gg = blockIdx.x * gpb + g.gib;  // global group id
    const int ngroups = gridDim.x * gpb;

    const GrpSmem L = grp_smem_layout(WP, GW, rows_cap, AG, stack_smem != 0);
    unsigned char *base = smem_raw + (size_t)g.gib * L.total;
    uint64_t *p0mix = (uint64_t *)(base + L.p0mix);
    unsigned long long *hist = (unsigned long long *)(base + L.hist);
    int32_t *p0 = (int32_t *)(base + L.p0);
    int32_t *cand = (int32_t *)(base + L.cand);
    uint32_t *cur = (uint32_t *)(base + L.cur);
    int *red = (int *)(base + L.red);
    int *misc = (int *)(base + L.misc);

    uint32_t *arena = C.arena + (size_t)gg * C.arena_words_per_group;
    uint32_t *stk;
    uint32_t *Arow;
    {
        uint32_t *q = arena;
        if (stack_smem) {
            stk = (uint32_t *)(base + L.stack);
        } else {
            stk = q;
            q += stack_words(WP, rows_cap);
        }
        if (AG) {
            Arow = q;
            q += (size_t)rows_cap * WP;
        } else {
            Arow = (uint32_t *)(base + L.a);
        }
        (void)q;
    }
    uint32_t *xrows = arena + (stack_smem ? 0 : stack_words(WP, rows_cap)) + (AG ? (size_t)rows_cap * WP : 0);
    uint32_t *xidx = xrows + (size_t)C.x_cap * WP;
    uint32_t *xscr = xidx + C.x_cap;

    const uint64_t deadline = globaltimer_ns() + C.timeout_ns;

    // per-group accumulators (meaningful in thread 0 of the group)
    unsigned long long acc_cnt = 0, acc_hash = 0, acc_nodes = 0, acc_don = 0;
    int acc_gid = -1, acc_maxsz = 0;
    unsigned descents = 0;
    for (int i = g.gl; i < rows_cap + 2; i += GT) hist[i] = 0;
    g.sync();

    auto flush = [&](void) {
        // add the group's accumulators to graph acc_gid and clear them
        if (acc_gid >= 0) {
            if (g.gl == 0) {
                if (acc_cnt) atomicAdd(&O.count[acc_gid], acc_cnt);
                if (acc_hash) atomicAdd(&O.hash[acc_gid], acc_hash);
            }
            for (int s = g.gl; s < rows_cap + 2; s += GT) {
                unsigned long long c = hist[s];
                if (c) {
                    if (s < O.hist_len) atomicAdd(&O.hist[(size_t)acc_gid * O.hist_len + s], c);
                    hist[s] = 0;
                }
            }
        }
        acc_cnt = 0;
        acc_hash = 0;
        g.sync();
    };

    int task_root = -1;  // rank of the current root
    bool have_mail = false;

    for (;;) {
        // ------------------------------------------------------- get a task
        if (g.gl == 0) {
            int r = -1, mail = 0;
            int idx = atomicAdd(&C.ctl[CTL_NEXT_ROOT], 1);
            if (idx < C.n_roots) {
                r = C.roots[idx];
            } else if (C.worker_list) {
                // join the worker list and wait for a donated subtree (Sec. III-C)
                atomicOr(&C.idle_bits[gg >> 5], 1u << (gg & 31));
                atomicAdd(&C.ctl[CTL_IDLE], 1);
                __threadfence();
                atomicSub(&C.ctl[CTL_ACTIVE], 1);
                unsigned ns = 64;
                for (;;) {
                    if (ld_acquire(&C.mail_flag[gg])) {
                        C.mail_flag[gg] = 0;
                        mail = 1;
                        r = (int)C.mail[(size_t)gg * C.mail_words + 0];
                        break;
                    }
                    if (ld_acquire(&C.ctl[CTL_ACTIVE]) == 0) break;
                    if (ld_relaxed(O.status) & ST_TIMEOUT) break;
                    if (globaltimer_ns() > deadline) {
                        atomicOr(O.status, ST_TIMEOUT);
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 4096) ns <<= 1;
                }
            }
            misc[0] = r;
            misc[1] = mail;
        }
        g.sync();
        task_root = misc[0];
        have_mail = misc[1] != 0;
        g.sync();
        if (task_root < 0) break;

        const int r = task_root;
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

        // ------------------------------------------- induced subgraph (Sec. III-D)
        for (int i = g.gl; i < n0; i += GT) {
            int32_t u = prow[i];
            p0[i] = u;
            p0mix[i] = G.mixid[u];
        }
        for (int i = g.gl; i < n0 * WP; i += GT) Arow[i] = 0u;
        g.sync();
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
        if (AG) __threadfence_block();
        g.sync();

        // ------------------------------------------ mailbox (donated subtree)
        const uint32_t *mb = C.mail + (size_t)gg * C.mail_words;
        // mail layout: [0] root, [1] level, [4..4+WP) R', then P', then XP'
        int l0 = 0;
        if (have_mail) l0 = (int)mb[1];

        // ------------------------------------------- X_X rows (Sec. III-E)
        int nx = 0;
        {
            int base_slot = 0;
            for (int it = 0; it < x0; it += GT) {
                int idx = it + g.gl;
                int hits = 0;
                int32_t x = 0;
                const int32_t *nr = nullptr;
                int len = 0;
                if (idx < x0) {
                    x = xrow[idx];
                    nr = G.out_col + G.out_ptr[x];
                    len = G.out_ptr[x + 1] - G.out_ptr[x];
                    int lo = 0;
                    for (int j = find_in(nr, 0, len, r + 1); j < len && lo < n0; j++) {
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
                    for (int j = find_in(nr, 0, len, r + 1); j < len && lo < n0; j++) {
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
                }
                base_slot += tot;
            }
            nx = base_slot;
        }
        __threadfence_block();
        g.sync();

        // ------------------------------------------------ initial node
        uint32_t *lv0 = stk + (size_t)l0 * LS;
        if (!have_mail) {
            for (int w = g.gl; w < WP; w += GT) {
                uint32_t full = 0;
                int lo = w * 32;
                if (lo < n0) full = (n0 - lo >= 32) ? 0xffffffffu : ((1u << (n0 - lo)) - 1u);
                lv0[Lvl<WP>::P + w] = full;
                lv0[Lvl<WP>::XP + w] = 0u;
            }
            if (g.gl == 0) {
                lv0[Lvl<WP>::LPX] = (uint32_t)nx;
                lv0[Lvl<WP>::NPEND] = 0u;
                uint64_t S = G.mixid[r];
                lv0[Lvl<WP>::SLO] = (uint32_t)S;
                lv0[Lvl<WP>::SHI] = (uint32_t)(S >> 32);
            }
        } else {
            // receiver: keep only X_X rows containing all of R' (they are the
            // excluded vertices adjacent to every vertex of R), set P, X_P, S
            const uint32_t *mR = mb + 4, *mP = mb + 4 + WP, *mX = mb + 4 + 2 * WP;
            int keep_n = 0;
            for (int it = 0; it < nx; it += GT) {
                int idx = it + g.gl;
                bool keep = false;
                uint32_t e = 0;
                if (idx < nx) {
                    e = xidx[idx];
                    keep = true;
                    for (int w = 0; w < W; w++) {
                        uint32_t rw = mR[w];
                        if ((xrows[(size_t)e * WP + w] & rw) != rw) { keep = false; break; }
                    }
                }
                int tot;
                int pos = grp_prefix(g, red, keep, &tot);
                if (keep) xidx[keep_n + pos] = e;  // keep_n + pos <= idx: already read
                keep_n += tot;
            }
            uint64_t S = G.mixid[r];
            for (int w = 0; w < W; w++) {
                uint32_t bits = mR[w];
                while (bits) {
                    int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    S += p0mix[w * 32 + b];
                }
            }
            for (int w = g.gl; w < WP; w += GT) {
                lv0[Lvl<WP>::P + w] = mP[w];
                lv0[Lvl<WP>::XP + w] = mX[w];
            }
            if (g.gl == 0) {
                lv0[Lvl<WP>::LPX] = (uint32_t)keep_n;
                lv0[Lvl<WP>::NPEND] = 0u;
                lv0[Lvl<WP>::SLO] = (uint32_t)S;
                lv0[Lvl<WP>::SHI] = (uint32_t)(S >> 32);
                // record the path R' so deeper donations can rebuild it
                int lv = 0;
                for (int w = 0; w < W; w++) {
                    uint32_t bits = mR[w];
                    while (bits) {
                        int b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        stk[(size_t)lv * LS + Lvl<WP>::VSEL] = (uint32_t)(w * 32 + b);
                        lv++;
                    }
                }
            }
        }
        __threadfence_block();
        g.sync();

        // ----------------------------------------------------- DFS (Algorithm 2)
        int l = l0;
        bool enter = true;
        bool timed_out = false;
        while (true) {
            if ((++descents & 1023u) == 0) {
                // group-uniform decision (every thread must leave together)
                if (grp_or(g, red, g.gl == 0 && globaltimer_ns() > deadline)) {
                    timed_out = true;
                    break;
                }
            }
            uint32_t *lv = stk + (size_t)l * LS;
            if (enter) {
                t_nodes++;
                // copy P to cur, build candidate list P u X_P
                for (int w = g.gl; w < WP; w += GT) cur[w] = lv[Lvl<WP>::P + w];
                if (g.warp == 0) {
                    int nc = 0;
                    for (int w = 0; w < W; w++) {
                        uint32_t bits = lv[Lvl<WP>::P + w] | lv[Lvl<WP>::XP + w];
                        if ((bits >> g.lane) & 1u) cand[nc + __popc(bits & ((1u << g.lane) - 1u))] = w * 32 + g.lane;
                        nc += __popc(bits);
                    }
                    if (g.lane == 0) misc[2] = nc;
                }
                g.sync();
                const int nc = misc[2];
                unsigned best = 0;
                for (int j = g.gl; j < nc; j += GT) {
                    const int c = cand[j];
                    const uint32_t *arow = Arow + (size_t)c * WP;
                    int s = 0;
                    if (WP % 4 == 0) {
                        const uint4 *a4 = reinterpret_cast<const uint4 *>(arow);
                        const uint4 *p4 = reinterpret_cast<const uint4 *>(cur);
                        for (int q = 0; q < (W + 3) / 4; q++) {
                            uint4 a = a4[q], p = p4[q];
                            s += __popc(a.x & p.x) + __popc(a.y & p.y) + __popc(a.z & p.z) + __popc(a.w & p.w);
                        }
                    } else {
                        for (int w = 0; w < W; w++) s += __popc(arow[w] & cur[w]);
                    }
                    unsigned key = ((unsigned)s << 16) | (unsigned)(0xffff - c);
                    best = max(best, key);
                }
                best = grp_max(g, red, best);
                const int piv = 0xffff - (int)(best & 0xffffu);
                for (int w = g.gl; w < WP; w += GT)
                    lv[Lvl<WP>::B + w] = cur[w] & ~Arow[(size_t)piv * WP + w];
                __threadfence_block();
                g.sync();
                enter = false;
            }
            // ------------------------------------------- next branch at level l
            if (g.warp == 0) {
                int v = -1;
                for (int w0 = 0; w0 < W; w0 += 32) {
                    int w = w0 + g.lane;
                    uint32_t bits = (w < W) ? lv[Lvl<WP>::B + w] : 0u;
                    unsigned nz = __ballot_sync(0xffffffffu, bits != 0u);
                    if (nz) {
                        int src = __ffs(nz) - 1;
                        uint32_t bw = __shfl_sync(0xffffffffu, bits, src);
                        v = (w0 + src) * 32 + (__ffs(bw) - 1);
                        break;
                    }
                }
                if (g.lane == 0) misc[3] = v;
            }
            g.sync();
            const int v = misc[3];
            g.sync();
            if (v < 0) {
                // all branches done: backtrack
                if (l == l0) break;
                l--;
                continue;
            }
            const int vw = v >> 5;
            const uint32_t vb = 1u << (v & 31);
            // child sets P n N(v), X_P n N(v) (into level l+1), then P -= v, X_P += v
            uint32_t *nv = lv + LS;
            int pc = 0, xa = 0;
            for (int w = g.gl; w < WP; w += GT) {
                uint32_t av = Arow[(size_t)v * WP + w];
                uint32_t cp = lv[Lvl<WP>::P + w] & av;
                uint32_t cx = lv[Lvl<WP>::XP + w] & av;
                nv[Lvl<WP>::P + w] = cp;
                nv[Lvl<WP>::XP + w] = cx;
                pc += __popc(cp);
                xa |= (cx != 0u);
            }
            pc = grp_sum(g, red, pc);
            xa = grp_or(g, red, xa);
            if (g.gl == 0) {
                lv[Lvl<WP>::B + vw] &= ~vb;
                lv[Lvl<WP>::P + vw] &= ~vb;
                lv[Lvl<WP>::XP + vw] |= vb;
                lv[Lvl<WP>::VSEL] = (uint32_t)v;
            }
            __threadfence_block();
            g.sync();
            const int lpx = (int)lv[Lvl<WP>::LPX];
            const uint64_t S = (uint64_t)lv[Lvl<WP>::SLO] | ((uint64_t)lv[Lvl<WP>::SHI] << 32);
            if (pc == 0) {
                // the child is a leaf: R u {v} is maximal iff X_P' and X_X' are empty
                t_nodes++;
                if (!xa) {
                    int found = 0;
                    for (int it = 0; it < lpx && !found; it += GT) {
                        int idx = it + g.gl;
                        int hit = 0;
                        if (idx < lpx) hit = (xrows[(size_t)xidx[idx] * WP + vw] & vb) != 0u;
                        found = grp_or(g, red, hit);
                    }
                    if (!found && g.gl == 0) {
                        const int sz = l + 2;
                        t_cnt++;
                        uint64_t h = mix64(S + p0mix[v] + (uint64_t)sz * kPhi);
                        t_hash += h;
                        hist[sz] += 1ull;
                        acc_maxsz = max(acc_maxsz, sz);
                    }
                }
                continue;
            }
            // ---------------------------------- donation (Sec. III-C)
            if (C.worker_list && pc >= C.donate_min_p) {
                int others_here = 0;
                for (int w = g.gl; w < W; w += GT) others_here |= (lv[Lvl<WP>::B + w] != 0u);
                others_here = grp_or(g, red, others_here);
                const int npend = (int)lv[Lvl<WP>::NPEND];
                if (others_here && npend >= 1) {
                    if (g.gl == 0) {
                        int claimed = -1;
                        if (ld_relaxed(&C.ctl[CTL_IDLE]) > 0) {
                            const int nwords = (ngroups + 31) >> 5;
                            for (int q = 0; q < nwords && claimed < 0; q++) {
                                int wi = (gg / 32 + 1 + q) % nwords;
                                unsigned bits = *((volatile unsigned *)&C.idle_bits[wi]);
                                while (bits) {
                                    int b = __ffs(bits) - 1;
                                    unsigned old = atomicAnd(&C.idle_bits[wi], ~(1u << b));
                                    if (old & (1u << b)) {
                                        claimed = wi * 32 + b;
                                        break;
                                    }
                                    bits &= bits - 1;
                                }
                            }
                            if (claimed >= 0) {
                                atomicSub(&C.ctl[CTL_IDLE], 1);
                                atomicAdd(&C.ctl[CTL_ACTIVE], 1);
                            }
                        }
                        misc[4] = claimed;
                    }
                    g.sync();
                    const int recv = misc[4];
                    g.sync();
                    if (recv >= 0) {
                        uint32_t *m = C.mail + (size_t)recv * C.mail_words;
                        // R' = path below the root at levels [0, l) plus v
                        for (int w = g.gl; w < WP; w += GT) {
                            m[4 + w] = 0u;
                            m[4 + WP + w] = nv[Lvl<WP>::P + w];
                            m[4 + 2 * WP + w] = nv[Lvl<WP>::XP + w];
                        }
                        g.sync();
                        if (g.gl == 0) {
                            for (int q = 0; q < l; q++) {
                                int u = (int)stk[(size_t)q * LS + Lvl<WP>::VSEL];
                                m[4 + (u >> 5)] |= 1u << (u & 31);
                            }
                            m[4 + vw] |= vb;
                            m[0] = (uint32_t)r;
                            m[1] = (uint32_t)(l + 1);
                            __threadfence();
                            st_release(&C.mail_flag[recv], 1);
                            acc_don++;
                        }
                        g.sync();
                        continue;
                    }
                }
            }
            // ---------------------------------- descend: partition X_X by v
            {
                int out = 0, nout = 0;
                for (int it = 0; it < lpx; it += GT) {
                    int idx = it + g.gl;
                    bool valid = idx < lpx;
                    uint32_t e = valid ? xidx[idx] : 0u;
                    bool surv = valid && (xrows[(size_t)e * WP + vw] & vb) != 0u;
                    int ts, tn;
                    int ps = grp_prefix(g, red, surv, &ts);
                    int pn = grp_prefix(g, red, valid && !surv, &tn);
                    if (surv) xidx[out + ps] = e;
                    else if (valid) xscr[nout + pn] = e;
                    out += ts;
                    nout += tn;
                }
                __threadfence_block();
                g.sync();
                for (int j = g.gl; j < nout; j += GT) xidx[out + j] = xscr[j];
                if (g.gl == 0) {
                    nv[Lvl<WP>::LPX] = (uint32_t)out;
                    int others = 0;
                    for (int w = 0; w < W; w++) others |= (lv[Lvl<WP>::B + w] != 0u);
                    nv[Lvl<WP>::NPEND] = lv[Lvl<WP>::NPEND] + (others ? 1u : 0u);
                    uint64_t S2 = S + p0mix[v];
                    nv[Lvl<WP>::SLO] = (uint32_t)S2;
                    nv[Lvl<WP>::SHI] = (uint32_t)(S2 >> 32);
                }
                __threadfence_block();
                g.sync();
            }
            l++;
            enter = true;
            if (l > rows_cap) {
                if (g.gl == 0) atomicOr(O.status, ST_OVERFLOW);
                break;
            }
        }
        if (timed_out && g.gl == 0) atomicOr(O.status, ST_TIMEOUT);
        g.sync();
        if (ld_relaxed(O.status) & (ST_TIMEOUT | ST_OVERFLOW)) break;
        // ------------------------------------------------------- task done
        if (g.gl == 0) {
            acc_nodes += t_nodes;
            acc_cnt += t_cnt;
            acc_hash += t_hash;
            const int id = G.order[r];
            if (O.root_nodes) atomicAdd(&O.root_nodes[id], t_nodes);
            if (O.root_count && t_cnt) atomicAdd(&O.root_count[id], t_cnt);
            if (O.root_hash && t_hash) atomicAdd(&O.root_hash[id], t_hash);
        }
        g.sync();
    }
    // kernel end: flush
    flush();
    if (g.gl == 0) {
        if (acc_nodes) atomicAdd(O.nodes, acc_nodes);
        if (acc_don) atomicAdd(O.donations, acc_don);
        if (acc_maxsz) atomicMax(O.max_size, acc_maxsz);
    }
}

}  // namespace mce
