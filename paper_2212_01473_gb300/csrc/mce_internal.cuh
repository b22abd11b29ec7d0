// Internal declarations of the GB300 maximal clique enumeration engine.
// Not part of the C ABI (include/mce.h); shared by the engine's .cu files only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mce.h"

namespace mce {

// Device status word values (a kernel never traps: it records and returns).
enum : int {
    ST_OK = 0,
    ST_TIMEOUT = 1,   // a bounded wait gave up
    ST_OVERFLOW = 2,  // an internal capacity was exceeded (engine bug guard)
    ST_BADGRAPH = 4,  // validation failed
    ST_BUDGET = 8,    // the run's time budget (opts.run_budget_ms) ran out
};

// Golden-ratio increment of the clique hash (h(C) in mce.h).
constexpr uint64_t kPhi = 0x9E3779B97F4A7C15ull;

// SplitMix64 output finaliser, restated here for the device (see mce.h).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire_u(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// First index of a sorted a[0, n) with a[idx] >= key[u], for U keys at once.
// The steps depend on n only (the range halves whatever the comparison), so
// the U searches advance in lock step and their loads overlap.
template <int U>
__device__ __forceinline__ void lower_bounds(const int32_t *a, int n, const int32_t (&key)[U], int (&pos)[U]) {
#pragma unroll
    for (int u = 0; u < U; u++) pos[u] = 0;
    if (n == 0) return;
    int len = n;
    while (len > 1) {
        const int half = len >> 1;
#pragma unroll
        for (int u = 0; u < U; u++) pos[u] = a[pos[u] + half] < key[u] ? pos[u] + half : pos[u];
        len -= half;
    }
#pragma unroll
    for (int u = 0; u < U; u++) pos[u] += a[pos[u]] < key[u] ? 1 : 0;
}

// One warp walks 32 sorted lists of ranks at once, lane l's list being
// col[jb_l, jb_l + cnt_l). The lists are laid end to end and dealt out at
// stride 32, U entries per lane in flight, so a long list no longer holds up
// the other lanes. Each entry is looked up in P0 (shared memory, n0 sorted
// ranks) and hit(l, k) runs for an entry of lane l's list found at index k.
template <int U, class F>
__device__ __forceinline__ void warp_walk_lists(const int32_t *col, int jb, int cnt, int lane, const int32_t *p0,
                                                int n0, F hit) {
    constexpr unsigned FULL = 0xffffffffu;
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const int tot = __shfl_sync(FULL, inc, 31);
    const int exc = inc - cnt;  // where lane l's list starts in the joined range
    for (int e0 = 0; e0 < tot; e0 += 32 * U) {
        int ow[U], j[U];
        int32_t w[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int e = min(e0 + u * 32 + lane, tot - 1);
            // the list holding e: the last lane whose start is <= e
            int l = 0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const int st = __shfl_sync(FULL, exc, l + s);
                if (st <= e) l += s;
            }
            ow[u] = l;
            j[u] = __shfl_sync(FULL, jb, l) + (e - __shfl_sync(FULL, exc, l));
        }
#pragma unroll
        for (int u = 0; u < U; u++) w[u] = col[j[u]];
        int k[U];
        lower_bounds<U>(p0, n0, w, k);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (e0 + u * 32 + lane < tot && k[u] < n0 && p0[k[u]] == w[u]) hit(ow[u], k[u]);
    }
}

// The worker-list wait of an idle group (one thread). It returns 1 when a
// donated subtree arrived (*flag was set; it is cleared), 0 when the launch
// is over (no active group left), and -1 when it gave up. It gives up with
// ST_TIMEOUT once timeout_ns have passed since the later of its own start and
// the last heartbeat a busy group posted in *beat (globaltimer ns), so a wait
// ends only when nothing has moved for that long; it gives up with ST_BUDGET
// past budget_end, and at once when another group has set either bit.
__device__ inline int idle_wait(int *flag, const int *active, int *status, const unsigned long long *beat,
                                uint64_t timeout_ns, uint64_t budget_end) {
    const uint64_t w0 = globaltimer_ns();
    unsigned ns = 64;
    for (unsigned spin = 1;; spin++) {
        if (ld_acquire(flag)) {
            *flag = 0;
            return 1;
        }
        // the shared termination word and the clock are read less often
        if ((spin & 7u) == 0) {
            if (ld_acquire(active) == 0) return 0;
            if (ld_relaxed(status) & (ST_TIMEOUT | ST_BUDGET)) return -1;
            const uint64_t now = globaltimer_ns();
            const uint64_t hb = ld_relaxed_u64(beat);
            const uint64_t since = hb > w0 ? hb : w0;
            if (now > since && now - since > timeout_ns) {
                atomicOr(status, ST_TIMEOUT);
                return -1;
            }
            if (now > budget_end) {
                atomicOr(status, ST_BUDGET);
                return -1;
            }
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
}

// Grid-wide barrier for a cooperatively launched (all blocks co-resident)
// kernel. The arrival count only grows: every block keeps the same running
// target (the count at which the barrier before this one completed) and the
// same generation, so a barrier is one release-ordered atomic add per block,
// and the block that brings the count to target + nblk publishes the next
// generation; the others poll it. Each wait is bounded: a block that has
// waited timeout_ns since it arrived (globaltimer ns) sets ST_TIMEOUT in the
// status word, and the barrier returns false in every block that sees it, so
// the kernel can return instead of hanging. Work between barriers is never
// timed. GridBar must start at zero, with target = gen = 0 in every block.
struct GridBar {
    unsigned count;
    unsigned gen;
};

// nblk: the number of blocks taking part (gridDim.x, or fewer once the others
// have returned for good); target and gen are the block's running copies.
__device__ __forceinline__ bool grid_barrier(GridBar *bar, int *status, uint64_t timeout_ns, unsigned nblk,
                                             unsigned &target, unsigned &gen) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned old;
        // acquire-release: this block's writes (ordered before it by the block
        // barrier) are released with the arrival, and the last arrival acquires
        // every earlier one before it releases the next generation
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&bar->count) : "memory");
        if (old == target + nblk - 1) {
            st_release_u(&bar->gen, gen + 1);
        } else {
            // poll the generation word back to back; the status word and the
            // clock are read every 64 polls, and long waits back off. The
            // global timer is not guaranteed to be monotonic: a reading below
            // the start restarts the measurement instead of wrapping the
            // unsigned difference into a false give-up.
            uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire_u(&bar->gen) == gen) {
                if ((++spins & 63u) == 0) {
                    if (ld_relaxed(status) & ST_TIMEOUT) { ok = 0; break; }
                    const uint64_t now = globaltimer_ns();
                    if (now < t0) {
                        t0 = now;
                    } else if (now - t0 > timeout_ns) {
                        atomicOr(status, ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    if (spins > 4096) __nanosleep(256);
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    target += nblk;
    gen += 1;
    return s_ok != 0;
}

// Record a message for mce_last_error() on this thread; returns code.
int set_last_error(int code, const char *msg);

// Kernel launches made by this host thread (reported by mce_get_stats).
inline uint64_t &launch_counter() {
    static thread_local uint64_t c = 0;
    return c;
}
inline void count_launch() { launch_counter()++; }

// ----------------------------------------------------------------- handles

// Everything the traversal needs about the oriented graph (device pointers).
struct DevGraph {
    int32_t n;
    int32_t G;             // number of graphs (1 unless batched)
    const int32_t *out_ptr;   // [n+1] later neighbours of rank r: out_col[out_ptr[r]..)
    const int32_t *out_col;   // ranks, ascending within a row
    const int32_t *in_ptr;    // [n+1] earlier neighbours
    const int32_t *in_col;    // ranks (any order)
    const int32_t *order;     // rank -> input id
    const uint64_t *mixid;    // rank -> mix64(input id + 1)
    const int32_t *gid;       // rank -> graph index (NULL when G == 1)
};

// Phases of the optional per-group cycle counters (mce_stats.phase_*).
enum Phase : int {
    PH_SETUP = 0,      // induced subgraph + X_X rows (+ receiver filter); count = tasks
    PH_PIVOT = 1,      // candidate list + pivot scan; count = candidates scored
    PH_BRANCH = 2,     // next branch + child sets; count = tree nodes
    PH_LEAF = 3,       // maximality test of leaf children; count = X_X rows tested
    PH_PARTITION = 4,  // X_X partition on descent; count = X_X rows moved
    PH_DONATE = 5,     // worker-list checks and donations; count = donations
    PH_IDLE = 6,       // waiting in the worker list; count = subtrees received
    PH_POP = 7,        // reloading the parent level on backtrack; count = backtracks
    PH_CENTRY = 8,     // entering a compact subtree from a wide node; count = X_X rows re-encoded
    kNumPhases = 9
};

// Per-launch traversal outputs (device pointers).
struct DevOut {
    unsigned long long *count;   // [G]
    unsigned long long *hash;    // [G]
    unsigned long long *hist;    // [G * hist_len]
    int32_t hist_len;
    unsigned long long *nodes;   // [1] total tree nodes
    unsigned long long *donations;  // [1]
    int *max_size;               // [1] (atomicMax)
    unsigned long long *root_count; // optional [n] by input id
    unsigned long long *root_hash;
    unsigned long long *root_nodes;
    int *status;
    unsigned long long *phase_cycles;  // [kNumPhases]
    unsigned long long *phase_counts;  // [kNumPhases]
    int32_t *list;                     // optional clique records [k, id_1 .. id_k]
    unsigned long long list_cap;       // words of list
    unsigned long long *list_used;     // [1] words the complete list needs
    unsigned long long *t0;            // [1] globaltimer at the run's first launch (set by k_init_ctl)
};

// Host-side launch of one width class of the traversal (mce_traverse*.cu).
struct ClassLaunch {
    int wp;            // padded 32-bit words per bitset row
    int gw;            // warps per cooperating group
    int blocks;        // persistent blocks
    int warps_per_block;
    size_t smem;       // dynamic shared memory per block
    bool a_global;     // A rows live in the global arena (too wide for smem)
};

struct ClassArgs {
    const int32_t *roots;   // roots of this class, in processing order
    int32_t n_roots;
    int32_t rows_cap;       // max |P0| in this class (rows of A)
    int32_t x_cap;          // max |X0| over this class's roots
    int32_t pivot_ipx;      // 1: pivot candidates include X_X
    int32_t worker_list;
    int32_t donate_min_p;
    int32_t donate_policy;  // MCE_DONATE_*
    int32_t root_chunk;     // roots claimed per atomic
    int32_t level2;         // 1: one task per edge (Algorithm 4), decoded through eoff
    const int32_t *eoff;    // level2: [n_roots + 1] exclusive prefix of the roots' |P0|
    int64_t n_tasks;        // roots, or edges when level2
    int32_t stats;          // 1: collect per-phase cycle counters
    uint64_t timeout_ns;    // bound of each wait (see idle_wait)
    uint64_t budget_ns;     // run time budget from *DevOut::t0; 0 = none
    // scratch (device), sized by the host for groups = blocks * warps_per_block / gw
    uint32_t *arena;        // per-group: stack, X rows, X index lists, (A if a_global)
    size_t arena_words_per_group;
    int *ctl;               // [8]: root counter, active, idle_count, ...
    unsigned *idle_bits;    // [ceil(groups/32)]
    int *mail_flag;         // [groups * kMailFlagStride]
    uint32_t *mail;         // [groups * mail_words]
    int32_t mail_words;
};

// Control words of a traversal launch, each on its own 128-byte line so that
// polling one does not slow atomics on another. CTL_BEAT holds a 64-bit
// heartbeat (globaltimer ns) that busy groups post for the idle wait.
enum CtlSlot { CTL_NEXT_ROOT = 0, CTL_ACTIVE = 32, CTL_IDLE = 64, CTL_BEAT = 96, CTL_NCTL = 128 };
constexpr int kMailFlagStride = 8;  // ints between two groups' mail flags (32 bytes)

// Width classes: padded words per row. A row stride w with w/4 odd keeps
// 128-bit shared loads of 8 consecutive lanes (one phase) on distinct banks.
constexpr int kNumClasses = 9;
__host__ __device__ constexpr int class_wp(int c) {
    return c == 0 ? 1 : c == 1 ? 2 : c == 2 ? 4 : c == 3 ? 12 : c == 4 ? 20 : c == 5 ? 28
         : c == 6 ? 36 : c == 7 ? 68 : 132;
}
// class of a root with |P0| = n0 >= 1
__host__ __device__ inline int class_of(int n0) {
    int w = (n0 + 31) >> 5;
    for (int c = 0; c < kNumClasses; c++)
        if (w <= class_wp(c)) return c;
    return -1;
}

}  // namespace mce
