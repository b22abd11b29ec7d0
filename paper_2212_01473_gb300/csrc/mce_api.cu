// C ABI of the engine (include/mce.h): handle creation (validation, peel,
// orientation, width classes), runs (persistent traversal launches per width
// class) and results.
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mce_learn.cuh"
#include "mce_prep.cuh"
#include "mce_trav_inst.cuh"

namespace mce {
#define MCE_EXTERN_WP(WP)                                                                             \
    extern template cudaError_t plan_wp<WP>(int, int, int, int, int, bool, ClassLaunch *);                  \
    extern template cudaError_t launch_wp<WP>(const ClassLaunch &, const DevGraph &, const DevOut &,  \
                                              const ClassArgs &, int, cudaStream_t);
MCE_EXTERN_WP(1)
MCE_EXTERN_WP(2)
MCE_EXTERN_WP(4)
MCE_EXTERN_WP(12)
MCE_EXTERN_WP(20)
MCE_EXTERN_WP(28)
MCE_EXTERN_WP(36)
MCE_EXTERN_WP(68)
MCE_EXTERN_WP(132)

static cudaError_t plan_class_wp(int wp, int rows, int sms, int smem, int req, int warps, bool bh, ClassLaunch *L) {
    switch (wp) {
        case 1: return plan_wp<1>(rows, sms, smem, req, warps, bh, L);
        case 2: return plan_wp<2>(rows, sms, smem, req, warps, bh, L);
        case 4: return plan_wp<4>(rows, sms, smem, req, warps, bh, L);
        case 12: return plan_wp<12>(rows, sms, smem, req, warps, bh, L);
        case 20: return plan_wp<20>(rows, sms, smem, req, warps, bh, L);
        case 28: return plan_wp<28>(rows, sms, smem, req, warps, bh, L);
        case 36: return plan_wp<36>(rows, sms, smem, req, warps, bh, L);
        case 68: return plan_wp<68>(rows, sms, smem, req, warps, bh, L);
        case 132: return plan_wp<132>(rows, sms, smem, req, warps, bh, L);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t launch_class_wp(const ClassLaunch &L, const DevGraph &g, const DevOut &o,
                                   const ClassArgs &a, int rows, cudaStream_t s) {
    switch (L.wp) {
        case 1: return launch_wp<1>(L, g, o, a, rows, s);
        case 2: return launch_wp<2>(L, g, o, a, rows, s);
        case 4: return launch_wp<4>(L, g, o, a, rows, s);
        case 12: return launch_wp<12>(L, g, o, a, rows, s);
        case 20: return launch_wp<20>(L, g, o, a, rows, s);
        case 28: return launch_wp<28>(L, g, o, a, rows, s);
        case 36: return launch_wp<36>(L, g, o, a, rows, s);
        case 68: return launch_wp<68>(L, g, o, a, rows, s);
        case 132: return launch_wp<132>(L, g, o, a, rows, s);
    }
    return cudaErrorInvalidValue;
}

// Roots with no later neighbours (|P0| = 0): the subtree is the root call
// alone; {r} is a maximal clique iff r has no earlier neighbour either.
// At level 2 (one subtree per edge) these vertices have no subtree and add no
// tree node; an isolated one is still a maximal clique.
__global__ void k_trivial_roots(DevGraph G, DevOut O, const int32_t *roots, int n_roots, int level2) {
    unsigned long long cnt = 0, hsh = 0;
    const int lane = threadIdx.x & 31;
    const int64_t lim = ((int64_t)n_roots + 31) / 32 * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lim;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool clique = false;
        int r = 0;
        if (i < n_roots) {
            r = roots[i];
            clique = G.in_ptr[r + 1] == G.in_ptr[r];
            const int id = G.order[r];
            uint64_t h = clique ? mix64(G.mixid[r] + kPhi) : 0ull;
            if (O.root_nodes && !level2) O.root_nodes[id] += 1ull;
            if (clique && O.root_count) O.root_count[id] += 1ull;
            if (clique && O.root_hash) O.root_hash[id] += h;
            if (clique && O.list) {
                // record [1, id]; the cursor counts it even when it does not fit
                const unsigned long long pos = atomicAdd(O.list_used, 2ull);
                if (pos + 2ull <= O.list_cap) {
                    O.list[pos] = 1;
                    O.list[pos + 1] = id;
                }
            }
            if (G.gid) {
                if (clique) {
                    const int gid = G.gid[r];
                    atomicAdd(&O.count[gid], 1ull);
                    atomicAdd(&O.hash[gid], (unsigned long long)h);
                    if (O.hist_len > 1) atomicAdd(&O.hist[(size_t)gid * O.hist_len + 1], 1ull);
                }
            } else if (clique) {
                cnt += 1;
                hsh += h;
            }
        }
        if (__any_sync(0xffffffffu, clique) && lane == 0) atomicMax(O.max_size, 1);
    }
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        hsh += __shfl_xor_sync(0xffffffffu, hsh, o);
    }
    if (lane == 0 && cnt) {
        atomicAdd(&O.count[0], cnt);
        atomicAdd(&O.hash[0], hsh);
        if (O.hist_len > 1) atomicAdd(&O.hist[1], cnt);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !level2) atomicAdd(O.nodes, (unsigned long long)n_roots);
}

__global__ void k_last_core(const int32_t *order, const int32_t *core, int n, int *out) {
    out[0] = n > 0 ? core[order[n - 1]] : 0;
}

__global__ void k_max_deg(const int32_t *outdeg, const int32_t *indeg, int n, int *out) {
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, outdeg[i] + indeg[i]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// every edge must stay inside its graph's vertex range
__global__ void k_check_batch(int n, const int32_t *rp, const int32_t *col, const int32_t *gptr, int G,
                              int *status) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (gptr[mid] <= v) lo = mid; else hi = mid;
        }
        const int a = gptr[lo], b = gptr[lo + 1];
        for (int j = rp[v]; j < rp[v + 1]; j++)
            if (col[j] < a || col[j] >= b) { atomicOr(status, ST_BADGRAPH); break; }
    }
}

}  // namespace mce

using namespace mce;

static thread_local std::string g_err = "ok";

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int mce::set_last_error(int code, const char *msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess) {                                                             \
            rc = fail(MCE_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e),     \
                      __FILE__, __LINE__);                                                   \
            goto cleanup;                                                                    \
        }                                                                                    \
    } while (0)

// Launch settings of one width class chosen by mce_autotune (0 / -1 = default).
struct Tuned {
    int dmp = 0;
    int policy = -1;
    int blocks = 0;
    int warps = 0;  // warps per block (0 = 16)
};

// One-warp width classes whose row width is at most this share one launch
// (default 12: all of them; 4: rows of 1-4 words share one, 12-word rows run
// alone; 1: every class alone).
constexpr int kMergeDefault = 12;

struct RunPlan;
static void free_plan(mce_graph *g, RunPlan *P);

struct mce_graph {
    int32_t n = 0;
    int64_t m = 0;
    int32_t G = 1;
    int32_t d = 0, max_deg = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mce_allocator alloc{};
    bool has_alloc = false;
    int sm_count = 0, smem_optin = 0;
    int32_t *out_ptr = nullptr, *out_col = nullptr, *in_ptr = nullptr, *in_col = nullptr;
    int32_t *order = nullptr, *rank = nullptr, *core = nullptr, *outdeg = nullptr, *gid = nullptr;
    uint64_t *mixid = nullptr;
    int32_t *class_roots[kNumClasses + 1] = {};
    int32_t class_count[kNumClasses + 1] = {};
    int32_t class_rows[kNumClasses + 1] = {};
    int32_t class_x[kNumClasses + 1] = {};
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    double ms_prep = 0;
    int64_t peel_rounds = 0;
    double peel_stage_ms[3] = {0, 0, 0};
    int32_t peel_stage_rounds[3] = {0, 0, 0};
    int32_t peel_cluster = 0;  // the narrow stage ran as a cluster
    uint64_t create_launches = 0;  // kernels launched by create
    mce_stats last{};              // facts of the last run
    Tuned tuned[kNumClasses];      // per width class, from mce_autotune
    int tuned_merge = kMergeDefault;  // merged one-warp launch width, from mce_autotune
    bool tuned_valid = false;
    struct RunPlan *prepared = nullptr;  // mce_prepare
    cudaGraphExec_t prepared_exec = nullptr;
};

static void *dalloc(mce_graph *g, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g->has_alloc) {
        p = g->alloc.alloc(bytes, g->alloc.ctx);
    } else if (cudaMallocAsync(&p, bytes, g->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void dfree(mce_graph *g, void *p) {
    if (!p) return;
    if (g->has_alloc) g->alloc.free(p, g->alloc.ctx);
    else cudaFreeAsync(p, g->stream);
}

template <typename T>
static T *dnew(mce_graph *g, size_t count, std::vector<void *> *track) {
    T *p = (T *)dalloc(g, count * sizeof(T));
    if (p && track) track->push_back(p);
    return p;
}

static void release_prepared(mce_graph *g);

static void release(mce_graph *g) {
    // nothing of this handle may still run when its memory goes back to the
    // allocator, which can hand it out at once to work on another stream
    if (g->stream) cudaStreamSynchronize(g->stream);
    release_prepared(g);
    void *ps[] = {g->out_ptr, g->out_col, g->in_ptr, g->in_col, g->order, g->rank,
                  g->core,    g->outdeg,  g->gid,    g->mixid,  g->scratch};
    for (void *p : ps) dfree(g, p);
    for (int c = 0; c <= kNumClasses; c++) dfree(g, g->class_roots[c]);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

extern "C" void mce_default_opts(mce_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->struct_size = (int32_t)sizeof(mce_opts);
    o->pivot = MCE_PIVOT_AUTO;
    o->order = MCE_ORDER_PLAIN;
    o->worker_list = 1;
    o->donate_min_p = 0;
    o->donate_policy = MCE_DONATE_EITHER;
    o->timeout_ms = 60000;
    o->run_budget_ms = 600000;
}

extern "C" const char *mce_last_error(void) { return g_err.c_str(); }

static int create_impl(const int32_t *graph_ptr_in, int32_t G, const int32_t *row_ptr, const int32_t *col,
                       int32_t n, int64_t m, uint32_t flags, const mce_allocator *alloc, void *stream,
                       mce_graph **out) {
    if (!out) return fail(MCE_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0 || m < 0 || 2 * m > INT32_MAX) return fail(MCE_EINVAL, "bad sizes n=%d m=%lld", n, (long long)m);
    if (n > 0 && !row_ptr) return fail(MCE_EINVAL, "row_ptr is NULL");
    if (m > 0 && !col) return fail(MCE_EINVAL, "col is NULL");
    if (G < 1) return fail(MCE_EINVAL, "G must be >= 1");
    if (G > 1 && !graph_ptr_in) return fail(MCE_EINVAL, "graph_ptr is NULL");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(MCE_EINVAL, "allocator without alloc/free");
    const bool dev_in = (flags & MCE_FLAG_DEVICE_PTRS) != 0;

    mce_graph *g = new mce_graph();
    g->n = n;
    g->m = m;
    g->G = G;
    int rc = MCE_OK;
    std::vector<void *> tmp;  // freed at the end of create
    int *status = nullptr;
    int h_status = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const int32_t *d_rp = row_ptr, *d_col = col, *d_gptr = nullptr;
    std::vector<int32_t> h_gptr;
    int dev = 0;
    uint64_t launch_base = launch_counter();
    if (alloc) {
        g->alloc = *alloc;
        g->has_alloc = true;
    }
    if (stream) {
        g->stream = (cudaStream_t)stream;
    } else {
        // blocking: ordered with the legacy default stream, whose pending work
        // may still touch memory the caller's allocator hands to this handle
        CK(cudaStreamCreateWithFlags(&g->stream, cudaStreamDefault));
        g->own_stream = true;
    }
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&g->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));

    // graph ranges (batched)
    if (G > 1 || graph_ptr_in) {
        h_gptr.resize((size_t)G + 1);
        if (dev_in) CK(cudaMemcpyAsync(h_gptr.data(), graph_ptr_in, ((size_t)G + 1) * 4, cudaMemcpyDeviceToHost, g->stream));
        else memcpy(h_gptr.data(), graph_ptr_in, ((size_t)G + 1) * 4);
        CK(cudaStreamSynchronize(g->stream));
        if (h_gptr[0] != 0 || h_gptr[G] != n) { rc = fail(MCE_EINVAL, "graph_ptr must start at 0 and end at n"); goto cleanup; }
        for (int i = 0; i < G; i++)
            if (h_gptr[i] > h_gptr[i + 1]) { rc = fail(MCE_EINVAL, "graph_ptr not non-decreasing"); goto cleanup; }
    }
    CK(cudaEventRecord(ev0, g->stream));
    launch_base = launch_counter();
    if (!dev_in) {
        int32_t *a = dnew<int32_t>(g, (size_t)n + 1, &tmp);
        int32_t *b = dnew<int32_t>(g, (size_t)2 * m + 1, &tmp);
        if (!a || !b) { rc = fail(MCE_ENOMEM, "device allocation of the input CSR failed"); goto cleanup; }
        CK(cudaMemcpyAsync(a, row_ptr, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, g->stream));
        if (m > 0) CK(cudaMemcpyAsync(b, col, (size_t)2 * m * 4, cudaMemcpyHostToDevice, g->stream));
        d_rp = a;
        d_col = b;
    }
    status = dnew<int>(g, 4, &tmp);
    if (!status) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
    CK(cudaMemsetAsync(status, 0, 16, g->stream));
    if (n == 0) {
        if (dev_in) {
            int32_t v0 = 0;
            CK(cudaMemcpyAsync(&v0, row_ptr, 4, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            if (v0 != 0 || m != 0) { rc = fail(MCE_EINVAL, "row_ptr[0] must be 0 and m 0 for n = 0"); goto cleanup; }
        } else if (row_ptr && (row_ptr[0] != 0 || m != 0)) {
            rc = fail(MCE_EINVAL, "row_ptr[0] must be 0 and m 0 for n = 0");
            goto cleanup;
        }
    }
    // ------------------------------------------------------------- validate
    CK(launch_validate(n, d_rp, d_col, 2 * m, status, g->stream, false));
    CK(cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (h_status) { rc = fail(MCE_EINVAL, "row_ptr is not a valid offset array (row_ptr[0]=0, non-decreasing, row_ptr[n]=2m)"); goto cleanup; }
    CK(launch_validate(n, d_rp, d_col, 2 * m, status, g->stream, true));
    if (!h_gptr.empty() && n > 0) {
        int32_t *gp = dnew<int32_t>(g, (size_t)G + 1, &tmp);
        if (!gp) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        CK(cudaMemcpyAsync(gp, h_gptr.data(), ((size_t)G + 1) * 4, cudaMemcpyHostToDevice, g->stream));
        d_gptr = gp;
        k_check_batch<<<(unsigned)std::min<int64_t>(65536, ((int64_t)n + 255) / 256), 256, 0, g->stream>>>(n, d_rp, d_col, gp, G, status);
        count_launch();
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (h_status) { rc = fail(MCE_EINVAL, "graph is not a canonical simple undirected CSR (rows sorted, symmetric, no self-loops or duplicates%s)", G > 1 ? ", no edge across graphs" : ""); goto cleanup; }

    {
        // --------------------------------------------------------------- peel
        PeelBufs pb{};
        const size_t nn = (size_t)n + 1;
        pb.deg = dnew<int32_t>(g, nn, &tmp);
        g->rank = pb.rank = dnew<int32_t>(g, nn, nullptr);
        g->core = pb.core = dnew<int32_t>(g, nn, nullptr);
        g->order = pb.order = dnew<int32_t>(g, nn, nullptr);
        pb.remA = dnew<int32_t>(g, nn, &tmp);
        pb.remB = dnew<int32_t>(g, nn, &tmp);
        pb.SA = dnew<int32_t>(g, nn, &tmp);
        pb.SB = dnew<int32_t>(g, nn, &tmp);
        pb.bitmap = dnew<unsigned>(g, ((size_t)n + 31) / 32 + 1, &tmp);
        pb.max_blocks = g->sm_count * 2;
        pb.blocksums = dnew<int>(g, (size_t)pb.max_blocks, &tmp);
        pb.ctl = dnew<PeelCtl>(g, 1, &tmp);
        pb.status = status;
        if (!pb.deg || !pb.rank || !pb.core || !pb.order || !pb.remA || !pb.remB || !pb.SA || !pb.SB ||
            !pb.bitmap || !pb.blocksums || !pb.ctl) { rc = fail(MCE_ENOMEM, "device allocation for the peel failed"); goto cleanup; }
        CK(cudaMemsetAsync(pb.bitmap, 0, (((size_t)n + 31) / 32 + 1) * 4, g->stream));
        CK(launch_peel_init(pb.ctl, n, g->stream));
        const auto peel_t0 = std::chrono::steady_clock::now();
        if (n > 0) CK(launch_peel(n, d_rp, d_col, pb, g->sm_count, kPeelWaitNs, g->stream));
        CK(cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, g->stream));
        PeelCtl hctl{};
        CK(cudaMemcpyAsync(&hctl, pb.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (h_status & ST_TIMEOUT) {
            const double peel_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - peel_t0).count();
            rc = fail(MCE_ETIMEOUT,
                      "degeneracy peel timed out: a barrier wait passed %.0f s (status 0x%x, %.1f ms on the host, "
                      "n = %d, narrow stage %s, one-block stage %s)",
                      kPeelWaitNs / 1e9, (unsigned)h_status, peel_ms, n,
                      hctl.t_narrow ? "reached" : "not reached", hctl.t_solo ? "reached" : "not reached");
            goto cleanup;
        }
        if (hctl.next != n) { rc = fail(MCE_ECUDA, "peel ended early (%d of %d ranked)", hctl.next, n); goto cleanup; }
        g->peel_rounds = hctl.rounds;
        {
            // time and sub-rounds of each peel stage (full grid, 16 blocks, one block)
            const unsigned long long te = hctl.t_end, tn = hctl.t_narrow ? hctl.t_narrow : te,
                                     ts = hctl.t_solo ? hctl.t_solo : te;
            const int rn = hctl.r_narrow >= 0 ? hctl.r_narrow : hctl.rounds,
                      rs = hctl.r_solo >= 0 ? hctl.r_solo : hctl.rounds;
            g->peel_stage_ms[0] = (double)(std::min(tn, ts) - hctl.t_start) / 1e6;
            g->peel_stage_ms[1] = hctl.t_narrow ? (double)(ts - tn) / 1e6 : 0.0;
            g->peel_stage_ms[2] = hctl.t_solo ? (double)(te - ts) / 1e6 : 0.0;
            g->peel_stage_rounds[0] = std::min(rn, rs);
            g->peel_stage_rounds[1] = hctl.r_narrow >= 0 ? rs - rn : 0;
            g->peel_stage_rounds[2] = hctl.r_solo >= 0 ? hctl.rounds - rs : 0;
            g->peel_cluster = hctl.rs_active ? 1 : 0;
        }

        // -------------------------------------------------------- orientation
        g->outdeg = dnew<int32_t>(g, nn, nullptr);
        int32_t *indeg = dnew<int32_t>(g, nn, &tmp);
        g->out_ptr = dnew<int32_t>(g, nn, nullptr);
        g->in_ptr = dnew<int32_t>(g, nn, nullptr);
        g->out_col = dnew<int32_t>(g, (size_t)m + 1, nullptr);
        g->in_col = dnew<int32_t>(g, (size_t)m + 1, nullptr);
        int32_t *scan_tmp = dnew<int32_t>(g, (size_t)scan_tmp_words(n + 1), &tmp);
        g->mixid = dnew<uint64_t>(g, nn, nullptr);
        if (G > 1) g->gid = dnew<int32_t>(g, nn, nullptr);
        int *small = dnew<int>(g, 64, &tmp);
        int *long_rows = dnew<int>(g, nn + 1, &tmp);
        if (!g->outdeg || !indeg || !g->out_ptr || !g->in_ptr || !g->out_col || !g->in_col || !scan_tmp ||
            !g->mixid || (G > 1 && !g->gid) || !small || !long_rows) { rc = fail(MCE_ENOMEM, "device allocation for orientation failed"); goto cleanup; }
        CK(launch_orient(n, d_rp, d_col, g->order, g->rank, g->outdeg, indeg, g->out_ptr, g->out_col,
                         g->in_ptr, g->in_col, scan_tmp, long_rows, g->stream));
        CK(launch_mix_gid(n, g->order, g->mixid, g->gid, d_gptr, G, g->stream));
        CK(cudaMemsetAsync(small, 0, 64 * 4, g->stream));
        k_last_core<<<1, 1, 0, g->stream>>>(g->order, g->core, n, small);
        count_launch();
        if (n > 0) k_max_deg<<<(unsigned)std::min<int64_t>(4096, ((int64_t)n + 255) / 256), 256, 0, g->stream>>>(g->outdeg, indeg, n, small + 1);
        count_launch();
        CK(cudaGetLastError());
        // width classes: small[8..8+K) rows, [24..) x cap, [40..) counts
        int *cls_rows = small + 8, *cls_x = small + 24, *cls_cnt = small + 40;
        CK(launch_classify(n, g->outdeg, indeg, cls_rows, cls_x, cls_cnt, g->stream));
        int hsmall[64];
        CK(cudaMemcpyAsync(hsmall, small, sizeof hsmall, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        g->d = hsmall[0];
        g->max_deg = hsmall[1];
        if (g->d > MCE_MAX_DEGENERACY) { rc = fail(MCE_EUNSUPPORTED, "degeneracy %d exceeds %d", g->d, MCE_MAX_DEGENERACY); goto cleanup; }
        int32_t *flags = dnew<int32_t>(g, nn, &tmp), *pos = dnew<int32_t>(g, nn + 1, &tmp);
        if (!flags || !pos) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        for (int c = 0; c <= kNumClasses; c++) {
            g->class_rows[c] = hsmall[8 + c];
            g->class_x[c] = hsmall[24 + c];
            g->class_count[c] = hsmall[40 + c];
            if (g->class_count[c] == 0) continue;
            g->class_roots[c] = dnew<int32_t>(g, (size_t)g->class_count[c], nullptr);
            if (!g->class_roots[c]) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
            CK(launch_class_list(n, g->outdeg, c, flags, pos, scan_tmp, g->class_roots[c], g->stream));
        }
    }
    CK(cudaEventRecord(ev1, g->stream));
    CK(cudaEventSynchronize(ev1));
    {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ev0, ev1));
        g->ms_prep = ms;
        g->create_launches = launch_counter() - launch_base;
    }
cleanup:
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : tmp) dfree(g, p);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (rc != MCE_OK) {
        release(g);
        return rc;
    }
    cudaStreamSynchronize(g->stream);
    *out = g;
    return MCE_OK;
}

extern "C" int mce_create(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t m, uint32_t flags,
                          const mce_allocator *alloc, void *stream, mce_graph **out) {
    return create_impl(nullptr, 1, row_ptr, col, n, m, flags, alloc, stream, out);
}

extern "C" int mce_batch_create(const int32_t *graph_ptr, int32_t G, const int32_t *row_ptr, const int32_t *col,
                                int32_t n_total, int64_t m_total, uint32_t flags, const mce_allocator *alloc,
                                void *stream, mce_graph **out) {
    if (!graph_ptr) return fail(MCE_EINVAL, "graph_ptr is NULL");
    return create_impl(graph_ptr, G, row_ptr, col, n_total, m_total, flags, alloc, stream, out);
}

static int grow_scratch(mce_graph *g, size_t bytes) {
    if (bytes <= g->scratch_bytes) return MCE_OK;
    if (g->scratch && g->stream) cudaStreamSynchronize(g->stream);  // the old scratch is no longer in use
    dfree(g, g->scratch);
    g->scratch = nullptr;
    g->scratch_bytes = 0;
    size_t want = bytes + bytes / 8;
    g->scratch = dalloc(g, want);
    if (!g->scratch) return fail(MCE_ENOMEM, "device allocation of %zu bytes of traversal scratch failed", want);
    g->scratch_bytes = want;
    return MCE_OK;
}

// ------------------------------------------------------------------ runs
//
// A run is planned (root lists, launch shapes, scratch, outputs), enqueued
// (device work only: memsets and kernels, so it can be captured into a CUDA
// graph), then collected (results copied back and checked).

// t0: the run's start for its time budget, taken by the first launch of the
// run (the outputs, t0 included, are zeroed when the run is enqueued)
__global__ void k_init_ctl(int *ctl, int groups, unsigned long long *t0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctl[CTL_ACTIVE] = groups;
        if (*t0 == 0ull) *t0 = globaltimer_ns();
    }
}

struct RunPlan {
    mce_opts opts{};
    int G = 1, HL = 2;
    unsigned long long *obuf = nullptr;
    size_t obuf_bytes = 0;
    DevGraph dg{};
    DevOut dout{};
    const int32_t *lists[kNumClasses + 1] = {};
    int32_t counts[kNumClasses + 1] = {};
    struct Cls {
        int c = 0, rows = 0, groups = 0;
        int x_cap = 0, wp_min = 0;  // with merged classes: largest X0, narrowest row width
        ClassLaunch L{};
        ClassArgs a{};
    } cls[kNumClasses];
    int ncls = 0;
    int merged_top = -1, merged_xcap = 0, merged_wp_min = 0;  // one-warp classes sharing one launch
    bool level2 = false;  // one subtree per edge (Algorithm 4)
    unsigned trivial_blocks = 0;
    std::vector<void *> tmp;
    std::vector<cudaEvent_t> ev;  // [0] start, [1] end, then one pair per launch
    uint64_t launch_base = 0;
    uint64_t plan_launches = 0;  // kernels run while planning (subsets, priority order)
    uint64_t run_launches = 0;   // kernels of one enqueued run
    bool replay = false;         // collected after a CUDA graph replay
    bool capturing = false;      // enqueued inside a stream capture
};

// Timing events: inside a capture they must be external record nodes to stay
// in the graph; outside a capture the plain record is the valid form.
static cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

static void free_plan(mce_graph *g, RunPlan *P) {
    if (!P) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
    for (void *q : P->tmp) dfree(g, q);
    dfree(g, P->obuf);
    delete P;
}

// class_mask: bit c set = launch width class c (bit kNumClasses: roots with |P0| = 0)
static int plan_run(mce_graph *g, const mce_opts *opts_in, unsigned class_mask, const Tuned *tune_override,
                    RunPlan **out, int merge_override = 0) {
    *out = nullptr;
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    RunPlan *P = new RunPlan();
    mce_opts &opts = P->opts;
    mce_default_opts(&opts);
    int rc = MCE_OK;
    if (opts_in) {
        if (opts_in->struct_size != (int32_t)sizeof(mce_opts)) { delete P; return fail(MCE_EINVAL, "opts.struct_size mismatch"); }
        opts = *opts_in;
    }
    if (opts.pivot < 0 || opts.pivot > 2) rc = fail(MCE_EINVAL, "bad opts.pivot");
    else if (opts.order != MCE_ORDER_PLAIN && opts.order != MCE_ORDER_PRIORITY) rc = fail(MCE_EINVAL, "bad opts.order");
    else if (opts.order == MCE_ORDER_PRIORITY && !opts.root_priority) rc = fail(MCE_EINVAL, "MCE_ORDER_PRIORITY needs opts.root_priority");
    else if (opts.donate_min_p < 0) rc = fail(MCE_EINVAL, "opts.donate_min_p < 0");
    else if (opts.donate_policy < 0 || opts.donate_policy > 2) rc = fail(MCE_EINVAL, "bad opts.donate_policy");
    else if (opts.roots && opts.n_roots < 0) rc = fail(MCE_EINVAL, "opts.n_roots < 0");
    else if (opts.tuned && !g->tuned_valid) rc = fail(MCE_EINVAL, "opts.tuned set but mce_autotune has not run on this handle");
    else if (opts.subtree_level < 0 || opts.subtree_level > 2) rc = fail(MCE_EINVAL, "bad opts.subtree_level");
    else if (opts.run_budget_ms < 0) rc = fail(MCE_EINVAL, "opts.run_budget_ms < 0");
    else if (opts.merge_wp != 0 && opts.merge_wp != 1 && opts.merge_wp != 4 && opts.merge_wp != 12)
        rc = fail(MCE_EINVAL, "opts.merge_wp must be 0, 1, 4 or 12");
    else if (opts.block_warps != 0 && opts.block_warps != 4 && opts.block_warps != 8 && opts.block_warps != 16 &&
             opts.block_warps != 24)
        rc = fail(MCE_EINVAL, "opts.block_warps must be 0, 4, 8, 16 or 24");
    if (rc != MCE_OK) { delete P; return rc; }
    if (opts.timeout_ms <= 0) opts.timeout_ms = 60000;
    P->level2 = opts.subtree_level == 2;
    const int G = g->G;
    P->G = G;
    P->HL = g->d + 2;  // every maximal clique has at most d + 1 vertices
    P->launch_base = launch_counter();
    // outputs: count[G], hash[G], hist[G*HL], nodes, donations | max_size, status, phase counters
    const size_t out_words64 = (size_t)2 * G + (size_t)G * P->HL + 4 + 2 * kNumPhases + 1;
    P->obuf_bytes = out_words64 * 8 + 64;
    P->obuf = (unsigned long long *)dalloc(g, P->obuf_bytes);
    if (!P->obuf) { free_plan(g, P); return fail(MCE_ENOMEM, "device allocation of outputs failed"); }
    DevGraph &dg = P->dg;
    DevOut &dout = P->dout;
    dg.n = g->n;
    dg.G = G;
    dg.out_ptr = g->out_ptr;
    dg.out_col = g->out_col;
    dg.in_ptr = g->in_ptr;
    dg.in_col = g->in_col;
    dg.order = g->order;
    dg.mixid = g->mixid;
    dg.gid = g->gid;
    dout.count = P->obuf;
    dout.hash = P->obuf + G;
    dout.hist = P->obuf + 2 * G;
    dout.hist_len = P->HL;
    dout.nodes = P->obuf + 2 * G + (size_t)G * P->HL;
    dout.donations = dout.nodes + 1;
    dout.max_size = (int *)(dout.nodes + 2);
    dout.status = dout.max_size + 1;
    dout.phase_cycles = dout.nodes + 4;
    dout.phase_counts = dout.phase_cycles + kNumPhases;
    dout.t0 = dout.phase_counts + kNumPhases;
    dout.root_count = (unsigned long long *)opts.root_count;
    dout.root_hash = (unsigned long long *)opts.root_hash;
    dout.root_nodes = (unsigned long long *)opts.root_nodes;
    for (int c = 0; c <= kNumClasses; c++) {
        const bool on = (class_mask >> c) & 1u;
        P->lists[c] = g->class_roots[c];
        P->counts[c] = on ? g->class_count[c] : 0;
    }
    size_t need_words = 0;
    if (opts.roots && g->n > 0) {
        int maxc = 1;
        for (int c = 0; c <= kNumClasses; c++) maxc = std::max(maxc, g->class_count[c]);
        int32_t *mask = (int32_t *)dalloc(g, (size_t)g->n * 4);
        int32_t *flags = (int32_t *)dalloc(g, (size_t)maxc * 4);
        int32_t *pos = (int32_t *)dalloc(g, ((size_t)maxc + 1) * 4);
        int32_t *stmp = (int32_t *)dalloc(g, (size_t)scan_tmp_words(maxc + 1) * 4);
        for (void *q : {(void *)mask, (void *)flags, (void *)pos, (void *)stmp}) P->tmp.push_back(q);
        if (!mask || !flags || !pos || !stmp) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        CK(cudaMemsetAsync(dout.status, 0, 4, g->stream));
        CK(cudaMemsetAsync(mask, 0, (size_t)g->n * 4, g->stream));
        CK(launch_mark_roots(opts.roots, opts.n_roots, g->rank, g->n, mask, dout.status, g->stream));
        int hst = 0;
        CK(cudaMemcpyAsync(&hst, dout.status, 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (hst) { rc = fail(MCE_EINVAL, "opts.roots holds an id outside [0, n)"); goto cleanup; }
        for (int c = 0; c <= kNumClasses; c++) {
            if (P->counts[c] == 0) continue;
            int32_t *o = (int32_t *)dalloc(g, (size_t)P->counts[c] * 4);
            P->tmp.push_back(o);
            if (!o) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
            CK(launch_subset(P->lists[c], P->counts[c], mask, flags, pos, stmp, o, g->stream));
            int kept = 0;
            CK(cudaMemcpyAsync(&kept, pos + P->counts[c], 4, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            P->lists[c] = o;
            P->counts[c] = kept;
        }
    }
    if (opts.order == MCE_ORDER_PRIORITY && g->n > 0) {
        int *hb = (int *)dalloc(g, 256 * sizeof(int));
        P->tmp.push_back(hb);
        if (!hb) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        int most = 0;
        for (int c = 0; c < kNumClasses; c++) most = std::max(most, (int)P->counts[c]);
        int32_t *pf = (int32_t *)dalloc(g, ((size_t)most + 1) * 4);
        int32_t *pp = (int32_t *)dalloc(g, ((size_t)most + 1) * 4);
        int32_t *pt = (int32_t *)dalloc(g, (size_t)scan_tmp_words((int64_t)most + 1) * 4);
        P->tmp.push_back(pf);
        P->tmp.push_back(pp);
        P->tmp.push_back(pt);
        if (!pf || !pp || !pt) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        for (int c = 0; c < kNumClasses; c++) {
            if (P->counts[c] == 0) continue;
            int32_t *o = (int32_t *)dalloc(g, (size_t)P->counts[c] * 4);
            P->tmp.push_back(o);
            if (!o) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
            CK(launch_priority_order(P->lists[c], P->counts[c], g->order, opts.root_priority, hb, pf, pp, pt, o,
                                     g->stream));
            P->lists[c] = o;
        }
    }
    if (P->counts[kNumClasses] > 0)
        P->trivial_blocks = (unsigned)std::min<int64_t>(4096, ((int64_t)P->counts[kNumClasses] + 255) / 256);
    // The one-warp classes (row width <= 12 words) share one launch of the
    // widest of them, its roots first: the narrow classes' roots fill the
    // groups that would otherwise idle at the end of each separate launch.
    {
        const int merge_wp = merge_override > 0 ? merge_override
                             : opts.merge_wp > 0 ? opts.merge_wp
                             : (opts.tuned ? g->tuned_merge : kMergeDefault);
        int top = -1, nmerge = 0;
        int64_t total = 0;
        for (int c = kNumClasses - 1; c >= 0; c--) {
            if (P->counts[c] == 0 || class_wp(c) > std::min(12, merge_wp)) continue;
            if (top < 0) top = c;
            nmerge++;
            total += P->counts[c];
            P->merged_xcap = std::max(P->merged_xcap, (int)g->class_x[c]);
            P->merged_wp_min = class_wp(c);
        }
        if (nmerge > 1) {
            int32_t *lst = (int32_t *)dalloc(g, (size_t)total * 4);
            P->tmp.push_back(lst);
            if (!lst) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
            int64_t at = 0;
            for (int c = top; c >= 0; c--) {
                if (P->counts[c] == 0 || class_wp(c) > std::min(12, merge_wp)) continue;
                CK(cudaMemcpyAsync(lst + at, P->lists[c], (size_t)P->counts[c] * 4, cudaMemcpyDeviceToDevice, g->stream));
                at += P->counts[c];
                if (c != top) P->counts[c] = 0;
            }
            P->lists[top] = lst;
            P->counts[top] = (int32_t)total;
            P->merged_top = top;
        }
    }
    // width classes, heaviest first: launch shapes, then one scratch for all
    for (int c = kNumClasses - 1; c >= 0; c--) {
        if (P->counts[c] == 0) continue;
        RunPlan::Cls &k = P->cls[P->ncls++];
        const Tuned *t = tune_override ? &tune_override[c] : (opts.tuned ? &g->tuned[c] : nullptr);
        k.c = c;
        k.rows = g->class_rows[c];
        k.x_cap = c == P->merged_top ? P->merged_xcap : g->class_x[c];
        k.wp_min = c == P->merged_top ? P->merged_wp_min : class_wp(c);
        const int blocks = (t && t->blocks > 0) ? t->blocks : opts.blocks;
        const int warps = (t && t->warps > 0) ? t->warps : opts.block_warps;
        CK(plan_class_wp(class_wp(c), k.rows, g->sm_count, g->smem_optin, blocks, warps, g->gid == nullptr, &k.L));
        k.groups = k.L.blocks * (k.L.warps_per_block / k.L.gw);
        const size_t aw = arena_words(k.L.wp, k.rows, k.x_cap, k.L.a_global, stack_in_smem(k.L.wp));
        const size_t idle_words = ((size_t)k.groups + 31) / 32;
        const size_t flag_words = (size_t)k.groups * kMailFlagStride;
        // a wide subtree: root, level, rows, kind, R', P', X_P'; a compact one
        // (one-warp classes): root, level, rows, kind, 32 rows, 32 indices, P, X_P, hash sum
        const int mail_words = std::max(4 + 3 * k.L.wp, 72);
        const size_t words = aw * k.groups + CTL_NCTL + idle_words + flag_words + (size_t)k.groups * mail_words + 64;
        need_words = std::max(need_words, words);
        ClassArgs &a = k.a;
        a.roots = P->lists[c];
        a.n_roots = P->counts[c];
        a.rows_cap = k.rows;
        a.x_cap = k.x_cap;
        // IPX: pivots may also come from X_X; AUTO follows the Sec. IV-E rule
        // (partial induced subgraphs when max degree / degeneracy > 200)
        a.pivot_ipx = opts.pivot == MCE_PIVOT_IPX ||
                      (opts.pivot == MCE_PIVOT_AUTO && g->d > 0 && (double)g->max_deg / g->d <= 200.0);
        a.worker_list = opts.worker_list ? 1 : 0;
        // 0 = automatic: a donated child must have at least 1/10 of the
        // class's widest root set, and never fewer than 10 candidates (Sec. III-C)
        const int dmp = (t && t->dmp > 0) ? t->dmp : opts.donate_min_p;
        a.donate_min_p = dmp > 0 ? dmp : std::max(10, k.rows / 10);
        a.donate_policy = (t && t->policy >= 0) ? t->policy : opts.donate_policy;
        a.root_chunk = 1;
        a.stats = opts.stats ? 1 : 0;
        a.timeout_ns = (uint64_t)opts.timeout_ms * 1000000ull;
        a.budget_ns = (uint64_t)opts.run_budget_ms * 1000000ull;
        a.arena_words_per_group = aw;
        a.mail_words = mail_words;
    }
    if ((rc = grow_scratch(g, need_words * 4)) != MCE_OK) goto cleanup;
    for (int i = 0; i < P->ncls; i++) {
        RunPlan::Cls &k = P->cls[i];
        uint32_t *sw = (uint32_t *)g->scratch;
        const size_t idle_words = ((size_t)k.groups + 31) / 32;
        const size_t flag_words = (size_t)k.groups * kMailFlagStride;
        k.a.arena = sw;
        k.a.ctl = (int *)(sw + k.a.arena_words_per_group * k.groups);
        k.a.idle_bits = (unsigned *)(k.a.ctl + CTL_NCTL);
        k.a.mail_flag = (int *)(k.a.idle_bits + idle_words);
        k.a.mail = (uint32_t *)(k.a.mail_flag + flag_words);
    }
    for (int i = 0; i < P->ncls; i++) {
        RunPlan::Cls &k = P->cls[i];
        k.a.level2 = P->level2 ? 1 : 0;
        k.a.eoff = nullptr;
        k.a.n_tasks = k.a.n_roots;
        if (!P->level2) continue;
        // tasks are the roots' edges to later neighbours: eoff[i] = sum of |P0| before root i
        int32_t *deg = (int32_t *)dalloc(g, ((size_t)k.a.n_roots + 1) * 4);
        int32_t *eo = (int32_t *)dalloc(g, ((size_t)k.a.n_roots + 1) * 4);
        int32_t *stmp = (int32_t *)dalloc(g, (size_t)scan_tmp_words((int64_t)k.a.n_roots + 1) * 4);
        for (void *q : {(void *)deg, (void *)eo, (void *)stmp}) P->tmp.push_back(q);
        if (!deg || !eo || !stmp) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        CK(launch_gather_outdeg(k.a.roots, k.a.n_roots, g->outdeg, deg, g->stream));
        CK(exclusive_scan(deg, eo, k.a.n_roots, stmp, g->stream));
        int32_t tot = 0;
        CK(cudaMemcpyAsync(&tot, eo + k.a.n_roots, 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        k.a.eoff = eo;
        k.a.n_tasks = tot;
    }
    {
        const int nev = 2 + 2 * (P->ncls + (P->trivial_blocks ? 1 : 0));
        for (int i = 0; i < nev; i++) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            P->ev.push_back(e);
        }
    }
    P->plan_launches = launch_counter() - P->launch_base;
    *out = P;
    return MCE_OK;
cleanup:
    free_plan(g, P);
    return rc;
}

// Device work of a planned run; no host synchronisation (capturable).
static int enqueue_run(mce_graph *g, RunPlan *P) {
    int rc = MCE_OK;
    const uint64_t base = launch_counter();
    const mce_opts &opts = P->opts;
    cudaStream_t s = g->stream;
    int e = 2;
    CK(cudaMemsetAsync(P->obuf, 0, P->obuf_bytes, s));
    if (opts.root_count) CK(cudaMemsetAsync(opts.root_count, 0, (size_t)g->n * 8, s));
    if (opts.root_hash) CK(cudaMemsetAsync(opts.root_hash, 0, (size_t)g->n * 8, s));
    if (opts.root_nodes) CK(cudaMemsetAsync(opts.root_nodes, 0, (size_t)g->n * 8, s));
    CK(record(P->ev[0], s, P->capturing));
    if (P->trivial_blocks) {
        CK(record(P->ev[e++], s, P->capturing));
        k_trivial_roots<<<P->trivial_blocks, 256, 0, s>>>(P->dg, P->dout, P->lists[kNumClasses],
                                                          P->counts[kNumClasses], P->level2 ? 1 : 0);
        count_launch();
        CK(cudaGetLastError());
        CK(record(P->ev[e++], s, P->capturing));
    }
    for (int i = 0; i < P->ncls; i++) {
        RunPlan::Cls &k = P->cls[i];
        const size_t idle_words = ((size_t)k.groups + 31) / 32;
        const size_t flag_words = (size_t)k.groups * kMailFlagStride;
        CK(cudaMemsetAsync(k.a.ctl, 0, (CTL_NCTL + idle_words + flag_words) * 4, s));
        k_init_ctl<<<1, 32, 0, s>>>(k.a.ctl, k.groups, P->dout.t0);
        count_launch();
        CK(record(P->ev[e++], s, P->capturing));
        CK(launch_class_wp(k.L, P->dg, P->dout, k.a, k.rows, s));
        count_launch();
        CK(record(P->ev[e++], s, P->capturing));
    }
    CK(record(P->ev[1], s, P->capturing));
    P->run_launches = launch_counter() - base;
cleanup:
    return rc;
}

// Copy results back, check the device status, fill the caller's outputs.
static int collect_run(mce_graph *g, RunPlan *P, mce_result *per_graph, uint64_t *hist, int32_t hist_len,
                       mce_result *total) {
    int rc = MCE_OK;
    const int G = P->G, HL = P->HL;
    const DevOut &dout = P->dout;
    std::vector<unsigned long long> hcnt(G), hhash(G), hhist((size_t)G * HL);
    unsigned long long hmisc[2] = {0, 0};
    int hflags[2] = {0, 0};
    mce_stats st{};
    st.struct_size = (int32_t)sizeof(mce_stats);
    CK(cudaMemcpyAsync(hcnt.data(), dout.count, (size_t)G * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hhash.data(), dout.hash, (size_t)G * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hhist.data(), dout.hist, (size_t)G * HL * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hmisc, dout.nodes, 2 * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hflags, dout.max_size, 2 * 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(st.phase_cycles, dout.phase_cycles, 2 * kNumPhases * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    {
        int e = 2;
        if (P->trivial_blocks) {
            const int k = st.n_classes++;
            float cms = 0;
            CK(cudaEventElapsedTime(&cms, P->ev[e], P->ev[e + 1]));
            e += 2;
            st.class_wp[k] = 0;
            st.class_roots[k] = P->counts[kNumClasses];
            st.class_blocks[k] = (int32_t)P->trivial_blocks;
            st.class_ms[k] = cms;
        }
        for (int i = 0; i < P->ncls; i++) {
            const RunPlan::Cls &c = P->cls[i];
            const int k = st.n_classes++;
            float cms = 0;
            CK(cudaEventElapsedTime(&cms, P->ev[e], P->ev[e + 1]));
            e += 2;
            st.class_wp[k] = c.L.wp;
            st.class_wp_min[k] = c.wp_min;
            st.class_roots[k] = P->counts[c.c];
            st.class_rows[k] = c.rows;
            st.class_blocks[k] = c.L.blocks;
            st.class_groups[k] = c.groups;
            st.class_group_warps[k] = c.L.gw;
            st.class_ms[k] = cms;
        }
    }
    st.kernel_launches = g->create_launches + (P->replay ? 0 : P->plan_launches) + P->run_launches;
    st.peel_rounds = g->peel_rounds;
    for (int i = 0; i < 3; i++) {
        st.peel_stage_ms[i] = g->peel_stage_ms[i];
        st.peel_stage_rounds[i] = g->peel_stage_rounds[i];
    }
    st.peel_cluster = g->peel_cluster;
    g->last = st;
    if (hflags[1] & ST_TIMEOUT) { rc = fail(MCE_ETIMEOUT, "a traversal wait exceeded %lld ms with no progress", (long long)P->opts.timeout_ms); goto cleanup; }
    if (hflags[1] & ST_BUDGET) { rc = fail(MCE_EBUDGET, "the run exceeded its time budget of %lld ms", (long long)P->opts.run_budget_ms); goto cleanup; }
    if (hflags[1] & ST_OVERFLOW) { rc = fail(MCE_ECUDA, "internal capacity exceeded in the traversal"); goto cleanup; }
    {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]));
        mce_result tot{};
        for (int gi = 0; gi < G; gi++) {
            mce_result r{};
            r.count = hcnt[gi];
            r.hash = hhash[gi];
            int mx = 0;
            for (int sz = HL - 1; sz > 0; sz--)
                if (hhist[(size_t)gi * HL + sz]) { mx = sz; break; }
            r.max_size = mx;
            r.degeneracy = g->d;
            r.ms_prep = g->ms_prep;
            r.ms_traverse = ms;
            if (per_graph) per_graph[gi] = r;
            tot.count += r.count;
            tot.hash += r.hash;
            tot.max_size = std::max(tot.max_size, mx);
        }
        tot.degeneracy = g->d;
        tot.tree_nodes = hmisc[0];
        tot.donations = hmisc[1];
        tot.ms_prep = g->ms_prep;
        tot.ms_traverse = ms;
        if (G == 1 && per_graph) {
            per_graph[0].tree_nodes = tot.tree_nodes;
            per_graph[0].donations = tot.donations;
        }
        if (total) *total = tot;
        if (hist && hist_len > 0) {
            for (int gi = 0; gi < G; gi++)
                for (int sz = 0; sz < hist_len; sz++)
                    hist[(size_t)gi * hist_len + sz] = sz < HL ? hhist[(size_t)gi * HL + sz] : 0ull;
        }
        if (hist && hist_len <= tot.max_size) rc = fail(MCE_ERANGE, "hist_len %d <= max clique size %d", hist_len, tot.max_size);
    }
cleanup:
    return rc;
}

constexpr unsigned kAllClasses = (1u << (kNumClasses + 1)) - 1u;

static int run_impl(mce_graph *g, const mce_opts *opts_in, mce_result *per_graph, uint64_t *hist,
                    int32_t hist_len, mce_result *total) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (hist && hist_len < 0) return fail(MCE_EINVAL, "hist_len < 0");
    RunPlan *P = nullptr;
    int rc = plan_run(g, opts_in, kAllClasses, nullptr, &P);
    if (rc != MCE_OK) return rc;
    rc = enqueue_run(g, P);
    if (rc == MCE_OK) rc = collect_run(g, P, per_graph, hist, hist_len, total);
    free_plan(g, P);
    return rc;
}

static void release_prepared(mce_graph *g) {
    if (g->prepared_exec) cudaGraphExecDestroy(g->prepared_exec);
    if (g->prepared) free_plan(g, g->prepared);
    g->prepared = nullptr;
    g->prepared_exec = nullptr;
}

extern "C" int mce_prepare(mce_graph *g, const mce_opts *opts) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    release_prepared(g);
    RunPlan *P = nullptr;
    int rc = plan_run(g, opts, kAllClasses, nullptr, &P);
    if (rc != MCE_OK) return rc;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        free_plan(g, P);
        return fail(MCE_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    P->capturing = true;
    rc = enqueue_run(g, P);
    P->capturing = false;
    e = cudaStreamEndCapture(g->stream, &graph);
    if (rc == MCE_OK && e != cudaSuccess) rc = fail(MCE_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    if (rc == MCE_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        rc = fail(MCE_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    if (graph) cudaGraphDestroy(graph);
    if (rc != MCE_OK) {
        free_plan(g, P);
        return rc;
    }
    g->prepared = P;
    g->prepared_exec = exec;
    return MCE_OK;
}

extern "C" int mce_run_prepared(mce_graph *g, mce_result *per_graph, uint64_t *hist, int32_t hist_len,
                                mce_result *total) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (!g->prepared) return fail(MCE_EINVAL, "no prepared run: call mce_prepare first");
    if (!per_graph && !total) return fail(MCE_EINVAL, "per_graph and total are both NULL");
    if (hist && hist_len < 0) return fail(MCE_EINVAL, "hist_len < 0");
    g->prepared->replay = true;
    cudaError_t e = cudaGraphLaunch(g->prepared_exec, g->stream);
    if (e != cudaSuccess) return fail(MCE_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    return collect_run(g, g->prepared, per_graph, hist, hist_len, total);
}

// Time one run of the classes in `mask` with these settings (device time of
// the traversal launches); a failed run returns a negative time.
static double time_setting(mce_graph *g, const mce_opts *base, unsigned mask, const Tuned *over, int merge_wp,
                           int *rc_out) {
    RunPlan *P = nullptr;
    int rc = plan_run(g, base, mask, over, &P, merge_wp);
    double ms = -1.0;
    if (rc == MCE_OK) {
        rc = enqueue_run(g, P);
        if (rc == MCE_OK) {
            mce_result tot{};
            rc = collect_run(g, P, nullptr, nullptr, 0, &tot);
            if (rc == MCE_OK) ms = tot.ms_traverse;
        }
        free_plan(g, P);
    }
    *rc_out = rc;
    return ms;
}

// The autotuner (config of the batched form: bitset width and block size are
// tuned). (1) Bitset width of the one-warp classes: their roots run in one
// launch at the widest of their row widths, or rows of 1-4 words share a
// 4-word launch and 12-word rows run alone, or each class runs alone at its
// own width; the fastest over all one-warp roots is kept. (2) Then, launch by
// launch, a coordinate search from the defaults over the donation threshold
// (|P0|max / 10, / 20, / 5, never below 10), the donation rule (EITHER,
// PAPER, ANY), the warps per block (24, 16, 8, 4) and the grid (all blocks that
// fit, or one per SM), keeping each change that is faster. Results never
// depend on any of these.
extern "C" int mce_autotune(mce_graph *g, const mce_opts *base, double budget_ms) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    int rc = MCE_OK;
    double spent = 0;
    const double budget = budget_ms > 0 ? budget_ms : 1e300;
    Tuned over[kNumClasses];
    for (int c = 0; c < kNumClasses; c++) g->tuned[c] = Tuned{};
    g->tuned_merge = kMergeDefault;
    unsigned one_warp = 0;
    int n_one = 0;
    for (int c = 0; c < kNumClasses; c++)
        if (g->class_count[c] > 0 && class_wp(c) <= 12) {
            one_warp |= 1u << c;
            n_one++;
        }
    // (1) bitset width of the one-warp launch
    if (n_one > 1) {
        double best = 1e300;
        for (int mw : {12, 4, 1}) {
            const double ms = time_setting(g, base, one_warp, nullptr, mw, &rc);
            if (rc != MCE_OK) return rc;
            spent += ms;
            if (ms < best) {
                best = ms;
                g->tuned_merge = mw;
            }
        }
    }
    // (2) launch by launch: the leading class of each launch and the classes it carries
    for (int c = kNumClasses - 1; c >= 0; c--) {
        if (g->class_count[c] == 0) continue;
        unsigned mask = 1u << c;
        if (class_wp(c) <= 12) {
            const int mw = std::min(12, g->tuned_merge);
            if (class_wp(c) <= mw) {
                // the widest merged class leads the launch; the others ride along
                bool leads = true;
                for (int q = c + 1; q < kNumClasses; q++)
                    if (g->class_count[q] > 0 && class_wp(q) <= mw) leads = false;
                if (!leads) continue;
                for (int q = 0; q < c; q++)
                    if (g->class_count[q] > 0) mask |= 1u << q;
            }
        }
        const int rows = g->class_rows[c];
        const int A = std::max(10, rows / 10);
        Tuned best_t{A, MCE_DONATE_EITHER, 0, 0};
        for (int q = 0; q < kNumClasses; q++) over[q] = Tuned{};
        over[c] = best_t;
        double best = time_setting(g, base, mask, over, g->tuned_merge, &rc);
        if (rc != MCE_OK) return rc;
        spent += best;
        auto attempt = [&](Tuned t) -> int {
            if (spent > budget) return MCE_OK;
            over[c] = t;
            const double ms = time_setting(g, base, mask, over, g->tuned_merge, &rc);
            if (rc != MCE_OK) return rc;
            spent += ms;
            if (ms < best) {
                best = ms;
                best_t = t;
            }
            return MCE_OK;
        };
        for (int d : {std::max(10, rows / 20), std::max(10, rows / 5)}) {
            Tuned t = best_t;
            t.dmp = d;
            if ((rc = attempt(t)) != MCE_OK) return rc;
        }
        for (int pol : {MCE_DONATE_PAPER, MCE_DONATE_ANY}) {
            Tuned t = best_t;
            t.policy = pol;
            if ((rc = attempt(t)) != MCE_OK) return rc;
        }
        for (int w : {16, 8, 4}) {
            Tuned t = best_t;
            t.warps = w;
            if (w >= group_warps(class_wp(c)) && (rc = attempt(t)) != MCE_OK) return rc;
        }
        {
            Tuned t = best_t;
            t.blocks = g->sm_count;
            if ((rc = attempt(t)) != MCE_OK) return rc;
        }
        g->tuned[c] = best_t;
    }
    g->tuned_valid = true;
    return MCE_OK;
}

extern "C" int mce_get_tuning(const mce_graph *g, int32_t *donate_min_p, int32_t *donate_policy, int32_t *blocks,
                              int32_t *warps, int32_t *merge_wp) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (!g->tuned_valid) return fail(MCE_EINVAL, "mce_autotune has not run on this handle");
    for (int c = 0; c < kNumClasses; c++) {
        if (donate_min_p) donate_min_p[c] = g->tuned[c].dmp;
        if (donate_policy) donate_policy[c] = g->tuned[c].policy;
        if (blocks) blocks[c] = g->tuned[c].blocks;
        if (warps) warps[c] = g->tuned[c].warps;
    }
    if (merge_wp) *merge_wp = g->tuned_merge;
    return MCE_OK;
}

extern "C" int mce_run(mce_graph *g, const mce_opts *opts, mce_result *out, uint64_t *hist, int32_t hist_len) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (g->G != 1) return fail(MCE_EINVAL, "batched handle: use mce_run_batch");
    if (!out) return fail(MCE_EINVAL, "out is NULL");
    return run_impl(g, opts, out, hist, hist_len, nullptr);
}

extern "C" int mce_run_list(mce_graph *g, const mce_opts *opts, int32_t *buf, int64_t cap_words, int64_t *words,
                            mce_result *out) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (g->G != 1) return fail(MCE_EINVAL, "batched handle: listing takes one graph");
    if (!out || !words) return fail(MCE_EINVAL, "out or words is NULL");
    if (cap_words < 0) return fail(MCE_EINVAL, "cap_words < 0");
    if (cap_words > 0 && !buf) return fail(MCE_EINVAL, "buf is NULL");
    if (buf) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, buf) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(MCE_EINVAL, "buf must be device memory");
        }
    }
    *words = 0;
    RunPlan *P = nullptr;
    int rc = plan_run(g, opts, kAllClasses, nullptr, &P);
    if (rc != MCE_OK) return rc;
    // the records' cursor sits in the spare words after the run's outputs
    unsigned long long *cursor = P->obuf + (P->obuf_bytes - 64) / 8;
    P->dout.list = buf ? buf : (int32_t *)P->obuf;  // non-null; with cap 0 nothing is written
    P->dout.list_cap = buf ? (unsigned long long)cap_words : 0ull;
    P->dout.list_used = cursor;
    rc = enqueue_run(g, P);
    if (rc == MCE_OK) rc = collect_run(g, P, out, nullptr, 0, nullptr);
    if (rc == MCE_OK) {
        unsigned long long used = 0;
        cudaError_t e = cudaMemcpyAsync(&used, cursor, 8, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) rc = fail(MCE_ECUDA, "reading the list cursor: %s", cudaGetErrorString(e));
        else {
            *words = (int64_t)used;
            if (buf && used > (unsigned long long)cap_words)
                rc = fail(MCE_ERANGE, "the list needs %llu words, buf holds %lld (split opts.roots)", used,
                          (long long)cap_words);
        }
    }
    free_plan(g, P);
    return rc;
}

extern "C" int mce_run_batch(mce_graph *g, const mce_opts *opts, mce_result *per_graph, uint64_t *hist,
                             int32_t hist_len, mce_result *total) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (!per_graph) return fail(MCE_EINVAL, "per_graph is NULL");
    return run_impl(g, opts, per_graph, hist, hist_len, total);
}

extern "C" int mce_graph_info(const mce_graph *g, int32_t *n, int64_t *m, int32_t *G, int32_t *degeneracy,
                              int32_t *max_degree) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (G) *G = g->G;
    if (degeneracy) *degeneracy = g->d;
    if (max_degree) *max_degree = g->max_deg;
    return MCE_OK;
}

extern "C" int mce_get_order(const mce_graph *g, int32_t *core, int32_t *rank, int32_t *out_degree) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    const size_t n = (size_t)g->n;
    std::vector<int32_t> hrank(n), hout(n);
    cudaError_t e = cudaSuccess;
    if (n) {
        if (core) e = cudaMemcpyAsync(core, g->core, n * 4, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hrank.data(), g->rank, n * 4, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hout.data(), g->outdeg, n * 4, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    }
    if (e != cudaSuccess) return fail(MCE_ECUDA, "copy failed: %s", cudaGetErrorString(e));
    if (rank) memcpy(rank, hrank.data(), n * 4);
    if (out_degree)
        for (size_t v = 0; v < n; v++) out_degree[v] = hout[(size_t)hrank[v]];
    return MCE_OK;
}

extern "C" int mce_root_features(mce_graph *g, int32_t *raw, float *feat) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (g->n == 0 || (!raw && !feat)) return MCE_OK;
    int rc = MCE_OK;
    CK(launch_root_features(g->n, g->out_ptr, g->out_col, g->in_ptr, g->in_col, g->order, g->core, g->d, g->sm_count,
                            raw, feat, nullptr, g->stream));
    CK(cudaStreamSynchronize(g->stream));
cleanup:
    return rc;
}

extern "C" int mce_predict_priority(mce_graph *g, mce_model *m, int32_t min_p, float *priority) {
    if (!g || !m || !priority) return fail(MCE_EINVAL, "NULL argument");
    if (g->n == 0) return MCE_OK;
    const int n = g->n;
    int rc = MCE_OK;
    int32_t *flags = (int32_t *)dalloc(g, (size_t)n * 4);
    int32_t *pos = (int32_t *)dalloc(g, ((size_t)n + 1) * 4);
    int32_t *stmp = (int32_t *)dalloc(g, (size_t)scan_tmp_words(n + 1) * 4);
    int32_t *list = nullptr;
    float *feat = nullptr, *pred = nullptr;
    int k = 0;
    if (!flags || !pos || !stmp) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
    CK(launch_select_roots(n, g->outdeg, min_p, flags, pos, stmp, nullptr, g->stream));  // count only
    CK(cudaMemcpyAsync(&k, pos + n, 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (k > 0) {
        list = (int32_t *)dalloc(g, (size_t)k * 4);
        feat = (float *)dalloc(g, (size_t)k * kNumFeatures * 4);
        pred = (float *)dalloc(g, (size_t)k * 4);
        if (!list || !feat || !pred) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        CK(launch_select_roots(n, g->outdeg, min_p, flags, pos, stmp, list, g->stream));
        CK(launch_root_features(k, g->out_ptr, g->out_col, g->in_ptr, g->in_col, g->order, g->core, g->d, g->sm_count,
                                nullptr, feat, list, g->stream));
        CK(launch_mlp_predict(model_params(m), feat, k, pred, g->sm_count, g->stream));
    }
    // roots below the threshold get the lowest priority
    CK(launch_fill_and_scatter(n, -1.0f, k, list, g->order, pred, priority, g->stream));
    CK(cudaStreamSynchronize(g->stream));
cleanup:
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *q : {(void *)flags, (void *)pos, (void *)stmp, (void *)list, (void *)feat, (void *)pred})
        dfree(g, q);
    return rc;
}

extern "C" int mce_get_stats(const mce_graph *g, mce_stats *out) {
    if (!g || !out) return fail(MCE_EINVAL, "NULL argument");
    if (out->struct_size != (int32_t)sizeof(mce_stats)) return fail(MCE_EINVAL, "mce_stats.struct_size mismatch");
    *out = g->last;
    return MCE_OK;
}

extern "C" void mce_destroy(mce_graph *g) {
    if (g) release(g);
}
