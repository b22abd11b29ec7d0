// C ABI of the engine (include/mce.h): handle creation (validation, peel,
// orientation, width classes), runs (persistent traversal launches per width
// class) and results.
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
    extern template cudaError_t plan_wp<WP>(int, int, int, int, bool, ClassLaunch *);                       \
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

static cudaError_t plan_class_wp(int wp, int rows, int sms, int smem, int req, bool bh, ClassLaunch *L) {
    switch (wp) {
        case 1: return plan_wp<1>(rows, sms, smem, req, bh, L);
        case 2: return plan_wp<2>(rows, sms, smem, req, bh, L);
        case 4: return plan_wp<4>(rows, sms, smem, req, bh, L);
        case 12: return plan_wp<12>(rows, sms, smem, req, bh, L);
        case 20: return plan_wp<20>(rows, sms, smem, req, bh, L);
        case 28: return plan_wp<28>(rows, sms, smem, req, bh, L);
        case 36: return plan_wp<36>(rows, sms, smem, req, bh, L);
        case 68: return plan_wp<68>(rows, sms, smem, req, bh, L);
        case 132: return plan_wp<132>(rows, sms, smem, req, bh, L);
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
__global__ void k_trivial_roots(DevGraph G, DevOut O, const int32_t *roots, int n_roots) {
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
            if (O.root_nodes) O.root_nodes[id] += 1ull;
            if (clique && O.root_count) O.root_count[id] += 1ull;
            if (clique && O.root_hash) O.root_hash[id] += h;
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
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(O.nodes, (unsigned long long)n_roots);
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
    uint64_t create_launches = 0;  // kernels launched by create
    mce_stats last{};              // facts of the last run
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

static void release(mce_graph *g) {
    void *ps[] = {g->out_ptr, g->out_col, g->in_ptr, g->in_col, g->order, g->rank,
                  g->core,    g->outdeg,  g->gid,    g->mixid,  g->scratch};
    for (void *p : ps) dfree(g, p);
    for (int c = 0; c <= kNumClasses; c++) dfree(g, g->class_roots[c]);
    if (g->stream) cudaStreamSynchronize(g->stream);
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
        CK(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
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
        int32_t zero = 0;
        if (dev_in) {
            int32_t v0 = 0;
            CK(cudaMemcpyAsync(&v0, row_ptr, 4, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            if (v0 != 0 || m != 0) { rc = fail(MCE_EINVAL, "row_ptr[0] must be 0 and m 0 for n = 0"); goto cleanup; }
        } else if (row_ptr && (row_ptr[0] != 0 || m != 0)) {
            rc = fail(MCE_EINVAL, "row_ptr[0] must be 0 and m 0 for n = 0");
            goto cleanup;
        }
        (void)zero;
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
        if (n > 0) CK(launch_peel(n, d_rp, d_col, pb, g->sm_count, 30ull * 1000000000ull, g->stream));
        CK(cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, g->stream));
        PeelCtl hctl{};
        CK(cudaMemcpyAsync(&hctl, pb.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (h_status & ST_TIMEOUT) { rc = fail(MCE_ETIMEOUT, "degeneracy peel timed out"); goto cleanup; }
        if (hctl.next != n) { rc = fail(MCE_ECUDA, "peel ended early (%d of %d ranked)", hctl.next, n); goto cleanup; }
        g->peel_rounds = hctl.rounds;

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
    dfree(g, g->scratch);
    g->scratch = nullptr;
    g->scratch_bytes = 0;
    size_t want = bytes + bytes / 8;
    g->scratch = dalloc(g, want);
    if (!g->scratch) return fail(MCE_ENOMEM, "device allocation of %zu bytes of traversal scratch failed", want);
    g->scratch_bytes = want;
    return MCE_OK;
}

// Shared implementation of mce_run / mce_run_batch.
static int run_impl(mce_graph *g, const mce_opts *opts_in, mce_result *per_graph, uint64_t *hist,
                    int32_t hist_len, mce_result *total) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    mce_opts opts;
    mce_default_opts(&opts);
    if (opts_in) {
        if (opts_in->struct_size != (int32_t)sizeof(mce_opts)) return fail(MCE_EINVAL, "opts.struct_size mismatch");
        opts = *opts_in;
    }
    if (opts.pivot < 0 || opts.pivot > 2) return fail(MCE_EINVAL, "bad opts.pivot");
    if (opts.order != MCE_ORDER_PLAIN && opts.order != MCE_ORDER_PRIORITY) return fail(MCE_EINVAL, "bad opts.order");
    if (opts.order == MCE_ORDER_PRIORITY && !opts.root_priority)
        return fail(MCE_EINVAL, "MCE_ORDER_PRIORITY needs opts.root_priority");
    if (opts.pivot == MCE_PIVOT_IPX) return fail(MCE_EINVAL, "IPX pivoting is not available in this build");
    if (opts.donate_min_p < 0) return fail(MCE_EINVAL, "opts.donate_min_p < 0");
    if (opts.donate_policy < 0 || opts.donate_policy > 2) return fail(MCE_EINVAL, "bad opts.donate_policy");
    if (opts.timeout_ms <= 0) opts.timeout_ms = 60000;
    if (hist && hist_len < 0) return fail(MCE_EINVAL, "hist_len < 0");
    const int G = g->G;
    const int HL = g->d + 2;  // every maximal clique has at most d + 1 vertices
    int rc = MCE_OK;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<unsigned long long> hcnt(G), hhash(G), hhist((size_t)G * HL);
    unsigned long long hmisc[4] = {0, 0, 0, 0};
    int hflags[4] = {0, 0, 0, 0};
    DevGraph dg{};
    DevOut dout{};
    // outputs: count[G], hash[G], hist[G*HL], nodes, donations | max_size, status,
    // phase cycles and counts
    const size_t out_words64 = (size_t)2 * G + (size_t)G * HL + 4 + 2 * kNumPhases;
    mce_stats st{};
    std::vector<cudaEvent_t> cev;
    uint64_t launches = 0;
    const uint64_t launch_base = launch_counter();
    // roots to enumerate per width class (all, or the subset opts.roots selects)
    const int32_t *lists[kNumClasses + 1];
    int32_t counts[kNumClasses + 1];
    for (int c = 0; c <= kNumClasses; c++) {
        lists[c] = g->class_roots[c];
        counts[c] = g->class_count[c];
    }
    std::vector<void *> run_tmp;
    unsigned long long *obuf = (unsigned long long *)dalloc(g, out_words64 * 8 + 64);
    if (!obuf) return fail(MCE_ENOMEM, "device allocation of outputs failed");
    CK(cudaMemsetAsync(obuf, 0, out_words64 * 8 + 64, g->stream));
    if (opts.root_count) CK(cudaMemsetAsync(opts.root_count, 0, (size_t)g->n * 8, g->stream));
    if (opts.root_hash) CK(cudaMemsetAsync(opts.root_hash, 0, (size_t)g->n * 8, g->stream));
    if (opts.root_nodes) CK(cudaMemsetAsync(opts.root_nodes, 0, (size_t)g->n * 8, g->stream));
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    dg.n = g->n;
    dg.G = G;
    dg.out_ptr = g->out_ptr;
    dg.out_col = g->out_col;
    dg.in_ptr = g->in_ptr;
    dg.in_col = g->in_col;
    dg.order = g->order;
    dg.mixid = g->mixid;
    dg.gid = g->gid;
    dout.count = obuf;
    dout.hash = obuf + G;
    dout.hist = obuf + 2 * G;
    dout.hist_len = HL;
    dout.nodes = obuf + 2 * G + (size_t)G * HL;
    dout.donations = dout.nodes + 1;
    dout.max_size = (int *)(dout.nodes + 2);
    dout.status = dout.max_size + 1;
    dout.phase_cycles = dout.nodes + 4;
    dout.phase_counts = dout.phase_cycles + kNumPhases;
    dout.root_count = (unsigned long long *)opts.root_count;
    dout.root_hash = (unsigned long long *)opts.root_hash;
    dout.root_nodes = (unsigned long long *)opts.root_nodes;
    st.struct_size = (int32_t)sizeof(mce_stats);
    if (opts.roots && opts.n_roots < 0) { rc = fail(MCE_EINVAL, "opts.n_roots < 0"); goto cleanup; }
    if (opts.roots && g->n > 0) {
        int maxc = 1;
        for (int c = 0; c <= kNumClasses; c++) maxc = std::max(maxc, g->class_count[c]);
        int32_t *mask = (int32_t *)dalloc(g, (size_t)g->n * 4);
        int32_t *flags = (int32_t *)dalloc(g, (size_t)maxc * 4);
        int32_t *pos = (int32_t *)dalloc(g, ((size_t)maxc + 1) * 4);
        int32_t *stmp = (int32_t *)dalloc(g, (size_t)scan_tmp_words(maxc + 1) * 4);
        for (void *q : {(void *)mask, (void *)flags, (void *)pos, (void *)stmp}) run_tmp.push_back(q);
        if (!mask || !flags || !pos || !stmp) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        CK(cudaMemsetAsync(mask, 0, (size_t)g->n * 4, g->stream));
        CK(launch_mark_roots(opts.roots, opts.n_roots, g->rank, g->n, mask, dout.status, g->stream));
        int hst = 0;
        CK(cudaMemcpyAsync(&hst, dout.status, 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (hst) { rc = fail(MCE_EINVAL, "opts.roots holds an id outside [0, n)"); goto cleanup; }
        for (int c = 0; c <= kNumClasses; c++) {
            if (counts[c] == 0) continue;
            int32_t *out = (int32_t *)dalloc(g, (size_t)counts[c] * 4);
            run_tmp.push_back(out);
            if (!out) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
            CK(launch_subset(lists[c], counts[c], mask, flags, pos, stmp, out, g->stream));
            int kept = 0;
            CK(cudaMemcpyAsync(&kept, pos + counts[c], 4, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            lists[c] = out;
            counts[c] = kept;
        }
    }
    if (opts.order == MCE_ORDER_PRIORITY && g->n > 0) {
        int *hb = (int *)dalloc(g, 256 * sizeof(int));
        run_tmp.push_back(hb);
        if (!hb) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
        for (int c = 0; c < kNumClasses; c++) {
            if (counts[c] == 0) continue;
            int32_t *out = (int32_t *)dalloc(g, (size_t)counts[c] * 4);
            run_tmp.push_back(out);
            if (!out) { rc = fail(MCE_ENOMEM, "device allocation failed"); goto cleanup; }
            CK(launch_priority_order(lists[c], counts[c], g->order, opts.root_priority, hb, out, g->stream));
            lists[c] = out;
        }
    }
    CK(cudaEventRecord(ev0, g->stream));
    if (counts[kNumClasses] > 0) {
        const int nr = counts[kNumClasses];
        const unsigned nb = (unsigned)std::min<int64_t>(4096, ((int64_t)nr + 255) / 256);
        cudaEvent_t a0, a1;
        CK(cudaEventCreate(&a0));
        cev.push_back(a0);
        CK(cudaEventCreate(&a1));
        cev.push_back(a1);
        CK(cudaEventRecord(a0, g->stream));
        k_trivial_roots<<<nb, 256, 0, g->stream>>>(dg, dout, lists[kNumClasses], nr);
        count_launch();
        CK(cudaGetLastError());
        CK(cudaEventRecord(a1, g->stream));
        launches++;
        const int k = st.n_classes++;
        st.class_wp[k] = 0;
        st.class_roots[k] = nr;
        st.class_blocks[k] = (int32_t)nb;
    }
    // heaviest width classes first
    for (int c = kNumClasses - 1; c >= 0; c--) {
        if (counts[c] == 0) continue;
        const int rows = g->class_rows[c];
        ClassLaunch L{};
        CK(plan_class_wp(class_wp(c), rows, g->sm_count, g->smem_optin, opts.blocks, g->gid == nullptr, &L));
        const int groups = L.blocks * (L.warps_per_block / L.gw);
        const size_t aw = arena_words(L.wp, rows, g->class_x[c], L.a_global, stack_in_smem(L.wp));
        const int mail_words = 4 + 3 * L.wp;
        const size_t ctl_words = CTL_NCTL, idle_words = ((size_t)groups + 31) / 32;
        const size_t flag_words = (size_t)groups * kMailFlagStride;
        const size_t total_words = aw * groups + ctl_words + idle_words + flag_words + (size_t)groups * mail_words + 64;
        if ((rc = grow_scratch(g, total_words * 4)) != MCE_OK) goto cleanup;
        uint32_t *sw = (uint32_t *)g->scratch;
        ClassArgs a{};
        a.roots = lists[c];
        a.n_roots = counts[c];
        a.rows_cap = rows;
        a.x_cap = g->class_x[c];
        a.pivot_ipx = 0;
        a.worker_list = opts.worker_list ? 1 : 0;
        // 0 = automatic: a donated child must have at least 1/8 of the
        // class's widest root set, and never fewer than 10 candidates (Sec. III-C)
        a.donate_min_p = opts.donate_min_p > 0 ? opts.donate_min_p : std::max(10, rows / 8);
        a.donate_policy = opts.donate_policy;
        a.root_chunk = 1;
        a.stats = opts.stats ? 1 : 0;
        a.timeout_ns = (uint64_t)opts.timeout_ms * 1000000ull;
        a.arena = sw;
        a.arena_words_per_group = aw;
        a.ctl = (int *)(sw + aw * groups);
        a.idle_bits = (unsigned *)(a.ctl + ctl_words);
        a.mail_flag = (int *)(a.idle_bits + idle_words);
        a.mail = (uint32_t *)(a.mail_flag + flag_words);
        a.mail_words = mail_words;
        CK(cudaMemsetAsync(a.ctl, 0, (ctl_words + idle_words + flag_words) * 4, g->stream));
        int hctl[CTL_NCTL] = {0};
        hctl[CTL_ACTIVE] = groups;
        CK(cudaMemcpyAsync(a.ctl, hctl, sizeof hctl, cudaMemcpyHostToDevice, g->stream));
        cudaEvent_t a0, a1;
        CK(cudaEventCreate(&a0));
        cev.push_back(a0);
        CK(cudaEventCreate(&a1));
        cev.push_back(a1);
        CK(cudaEventRecord(a0, g->stream));
        CK(launch_class_wp(L, dg, dout, a, rows, g->stream));
        CK(cudaEventRecord(a1, g->stream));
        launches++;
        const int k = st.n_classes++;
        st.class_wp[k] = L.wp;
        st.class_roots[k] = counts[c];
        st.class_rows[k] = rows;
        st.class_blocks[k] = L.blocks;
        st.class_groups[k] = groups;
        st.class_group_warps[k] = L.gw;
    }
    CK(cudaEventRecord(ev1, g->stream));
    CK(cudaMemcpyAsync(hcnt.data(), dout.count, (size_t)G * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hhash.data(), dout.hash, (size_t)G * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hhist.data(), dout.hist, (size_t)G * HL * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hmisc, dout.nodes, 2 * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hflags, dout.max_size, 2 * 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(st.phase_cycles, dout.phase_cycles, 2 * kNumPhases * 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    for (int k = 0; k < st.n_classes; k++) {
        float cms = 0;
        CK(cudaEventElapsedTime(&cms, cev[2 * k], cev[2 * k + 1]));
        st.class_ms[k] = cms;
    }
    st.kernel_launches = g->create_launches + (launch_counter() - launch_base) + launches;
    st.peel_rounds = g->peel_rounds;
    g->last = st;
    if (hflags[1] & ST_TIMEOUT) { rc = fail(MCE_ETIMEOUT, "a traversal wait exceeded %lld ms", (long long)opts.timeout_ms); goto cleanup; }
    if (hflags[1] & ST_OVERFLOW) { rc = fail(MCE_ECUDA, "internal capacity exceeded in the traversal"); goto cleanup; }
    {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ev0, ev1));
        mce_result tot{};
        for (int gi = 0; gi < G; gi++) {
            mce_result r{};
            r.count = hcnt[gi];
            r.hash = hhash[gi];
            int mx = 0;
            for (int s = HL - 1; s > 0; s--)
                if (hhist[(size_t)gi * HL + s]) { mx = s; break; }
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
                for (int s = 0; s < hist_len; s++)
                    hist[(size_t)gi * hist_len + s] = s < HL ? hhist[(size_t)gi * HL + s] : 0ull;
        }
        if (hist && hist_len <= tot.max_size) rc = fail(MCE_ERANGE, "hist_len %d <= max clique size %d", hist_len, tot.max_size);
    }
cleanup:
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (cudaEvent_t e : cev) cudaEventDestroy(e);
    for (void *q : run_tmp) dfree(g, q);
    dfree(g, obuf);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    return rc;
}

extern "C" int mce_run(mce_graph *g, const mce_opts *opts, mce_result *out, uint64_t *hist, int32_t hist_len) {
    if (!g) return fail(MCE_EINVAL, "graph handle is NULL");
    if (g->G != 1) return fail(MCE_EINVAL, "batched handle: use mce_run_batch");
    if (!out) return fail(MCE_EINVAL, "out is NULL");
    return run_impl(g, opts, out, hist, hist_len, nullptr);
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
    const int threads = 256;
    const int blocks = std::min<int64_t>((int64_t)g->sm_count * 16, ((int64_t)g->n * 32 + threads - 1) / threads);
    const int warps = blocks * (threads / 32);
    const int stride = g->d + 1;
    int rc = MCE_OK;
    int32_t *scratch = (int32_t *)dalloc(g, (size_t)warps * stride * sizeof(int32_t));
    if (!scratch) return fail(MCE_ENOMEM, "device allocation failed");
    CK(launch_root_features(g->n, g->out_ptr, g->out_col, g->in_ptr, g->in_col, g->order, g->core, scratch, stride,
                            warps, raw, feat, g->stream));
    CK(cudaStreamSynchronize(g->stream));
cleanup:
    dfree(g, scratch);
    if (g->stream) cudaStreamSynchronize(g->stream);
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
