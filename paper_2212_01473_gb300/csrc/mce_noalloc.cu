// mce_peel_noalloc: the degeneracy peel (core numbers and order) for callers
// that cannot allocate device memory. All scratch lives in one file-scope
// static device array; the caller passes the graph and the output buffers.
#include <cstdio>

#include "mce_prep.cuh"

namespace mce {

// Scratch capacity: per vertex five int32 arrays (degree, two remaining-vertex
// lists, two frontiers), plus the frontier bitmap, per-block sums, the peel's
// control block and a status word.
constexpr int kNoAllocMaxN = MCE_NOALLOC_MAX_VERTICES;
constexpr int kNoAllocMaxBlocks = 1024;
constexpr size_t kNoAllocWords = 5ull * kNoAllocMaxN + (kNoAllocMaxN / 32 + 32) + kNoAllocMaxBlocks + 64 + 64;

// Shared by every call on a device and kept between calls.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

}  // namespace mce

using namespace mce;

namespace {

int noalloc_fail(int code, const char *msg) {
    char buf[256];
    snprintf(buf, sizeof buf, "mce_peel_noalloc: %s", msg);
    return mce::set_last_error(code, buf);  // reported by mce_last_error()
}

}  // namespace

extern "C" int mce_peel_noalloc(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t m,
                                int32_t *core, int32_t *rank, int32_t *order, void *stream) {
    if (n < 0 || m < 0 || 2 * m > INT32_MAX) return noalloc_fail(MCE_EINVAL, "bad sizes");
    if (n > kNoAllocMaxN) return noalloc_fail(MCE_EUNSUPPORTED, "n exceeds MCE_NOALLOC_MAX_VERTICES");
    if (n > 0 && (!row_ptr || !core || !rank || !order)) return noalloc_fail(MCE_EINVAL, "NULL pointer");
    if (m > 0 && !col) return noalloc_fail(MCE_EINVAL, "col is NULL");
    if (n == 0) return MCE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(MCE_ECUDA, "cudaGetDevice failed");
    if (s) {
        // the array and the launch belong to the current device: the stream must too
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return noalloc_fail(MCE_ECUDA, "cudaStreamGetDevice failed");
        if (sdev != dev) return noalloc_fail(MCE_EINVAL, "the stream belongs to another device than the current one");
    }
    // The array's device address in the current context, looked up on every
    // call (no allocation): a cached address would go stale if the context
    // were destroyed and created again (cudaDeviceReset).
    uint32_t *base = nullptr;
    {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return noalloc_fail(MCE_ECUDA, "cudaGetSymbolAddress failed");
        base = (uint32_t *)p;
    }
    int sm_count = 0;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return noalloc_fail(MCE_ECUDA, "cudaDeviceGetAttribute failed");

    PeelBufs pb{};
    uint32_t *q = base;
    pb.deg = (int32_t *)q;
    q += kNoAllocMaxN;
    pb.remA = (int32_t *)q;
    q += kNoAllocMaxN;
    pb.remB = (int32_t *)q;
    q += kNoAllocMaxN;
    pb.SA = (int32_t *)q;
    q += kNoAllocMaxN;
    pb.SB = (int32_t *)q;
    q += kNoAllocMaxN;
    pb.bitmap = q;
    q += kNoAllocMaxN / 32 + 32;
    pb.blocksums = (int *)q;
    q += kNoAllocMaxBlocks;
    static_assert(sizeof(PeelCtl) <= 64 * sizeof(uint32_t), "PeelCtl outgrew its scratch slot");
    pb.ctl = (PeelCtl *)q;
    q += 64;
    pb.status = (int *)q;
    pb.rank = rank;
    pb.core = core;
    pb.order = order;
    pb.max_blocks = sm_count * 2 < kNoAllocMaxBlocks ? sm_count * 2 : kNoAllocMaxBlocks;

    // the array keeps the previous call's contents: clear what must start at zero
    int h_status = 0;
    if (cudaMemsetAsync(pb.status, 0, 4 * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(pb.bitmap, 0, ((size_t)n + 31) / 32 * sizeof(uint32_t), s) != cudaSuccess)
        return noalloc_fail(MCE_ECUDA, "cudaMemsetAsync failed");
    if (launch_validate(n, row_ptr, col, 2 * m, pb.status, s, false) != cudaSuccess ||
        cudaMemcpyAsync(&h_status, pb.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(MCE_ECUDA, "validation launch failed");
    if (h_status) return noalloc_fail(MCE_EINVAL, "row_ptr is not a valid offset array");
    if (launch_validate(n, row_ptr, col, 2 * m, pb.status, s, true) != cudaSuccess ||
        cudaMemcpyAsync(&h_status, pb.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(MCE_ECUDA, "validation launch failed");
    if (h_status) return noalloc_fail(MCE_EINVAL, "graph is not a canonical simple undirected CSR");

    PeelCtl hctl{};
    if (launch_peel_init(pb.ctl, n, s) != cudaSuccess ||
        launch_peel(n, row_ptr, col, pb, sm_count, kPeelWaitNs, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_status, pb.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hctl, pb.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(MCE_ECUDA, "peel launch failed");
    if (h_status & ST_TIMEOUT) return noalloc_fail(MCE_ETIMEOUT, "a grid-barrier wait of the peel exceeded 60 s");
    if (hctl.next != n) return noalloc_fail(MCE_ECUDA, "peel ended early");
    return MCE_OK;
}
