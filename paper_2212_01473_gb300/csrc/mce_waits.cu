// mce_selftest_waits: runs the engine's two kinds of device-side wait (the
// worker list's idle wait and the peel's grid barrier) on their own, where
// the outcome is known, so that the give-up path is tested without a fault.
#include <cstdio>

#include "mce_internal.cuh"

namespace mce {

// One thread waits on a flag that nothing sets, with one group counted as
// active and no heartbeat: the wait must give up with ST_TIMEOUT.
__global__ void k_selftest_idle(int *words, uint64_t timeout_ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int *flag = words, *active = words + 32, *status = words + 64;
    const unsigned long long *beat = reinterpret_cast<const unsigned long long *>(words + 96);
    idle_wait(flag, active, status, beat, timeout_ns, ~0ull);
}

// Block 0 waits as an idle group; block 1 plays a busy group that posts a
// heartbeat every timeout/4 for three timeouts and then ends the launch
// (active = 0). The wait must outlast its own bound and end without a status.
__global__ void k_selftest_beat(int *words, uint64_t timeout_ns) {
    if (threadIdx.x != 0) return;
    int *flag = words, *active = words + 32, *status = words + 64;
    unsigned long long *beat = reinterpret_cast<unsigned long long *>(words + 96);
    if (blockIdx.x == 0) {
        if (idle_wait(flag, active, status, beat, timeout_ns, ~0ull) == 0) words[65] = 1;  // ended by the launch end
    } else {
        uint64_t t0 = globaltimer_ns();
        uint64_t last = 0;
        for (;;) {
            const uint64_t now = globaltimer_ns();
            if (now < t0) t0 = now;  // the global timer stepped back: measure from here
            if (now - t0 > 3 * timeout_ns) break;
            if (now < last || now - last > timeout_ns / 4) {
                st_relaxed_u64(beat, now);
                last = now;
            }
            __nanosleep(1000);
        }
        __threadfence();
        atomicExch(active, 0);
    }
}

// Two co-resident blocks meet at a grid barrier that expects three: nobody
// releases it, so each block's wait must give up with ST_TIMEOUT.
__global__ void k_selftest_barrier(int *words, uint64_t timeout_ns) {
    GridBar *bar = reinterpret_cast<GridBar *>(words);
    int *status = words + 64;
    unsigned target = 0, gen = 0;
    grid_barrier(bar, status, timeout_ns, gridDim.x + 1, target, gen);
}

}  // namespace mce

using namespace mce;

/* which: 0 = idle wait on a flag nothing sets (expects MCE_ETIMEOUT),
 * 1 = grid barrier one block short (expects MCE_ETIMEOUT), 2 = idle wait
 * kept alive by heartbeats past its bound, then released (expects MCE_OK). */
extern "C" int mce_selftest_waits(int32_t which, int64_t timeout_ms, void *stream) {
    if (which < 0 || which > 2 || timeout_ms <= 0 || timeout_ms > 10000)
        return set_last_error(MCE_EINVAL, "mce_selftest_waits: which in 0..2, timeout_ms in 1..10000");
    cudaStream_t s = (cudaStream_t)stream;
    int *words = nullptr;
    if (cudaMallocAsync((void **)&words, 128 * sizeof(int), s) != cudaSuccess)
        return set_last_error(MCE_ENOMEM, "mce_selftest_waits: device allocation failed");
    int rc = MCE_OK;
    int h[2] = {0, 0};
    uint64_t tns = (uint64_t)timeout_ms * 1000000ull;
    cudaError_t e = cudaMemsetAsync(words, 0, 128 * sizeof(int), s);
    if (e == cudaSuccess && which != 1) {
        int one = 1;
        e = cudaMemcpyAsync(words + 32, &one, sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `one` lives on this frame
    }
    if (e == cudaSuccess) {
        void *args[] = {(void *)&words, (void *)&tns};
        const void *fn = which == 0 ? (const void *)k_selftest_idle
                       : which == 1 ? (const void *)k_selftest_barrier : (const void *)k_selftest_beat;
        const int blocks = which == 0 ? 1 : 2;
        count_launch();
        e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(32), args, 0, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, words + 64, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(words, s);
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof buf, "mce_selftest_waits: %s", cudaGetErrorString(e));
        return set_last_error(MCE_ECUDA, buf);
    }
    if (h[0] & ST_TIMEOUT) rc = set_last_error(MCE_ETIMEOUT, "mce_selftest_waits: the wait gave up");
    else if (which == 2 && h[1] != 1) rc = set_last_error(MCE_ECUDA, "mce_selftest_waits: the wait did not see the end");
    cudaStreamSynchronize(s);
    return rc;
}
