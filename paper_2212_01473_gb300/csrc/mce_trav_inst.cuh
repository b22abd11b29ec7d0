// Instantiation helper: plan and launch the traversal for one row width.
#pragma once
#include "mce_traverse.cuh"

namespace mce {

__host__ __device__ constexpr int group_warps(int wp) { return wp <= 12 ? 1 : wp <= 20 ? 4 : 8; }
// A rows in global memory (L1/L2) instead of shared memory: always when too
// wide for shared memory, and for WP = 12, where one-warp groups on rows of up
// to 340 x 12 words would fit only 11 per SM in shared memory while registers
// allow 16. Compact subtrees, where most nodes are, do not read A; the extra
// groups win (chunglu_1m widest class 69 -> 55 ms).
__host__ __device__ constexpr bool a_in_global(int wp) { return wp == 12 || wp >= 68; }
__host__ __device__ constexpr bool stack_in_smem(int wp) { return wp <= 4; }

template <int WP>
cudaError_t plan_wp(int rows, int sm_count, int max_smem_optin, int requested_blocks, int requested_warps,
                    bool block_hist, ClassLaunch *L) {
    constexpr int GW = group_warps(WP);
    constexpr bool AG = a_in_global(WP);
    const GrpSmem lay = grp_smem_layout(WP, GW, rows, AG, stack_in_smem(WP), block_hist && GW > 1);
    // groups per block: kTravMaxWarps warps by default, or the requested warps (a multiple of the group width)
    int gpb = (requested_warps >= GW && requested_warps <= kTravMaxWarps ? requested_warps : kTravMaxWarps) / GW;
    while (gpb > 1 && smem_bytes(lay, gpb) > (size_t)max_smem_optin) gpb--;
    if (smem_bytes(lay, gpb) > (size_t)max_smem_optin) return cudaErrorInvalidConfiguration;
    L->wp = WP;
    L->gw = GW;
    L->warps_per_block = gpb * GW;
    L->smem = smem_bytes(lay, gpb);
    L->a_global = AG;
    auto kern = k_traverse<WP, GW, AG, false, false, false, 0>;
    for (auto variant : {k_traverse<WP, GW, AG, false, false, false, 0>, k_traverse<WP, GW, AG, false, false, false, 1>,
                         k_traverse<WP, GW, AG, true, false>, k_traverse<WP, GW, AG, false, true>,
                         k_traverse<WP, GW, AG, true, true>, k_traverse<WP, GW, AG, false, false, true>}) {
        cudaError_t e = cudaFuncSetAttribute(variant, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->smem);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaSuccess;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L->warps_per_block * 32, L->smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int blocks = per_sm * sm_count;
    if (requested_blocks > 0 && requested_blocks < blocks) blocks = requested_blocks;
    L->blocks = blocks;
    return cudaSuccess;
}

template <int WP>
cudaError_t launch_wp(const ClassLaunch &L, const DevGraph &g, const DevOut &o, const ClassArgs &a,
                      int rows, cudaStream_t s) {
    constexpr int GW = group_warps(WP);
    constexpr bool AG = a_in_global(WP);
    const dim3 grid(L.blocks), block(L.warps_per_block * 32);
    const int ss = stack_in_smem(WP) ? 1 : 0;
    if (o.list && a.level2) k_traverse<WP, GW, AG, true, true><<<grid, block, L.smem, s>>>(g, o, a, rows, ss);
    else if (o.list) k_traverse<WP, GW, AG, true, false><<<grid, block, L.smem, s>>>(g, o, a, rows, ss);
    else if (a.level2) k_traverse<WP, GW, AG, false, true><<<grid, block, L.smem, s>>>(g, o, a, rows, ss);
    else if (a.stats) k_traverse<WP, GW, AG, false, false, true><<<grid, block, L.smem, s>>>(g, o, a, rows, ss);
    else if (a.pivot_ipx) k_traverse<WP, GW, AG, false, false, false, 1><<<grid, block, L.smem, s>>>(g, o, a, rows, ss);
    else k_traverse<WP, GW, AG, false, false, false, 0><<<grid, block, L.smem, s>>>(g, o, a, rows, ss);
    return cudaGetLastError();
}

#define MCE_INSTANTIATE_WP(WP)                                                                        \
    template cudaError_t plan_wp<WP>(int, int, int, int, int, bool, ClassLaunch *);                         \
    template cudaError_t launch_wp<WP>(const ClassLaunch &, const DevGraph &, const DevOut &,         \
                                       const ClassArgs &, int, cudaStream_t);

}  // namespace mce
