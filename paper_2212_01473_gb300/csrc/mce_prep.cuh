// Pre-processing kernels (validation, peel, orientation): host launchers.
#pragma once
#include "mce_internal.cuh"

namespace mce {

struct PeelCtl {
    int k, next, rounds;  // written at the end of the peel
    int cnt[3];           // sub-round sizes, a ring indexed by sub-round % 3
    int nrem2[3];         // next remaining-list size, a ring indexed by level % 3
    int minval[3];        // smallest live degree at a level start, by level % 3
    unsigned long long sumdeg[3];  // live degree sum at a level start, by level % 3
    GridBar bar;
    // globaltimer (ns) at the start, at the narrow and one-block stages (0 if
    // never reached) and at the end, by block 0; stage sub-rounds likewise
    unsigned long long t_start, t_narrow, t_solo, t_end;
    int r_narrow, r_solo;
    // handoff to the cluster kernel of the narrow stage: set by block 0 of the
    // full-grid kernel when it stops there (rs_active = 1), read by every CTA
    // of the cluster: level k, next guess, ranked so far, remaining-list size,
    // sub-round, phase and level counters, remaining-list buffer, S size
    int rs_active, rs_k, rs_guess, rs_next, rs_nrem, rs_t, rs_r, rs_L, rs_remsel, rs_ns;
};

struct PeelBufs {
    int32_t *deg, *rank, *core, *order, *remA, *remB;
    int32_t *SA;  // n ints: start of each removal sub-round in order
    int32_t *SB;  // unused
    unsigned *bitmap;  // ceil(n/32) words, zero on entry and on exit
    int *blocksums;    // max_blocks
    PeelCtl *ctl;
    int *status;
    int max_blocks;
};

cudaError_t launch_validate(int n, const int32_t *rp, const int32_t *col, int64_t m2, int *status,
                            cudaStream_t s, bool cols);
cudaError_t launch_peel_init(PeelCtl *ctl, int n, cudaStream_t s);
// bound of each grid-barrier wait of the peel (mce_create, mce_peel_noalloc)
constexpr uint64_t kPeelWaitNs = 60ull * 1000000000ull;
cudaError_t launch_peel(int n, const int32_t *rp, const int32_t *col, PeelBufs &b, int sm_count,
                        uint64_t timeout_ns, cudaStream_t s);
cudaError_t exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s);
// out[i] = outdeg[roots[i]] for i < k
cudaError_t launch_gather_outdeg(const int32_t *roots, int64_t k, const int32_t *outdeg, int32_t *out,
                                 cudaStream_t s);
int64_t scan_tmp_words(int64_t n);
cudaError_t launch_orient(int n, const int32_t *rp, const int32_t *col, const int32_t *order,
                          const int32_t *rank, int32_t *outdeg, int32_t *indeg, int32_t *out_ptr,
                          int32_t *out_col, int32_t *in_ptr, int32_t *in_col, int32_t *scan_tmp,
                          int *long_rows /* n + 1 ints */, cudaStream_t s);
cudaError_t launch_mix_gid(int n, const int32_t *order, uint64_t *mixid, int32_t *gid,
                           const int32_t *graph_ptr, int G, cudaStream_t s);
cudaError_t launch_classify(int n, const int32_t *outdeg, const int32_t *indeg, int *cls_rows,
                            int *cls_x, int *cls_count, cudaStream_t s);
cudaError_t launch_class_list(int n, const int32_t *outdeg, int c, int32_t *flags, int32_t *pos,
                              int32_t *scan_tmp, int32_t *out, cudaStream_t s);

// keep the entries of list[0..cnt) (ranks) whose mask[rank] is set, in order
cudaError_t launch_mark_roots(const int32_t *ids, int64_t k, const int32_t *rank, int n, int32_t *mask,
                              int *status, cudaStream_t s);
cudaError_t launch_subset(const int32_t *list, int cnt, const int32_t *mask, int32_t *flags, int32_t *pos,
                          int32_t *scan_tmp, int32_t *out, cudaStream_t s);

// roots of list[0..cnt) by descending prio[order[r]] (quarter-unit buckets,
// any order inside a bucket); hist: 256 ints of scratch
// Roots of list[0..cnt) by descending prio (256 buckets of a quarter unit);
// roots with prio < 0 or NaN keep their list order after all others. flags
// and pos hold cnt + 1 ints, scan_tmp scan_tmp_words(cnt + 1).
cudaError_t launch_priority_order(const int32_t *list, int cnt, const int32_t *order, const float *prio,
                                  int *hist, int32_t *flags, int32_t *pos, int32_t *scan_tmp, int32_t *out,
                                  cudaStream_t s);

}  // namespace mce
