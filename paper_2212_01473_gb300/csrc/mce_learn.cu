// Learned work estimator: per-root features, and an MLP 16-64-64-1 (ReLU,
// BF16 weights, FP32 accumulation) with inference, training (forward,
// backward, Adam) and gradient kernels. The estimate orders, and can split,
// roots for the traversal; it never changes a result.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <algorithm>

#include "mce_learn.cuh"
#include "mce_prep.cuh"

namespace mce {

// ------------------------------------------------------------- features

__device__ __forceinline__ int find_sorted(const int32_t *a, int lo, int hi, int32_t key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int32_t sat32(long long x) { return x > INT32_MAX ? INT32_MAX : (int32_t)x; }

// excluded vertices whose adjacency to P0 the features examine (bounds the
// per-root cost for hubs with tens of thousands of earlier neighbours)
constexpr int kXCap = 256;

// One warp per root. Roots are all ranks 0..n-1 (list == NULL; outputs
// indexed by input id) or list[0..n) (outputs indexed by list position).
// Each warp stages the root's P0, the in-P0 degree counters and 32 per-list
// hit counters in shared memory (2 * stride + 32 ints per warp, stride >=
// degeneracy + 1). The later lists are walked 32 at a time by the whole warp
// (warp_walk_lists), as the traversal builds a root's rows.
__global__ void k_root_features(int n, const int32_t *out_ptr, const int32_t *out_col, const int32_t *in_ptr,
                                const int32_t *in_col, const int32_t *order, const int32_t *core_by_id,
                                int stride, int32_t *raw, float *feat, const int32_t *list) {
    extern __shared__ int32_t fsm[];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t *P0 = fsm + (size_t)(threadIdx.x >> 5) * (2 * stride + 32);
    int32_t *dg = P0 + stride;
    int32_t *xcnt = dg + stride;
    for (int64_t it = w0; it < n; it += nw) {
        const int64_t r = list ? list[it] : it;
        const int32_t *P0g = out_col + out_ptr[r];
        const int n0 = out_ptr[r + 1] - out_ptr[r];
        const int32_t *X0 = in_col + in_ptr[r];
        const int x0 = in_ptr[r + 1] - in_ptr[r];
        for (int i = lane; i < n0; i += 32) {
            P0[i] = P0g[i];
            dg[i] = 0;
        }
        __syncwarp();
        // edges inside P0: u = P0[i] finds its later neighbours w in P0 (all
        // of u's later list lies after u; only its part up to P0's last rank
        // can hold w)
        const int32_t maxp = n0 > 0 ? P0[n0 - 1] : -1;
        long long eP = 0;
        for (int i0 = 0; i0 < n0; i0 += 32) {
            const int i = i0 + lane;
            int jb = 0, cnt = 0;
            if (i < n0) {
                const int32_t u = P0[i];
                jb = out_ptr[u];
                const int lu = out_ptr[u + 1] - jb;
                cnt = (lu == 0 || out_col[jb + lu - 1] <= maxp) ? lu : find_sorted(out_col + jb, 0, lu, maxp + 1);
            }
            warp_walk_lists<4>(out_col, jb, cnt, lane, P0, n0, [&](int l, int k) {
                atomicAdd(&dg[i0 + l], 1);
                atomicAdd(&dg[k], 1);
                eP++;
            });
        }
        __syncwarp();
        long long core_sum = 0, two_hop = 0;
        int degmax = 0, degmin = INT32_MAX, univ = 0, core_max = 0;
        for (int i = lane; i < n0; i += 32) {
            const int d = dg[i];
            degmax = max(degmax, d);
            degmin = min(degmin, d);
            univ += (d == n0 - 1);
            const int32_t u = P0[i];
            const int cu = core_by_id[order[u]];
            core_max = max(core_max, cu);
            core_sum += cu;
            two_hop += (out_ptr[u + 1] - out_ptr[u]) + (in_ptr[u + 1] - in_ptr[u]);
        }
        // edges between X0' and P0, X0' = the first kXCap vertices of X0 by
        // input id (X0 keeps the input's ascending-id order); x is earlier than
        // r, so x->w with w in P0 is one of x's later edges
        long long eX = 0;
        int xmax = 0;
        for (int i = lane; i < x0; i += 32) {
            const int32_t x = X0[i];
            two_hop += (out_ptr[x + 1] - out_ptr[x]) + (in_ptr[x + 1] - in_ptr[x]);
        }
        const int xc = min(x0, kXCap);
        for (int i0 = 0; i0 < xc; i0 += 32) {
            const int i = i0 + lane;
            int jb = 0, cnt = 0;
            if (i < xc) {
                const int32_t x = X0[i];
                jb = out_ptr[x];
                const int lx = out_ptr[x + 1] - jb;
                const int32_t *nx = out_col + jb;
                const int j0 = find_sorted(nx, 0, lx, (int32_t)r + 1);
                const int j1 = (j0 == lx || nx[lx - 1] <= maxp) ? lx : find_sorted(nx, j0, lx, maxp + 1);
                jb += j0;
                cnt = j1 - j0;
            }
            xcnt[lane] = 0;
            __syncwarp();
            warp_walk_lists<4>(out_col, jb, cnt, lane, P0, n0, [&](int l, int) { atomicAdd(&xcnt[l], 1); });
            __syncwarp();
            if (i < xc) {
                const int c = xcnt[lane];
                eX += c;
                xmax = max(xmax, c);
            }
            __syncwarp();
        }
        for (int o = 16; o; o >>= 1) {
            eP += __shfl_xor_sync(0xffffffffu, eP, o);
            eX += __shfl_xor_sync(0xffffffffu, eX, o);
            core_sum += __shfl_xor_sync(0xffffffffu, core_sum, o);
            two_hop += __shfl_xor_sync(0xffffffffu, two_hop, o);
            degmax = max(degmax, __shfl_xor_sync(0xffffffffu, degmax, o));
            degmin = min(degmin, __shfl_xor_sync(0xffffffffu, degmin, o));
            univ += __shfl_xor_sync(0xffffffffu, univ, o);
            core_max = max(core_max, __shfl_xor_sync(0xffffffffu, core_max, o));
            xmax = max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        }
        if (lane < kNumFeatures) {
            const long long pairs = (long long)n0 * (n0 - 1) / 2;
            long long f = 0;
            switch (lane) {
                case 0: f = (long long)n0 + x0; break;                       // degree
                case 1: f = core_by_id[order[r]]; break;                     // core number
                case 2: f = n0; break;                                       // |P0|
                case 3: f = x0; break;                                       // |X0|
                case 4: f = eP + eX; break;                                  // e(P0) + e(P0, X0')
                case 5: f = eP; break;                                       // e(P0)
                case 6: f = eX; break;                                       // e(P0, X0')
                case 7: f = pairs > 0 ? (eP * 65536) / pairs : 0; break;     // floor(2^16 density(P0))
                case 8: f = two_hop; break;                                  // sum of neighbour degrees
                case 9: f = n0 ? degmax : 0; break;                          // max degree inside P0
                case 10: f = n0 ? degmin : 0; break;                         // min degree inside P0
                case 11: f = univ; break;                                    // vertices adjacent to all of P0
                case 12: f = core_max; break;                                // max core over P0
                case 13: f = core_sum; break;                                // sum of cores over P0
                case 14: f = xmax; break;                                    // max |N(x) n P0|, x in X0'
                case 15: f = pairs - eP; break;                              // missing edges in P0
            }
            const int32_t v = sat32(f);
            const size_t at = list ? (size_t)it : (size_t)order[r];
            if (raw) raw[at * kNumFeatures + lane] = v;
            if (feat) feat[at * kNumFeatures + lane] = log2f(1.0f + (float)v);
        }
        __syncwarp();
    }
}

cudaError_t launch_root_features(int n, const int32_t *out_ptr, const int32_t *out_col, const int32_t *in_ptr,
                                 const int32_t *in_col, const int32_t *order, const int32_t *core_by_id,
                                 int degeneracy, int sm_count, int32_t *raw, float *feat, const int32_t *list,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int threads = 128;  // 4 warps, each with 2 * stride + 32 ints of shared memory
    const int stride = (degeneracy + 4) / 4 * 4;
    const size_t smem = (size_t)(threads / 32) * (2 * stride + 32) * sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_root_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_root_features, threads, smem);
    if (e != cudaSuccess) return e;
    const int64_t want = ((int64_t)n + 3) / 4;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)sm_count * std::max(per_sm, 1));
    k_root_features<<<blocks, threads, smem, s>>>(n, out_ptr, out_col, in_ptr, in_col, order, core_by_id, stride,
                                                  raw, feat, list);
    count_launch();
    return cudaGetLastError();
}

// roots whose |P0| >= min_p (ranks, ascending) and the priority fill
__global__ void k_flag_min_p(int n, const int32_t *outdeg, int min_p, int32_t *flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        flags[r] = outdeg[r] >= min_p;
}

__global__ void k_gather_ranks(int n, const int32_t *flags, const int32_t *pos, int32_t *list) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        if (flags[r]) list[pos[r]] = (int32_t)r;
}

__global__ void k_fill_f32(float *a, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_scatter_pred(int k, const int32_t *list, const int32_t *order, const float *pred, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        out[order[list[i]]] = pred[i];
}

cudaError_t launch_select_roots(int n, const int32_t *outdeg, int min_p, int32_t *flags, int32_t *pos,
                                int32_t *scan_tmp, int32_t *list, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned b = (unsigned)std::min<int64_t>(65536, ((int64_t)n + 255) / 256);
    k_flag_min_p<<<b, 256, 0, s>>>(n, outdeg, min_p, flags);
    count_launch();
    cudaError_t e = exclusive_scan(flags, pos, n, scan_tmp, s);
    if (e != cudaSuccess) return e;
    if (list) {  // NULL: only count (pos[n])
        k_gather_ranks<<<b, 256, 0, s>>>(n, flags, pos, list);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_and_scatter(int64_t n, float fill, int k, const int32_t *list, const int32_t *order,
                                    const float *pred, float *out, cudaStream_t s) {
    k_fill_f32<<<(unsigned)std::min<int64_t>(65536, (n + 255) / 256 + 1), 256, 0, s>>>(out, n, fill);
    count_launch();
    if (k > 0) {
        k_scatter_pred<<<(unsigned)std::min<int64_t>(65536, ((int64_t)k + 255) / 256), 256, 0, s>>>(k, list, order,
                                                                                                    pred, out);
        count_launch();
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ MLP

// Parameter layout (floats): W1[64][16] b1[64] W2[64][64] b2[64] W3[64] b3[1]
// mean[16] std[16]; the standardisation pair is not trained.
constexpr int H = kHidden, F = kNumFeatures;
constexpr int OW1 = 0, OB1 = OW1 + H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H,
              OMEAN = OB3 + 1, OSTD = OMEAN + F, NTRAIN = OMEAN;
static_assert(OSTD + F == kModelParams, "parameter layout");

__device__ __forceinline__ float bf(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// Forward of one sample; weights (bf16-rounded) and biases in shared memory.
struct SmemMLP {
    float W1[H * F], b1[H], W2[H * H], b2[H], W3[H], b3, mean[F], std_[F];
};

__device__ void load_mlp(SmemMLP &m, const float *params) {
    for (int i = threadIdx.x; i < H * F; i += blockDim.x) m.W1[i] = bf(params[OW1 + i]);
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) m.W2[i] = bf(params[OW2 + i]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        m.b1[i] = params[OB1 + i];
        m.b2[i] = params[OB2 + i];
        m.W3[i] = bf(params[OW3 + i]);
    }
    for (int i = threadIdx.x; i < F; i += blockDim.x) {
        m.mean[i] = params[OMEAN + i];
        m.std_[i] = params[OSTD + i];
    }
    if (threadIdx.x == 0) m.b3 = params[OB3];
    __syncthreads();
}

__device__ __forceinline__ float mlp_forward(const SmemMLP &m, const float *xin, float *h1, float *h2) {
    float x[F];
#pragma unroll
    for (int j = 0; j < F; j++) x[j] = (xin[j] - m.mean[j]) / m.std_[j];
    for (int i = 0; i < H; i++) {
        float a = m.b1[i];
#pragma unroll
        for (int j = 0; j < F; j++) a = fmaf(m.W1[i * F + j], x[j], a);
        h1[i] = a > 0.f ? a : 0.f;
    }
    for (int i = 0; i < H; i++) {
        float a = m.b2[i];
        for (int j = 0; j < H; j++) a = fmaf(m.W2[i * H + j], h1[j], a);
        h2[i] = a > 0.f ? a : 0.f;
    }
    float y = m.b3;
    for (int j = 0; j < H; j++) y = fmaf(m.W3[j], h2[j], y);
    return y;
}

__global__ void __launch_bounds__(128) k_mlp_predict(const float *params, const float *feat, int64_t n, float *out) {
    __shared__ SmemMLP m;
    load_mlp(m, params);
    float h1[H], h2[H];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mlp_forward(m, feat + i * F, h1, h2);
}

// Gradients of L = (1/B) sum_s (y_s - t_s)^2 with respect to the FP32 master
// parameters (the BF16 rounding passes gradients straight through).
// Per block: kGradTile samples; activations and deltas staged in shared
// memory, then the block's partial weight gradients are added atomically.
constexpr int kGradTile = 16;

__global__ void __launch_bounds__(128) k_mlp_grad(const float *params, const float *feat, const float *label,
                                                  int B, float *grad, float *loss_sum) {
    __shared__ SmemMLP m;
    __shared__ float X[kGradTile][F], A1[kGradTile][H], A2[kGradTile][H], D2[kGradTile][H], D1[kGradTile][H];
    __shared__ float DY[kGradTile];
    load_mlp(m, params);
    const int s0 = blockIdx.x * kGradTile;
    const int t = threadIdx.x;
    // forward + output delta: one thread per sample
    if (t < kGradTile) {
        const int s = s0 + t;
        float h1[H], h2[H];
        if (s < B) {
            const float y = mlp_forward(m, feat + (size_t)s * F, h1, h2);
            const float dy = 2.f * (y - label[s]) / (float)B;
            DY[t] = dy;
            atomicAdd(loss_sum, (y - label[s]) * (y - label[s]));
            for (int j = 0; j < F; j++) X[t][j] = (feat[(size_t)s * F + j] - m.mean[j]) / m.std_[j];
            for (int i = 0; i < H; i++) {
                A1[t][i] = h1[i];
                A2[t][i] = h2[i];
            }
        } else {
            DY[t] = 0.f;
            for (int j = 0; j < F; j++) X[t][j] = 0.f;
            for (int i = 0; i < H; i++) A1[t][i] = A2[t][i] = 0.f;
        }
    }
    __syncthreads();
    // delta of layer 2 pre-activations: d2_i = dy * W3_i * [h2_i > 0]
    for (int k = t; k < kGradTile * H; k += blockDim.x) {
        const int s = k / H, i = k % H;
        D2[s][i] = A2[s][i] > 0.f ? DY[s] * m.W3[i] : 0.f;
    }
    __syncthreads();
    // delta of layer 1: d1_j = (sum_i W2_ij d2_i) * [h1_j > 0]
    for (int k = t; k < kGradTile * H; k += blockDim.x) {
        const int s = k / H, j = k % H;
        float a = 0.f;
        for (int i = 0; i < H; i++) a = fmaf(m.W2[i * H + j], D2[s][i], a);
        D1[s][j] = A1[s][j] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // partial gradients of this block's samples
    for (int k = t; k < H * F; k += blockDim.x) {
        const int i = k / F, j = k % F;
        float a = 0.f;
        for (int s = 0; s < kGradTile; s++) a = fmaf(D1[s][i], X[s][j], a);
        atomicAdd(&grad[OW1 + k], a);
    }
    for (int k = t; k < H * H; k += blockDim.x) {
        const int i = k / H, j = k % H;
        float a = 0.f;
        for (int s = 0; s < kGradTile; s++) a = fmaf(D2[s][i], A1[s][j], a);
        atomicAdd(&grad[OW2 + k], a);
    }
    for (int i = t; i < H; i += blockDim.x) {
        float g1 = 0.f, g2 = 0.f, g3 = 0.f;
        for (int s = 0; s < kGradTile; s++) {
            g1 += D1[s][i];
            g2 += D2[s][i];
            g3 = fmaf(DY[s], A2[s][i], g3);
        }
        atomicAdd(&grad[OB1 + i], g1);
        atomicAdd(&grad[OB2 + i], g2);
        atomicAdd(&grad[OW3 + i], g3);
    }
    if (t == 0) {
        float g = 0.f;
        for (int s = 0; s < kGradTile; s++) g += DY[s];
        atomicAdd(&grad[OB3], g);
    }
}

// Adam (Kingma & Ba 2015) on the trained parameters; FP32 master weights.
__global__ void k_adam(float *params, const float *grad, float *m1, float *m2, int count, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float v = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = v;
        params[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

cudaError_t launch_mlp_predict(const float *params, const float *feat, int64_t n, float *out, int sm_count,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 127) / 128;
    if (blocks > (int64_t)sm_count * 16) blocks = (int64_t)sm_count * 16;
    k_mlp_predict<<<(unsigned)blocks, 128, 0, s>>>(params, feat, n, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float *params, const float *feat, const float *label, int B, float *grad,
                            float *loss_sum, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(grad, 0, NTRAIN * sizeof(float), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(loss_sum, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (B <= 0) return cudaSuccess;
    k_mlp_grad<<<(B + kGradTile - 1) / kGradTile, 128, 0, s>>>(params, feat, label, B, grad, loss_sum);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam(float *params, const float *grad, float *m1, float *m2, float lr, int step,
                        cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(NTRAIN + 255) / 256, 256, 0, s>>>(params, grad, m1, m2, NTRAIN, lr, b1, b2, eps, c1, c2);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mce

// ------------------------------------------------------------ model ABI

struct mce_model {
    float *buf = nullptr;  // params | grad | m1 | m2 | loss
    float *params = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *loss = nullptr;
    int step = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mce_allocator alloc{};
    bool has_alloc = false;
};

using mce::kModelParams;

const float *mce::model_params(const mce_model *m) { return m->params; }

static int model_fail(int code, const char *what, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    else snprintf(buf, sizeof buf, "%s", what);
    return mce::set_last_error(code, buf);
}

extern "C" int mce_model_create(const float *params, const mce_allocator *alloc, void *stream, mce_model **out) {
    if (!out || !params) return model_fail(MCE_EINVAL, "NULL argument");
    *out = nullptr;
    for (int i = mce::OMEAN + mce::F; i < kModelParams; i++)
        if (!(params[i] > 0.f)) return model_fail(MCE_EINVAL, "standardisation std must be > 0");
    if (alloc && (!alloc->alloc || !alloc->free)) return model_fail(MCE_EINVAL, "allocator without alloc/free");
    mce_model *m = new mce_model();
    cudaError_t e = cudaSuccess;
    int dev = 0;
    if (stream) {
        m->stream = (cudaStream_t)stream;
    } else if ((e = cudaStreamCreateWithFlags(&m->stream, cudaStreamDefault)) != cudaSuccess) {
        delete m;
        return model_fail(MCE_ECUDA, "cudaStreamCreate", e);
    } else {
        m->own_stream = true;
    }
    if (alloc) {
        m->alloc = *alloc;
        m->has_alloc = true;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
    const size_t words = (size_t)kModelParams + 3 * (size_t)mce::NTRAIN + 8;
    if (m->has_alloc) {
        m->buf = (float *)m->alloc.alloc(words * sizeof(float), m->alloc.ctx);
    } else if (cudaMallocAsync((void **)&m->buf, words * sizeof(float), m->stream) != cudaSuccess) {
        cudaGetLastError();
        m->buf = nullptr;
    }
    if (!m->buf) {
        if (m->own_stream) cudaStreamDestroy(m->stream);
        delete m;
        return model_fail(MCE_ENOMEM, "model allocation failed");
    }
    m->params = m->buf;
    m->grad = m->params + kModelParams;
    m->m1 = m->grad + mce::NTRAIN;
    m->m2 = m->m1 + mce::NTRAIN;
    m->loss = m->m2 + mce::NTRAIN;
    if ((e = cudaMemcpyAsync(m->params, params, kModelParams * sizeof(float), cudaMemcpyHostToDevice, m->stream)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(m->grad, 0, (3 * (size_t)mce::NTRAIN + 8) * sizeof(float), m->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
        mce_model_destroy(m);
        return model_fail(MCE_ECUDA, "model upload", e);
    }
    *out = m;
    return MCE_OK;
}

extern "C" int mce_model_get_params(const mce_model *m, float *params) {
    if (!m || !params) return model_fail(MCE_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(params, m->params, kModelParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? MCE_OK : model_fail(MCE_ECUDA, "copy", e);
}

extern "C" int mce_model_predict(mce_model *m, const float *feat, int64_t n, float *out) {
    if (!m || n < 0 || (n > 0 && (!feat || !out))) return model_fail(MCE_EINVAL, "bad argument");
    cudaError_t e = mce::launch_mlp_predict(m->params, feat, n, out, m->sm_count, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? MCE_OK : model_fail(MCE_ECUDA, "predict", e);
}

extern "C" int mce_model_gradient(mce_model *m, const float *feat, const float *label, int32_t batch, float *grad,
                                  float *loss) {
    if (!m || batch < 0 || (batch > 0 && (!feat || !label)) || !grad) return model_fail(MCE_EINVAL, "bad argument");
    cudaError_t e = mce::launch_mlp_grad(m->params, feat, label, batch, m->grad, m->loss, m->stream);
    float lsum = 0.f;
    std::vector<float> g(kModelParams, 0.f);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.data(), m->grad, mce::NTRAIN * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lsum, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return model_fail(MCE_ECUDA, "gradient", e);
    memcpy(grad, g.data(), kModelParams * sizeof(float));
    if (loss) *loss = batch > 0 ? lsum / (float)batch : 0.f;
    return MCE_OK;
}

extern "C" int mce_model_train_step(mce_model *m, const float *feat, const float *label, int32_t batch, float lr,
                                    float *loss) {
    if (!m || batch <= 0 || !feat || !label || !(lr > 0.f)) return model_fail(MCE_EINVAL, "bad argument");
    cudaError_t e = mce::launch_mlp_grad(m->params, feat, label, batch, m->grad, m->loss, m->stream);
    if (e == cudaSuccess) e = mce::launch_adam(m->params, m->grad, m->m1, m->m2, lr, ++m->step, m->stream);
    if (e == cudaSuccess && loss) {
        float lsum = 0.f;
        e = cudaMemcpyAsync(&lsum, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        *loss = lsum / (float)batch;
    }
    return e == cudaSuccess ? MCE_OK : model_fail(MCE_ECUDA, "train step", e);
}

extern "C" void mce_model_destroy(mce_model *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);  // before the memory goes back to the allocator
    if (m->buf) {
        if (m->has_alloc) m->alloc.free(m->buf, m->alloc.ctx);
        else cudaFreeAsync(m->buf, m->stream);
    }
    cudaStreamSynchronize(m->stream);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}
