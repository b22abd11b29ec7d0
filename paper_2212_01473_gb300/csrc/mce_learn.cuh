// Learned work estimator: kernels and host launchers (mce_learn.cu).
#pragma once
#include "mce_internal.cuh"

namespace mce {

constexpr int kNumFeatures = MCE_NUM_FEATURES;
constexpr int kHidden = MCE_MODEL_HIDDEN;
constexpr int kModelParams = MCE_MODEL_PARAMS;

cudaError_t launch_root_features(int n, const int32_t *out_ptr, const int32_t *out_col, const int32_t *in_ptr,
                                 const int32_t *in_col, const int32_t *order, const int32_t *core_by_id,
                                 int degeneracy, int sm_count, int32_t *raw, float *feat, const int32_t *list,
                                 cudaStream_t s);
cudaError_t launch_select_roots(int n, const int32_t *outdeg, int min_p, int32_t *flags, int32_t *pos,
                                int32_t *scan_tmp, int32_t *list, cudaStream_t s);
cudaError_t launch_fill_and_scatter(int64_t n, float fill, int k, const int32_t *list, const int32_t *order,
                                    const float *pred, float *out, cudaStream_t s);
// the network's parameters on the device (for mce_predict_priority)
const float *model_params(const struct ::mce_model *m);
cudaError_t launch_mlp_predict(const float *params, const float *feat, int64_t n, float *out, int sm_count,
                               cudaStream_t s);
cudaError_t launch_mlp_grad(const float *params, const float *feat, const float *label, int B, float *grad,
                            float *loss_sum, cudaStream_t s);
cudaError_t launch_adam(float *params, const float *grad, float *m1, float *m2, float lr, int step,
                        cudaStream_t s);

}  // namespace mce
