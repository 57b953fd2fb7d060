// Brick kernels (spo_brick.cuh) for FP32 tables.
#include "spo_brick.cuh"

namespace spo_detail {

template cudaError_t brick_eval_typed<float>(spo_kind, const spo_set *, const Workspace &, int64_t, float *,
                                           cudaStream_t);
template cudaError_t brick_ratio_typed<float>(const spo_set *, const Workspace &, int64_t, float *,
                                            const RatioArgs &, cudaStream_t);

}  // namespace spo_detail
