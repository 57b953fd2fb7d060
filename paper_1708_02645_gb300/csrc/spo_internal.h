// Internal declarations shared by the host API (spo_api.cu) and the kernels
// (spo_eval.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spo.h"

struct spo_set {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    int64_t N = 0;     // orbitals
    int64_t Np = 0;    // padded orbital stride of the table (multiple of 8)
    spo_dtype storage = SPO_F32;
    void *table = nullptr;       // [nx][ny][nz][Np] of the storage type
    size_t table_bytes = 0;

    // staging for spo_eval_host: two streams, each with its own device
    // buffers for one chunk of positions and outputs
    cudaStream_t hstream[2] = {nullptr, nullptr};
    cudaEvent_t hevent[2] = {nullptr, nullptr};
    float *hpos[2] = {nullptr, nullptr};
    float *hout[2] = {nullptr, nullptr};
    size_t hpos_cap = 0, hout_cap = 0;   // bytes per buffer
};

namespace spo_detail {

// Records a formatted message for spo_last_error() and returns `status`.
spo_status fail(spo_status status, const char *fmt, ...);

// Arguments of one evaluation launch.
struct EvalArgs {
    const void *table;
    int nx, ny, nz;
    int64_t N, Np;
    const float *pos;   // [P][3]
    int64_t P;
    float *out;         // [P][rows][N]
};

// Queue the evaluation kernel for `kind` on `stream`.  P must be > 0.
cudaError_t launch_eval(spo_dtype storage, spo_kind kind, const EvalArgs &args,
                        cudaStream_t stream);

// Convert `rows` rows of `N` source coefficients (src_dtype, row stride N)
// into the table layout (storage, row stride Np, zero padding).
cudaError_t launch_convert(const void *src, spo_dtype src_dtype, void *dst, spo_dtype storage,
                           int64_t rows, int64_t N, int64_t Np, cudaStream_t stream);

}  // namespace spo_detail
