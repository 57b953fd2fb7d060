// Internal declarations of the learned surrogate shared by its host code and
// its tensor-core perceptron.  Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spo_detail {

constexpr int kSurrMaxLevels = 32;
constexpr int kSurrMaxMats = 8;   // weight matrices (hidden layers + output)

// Level geometry of the hashed grid, passed by value to the kernels.
struct SurrLevels {
    int levels = 0, features = 0;
    int table = 0;          // entries per level (a power of two)
    uint32_t mask = 0;      // table - 1
    int R[kSurrMaxLevels] = {};
    int dense[kSurrMaxLevels] = {};   // R^3 <= table: direct indexing
};

// The inference copy of the perceptron: BF16 weights W[l] ([out][in], row
// major), FP32 biases b[l] ([out]).
struct SurrMlpView {
    int nl = 0;
    int widths[kSurrMaxMats + 1] = {};
    const __nv_bfloat16 *W[kSurrMaxMats] = {};
    const float *b[kSurrMaxMats] = {};
};

// The fused kernel streams the weights from an image in global memory: one
// block per hidden layer (128 rows in the 128-byte swizzle layout, one
// K-block for the first layer, two for the others) and one per chunk of
// kSurrOutChunk output rows (two K-blocks of 128 rows, rows past the last
// output zero), in the order the kernel uses them.
constexpr int kSurrOutChunk = 128;
constexpr int kSurrMaxLoads = 8;

struct SurrImagePlan {
    uint32_t off[kSurrMaxLoads] = {}, bytes[kSurrMaxLoads] = {};
    int nloads = 0;
    uint32_t total = 0;
};

// True when the fused tensor-core kernel serves this network: 2 features per
// level, 16..64 encoded features (a multiple of 16), hidden layers of 128,
// 1..3 hidden layers, N a multiple of 16 up to 384.
bool surrogate_tc_supported(const SurrMlpView &v, const SurrLevels &lv);

SurrImagePlan surrogate_image_plan(const SurrMlpView &v);

// Writes the weight image of v (BF16 weights) into img (plan.total bytes).
cudaError_t surrogate_write_image(const SurrMlpView &v, const SurrImagePlan &plan, uint8_t *img,
                                  cudaStream_t stream);

// Fused inference on the tcgen05 tensor cores: encoding of pos [P][3] with
// the FP16 grid ([levels][table][2]), BF16 layer inputs, FP32 accumulation;
// out is [P][5][N] FP32, or [P][N] (value channel only) when values_only.
// The encoding runs first as its own kernel, writing per tile the images of
// the first layer's operands into feat (surrogate_feature_bytes(P, ...)
// bytes); the fused kernel copies them in.
size_t surrogate_feature_bytes(int64_t P, bool values_only, int num_sms);
cudaError_t surrogate_fused_tc(const SurrMlpView &v, const uint8_t *img, const SurrImagePlan &plan,
                               const __half *grid, const SurrLevels &lv, const float *pos, int64_t P,
                               float *out, bool values_only, int num_sms, uint8_t *feat,
                               cudaStream_t stream);

// BF16 tile images of GEMM operands (tiles of 128 rows x 64 K-columns in the
// 128-byte swizzle layout, zero beyond the matrix) and the tensor-core GEMM
// that reads them (spo_tc_gemm.cu).  Tile (mt, kb) of an image with KB
// K-blocks starts at byte (mt * KB + kb) * kImgTileBytes; a 16-byte chunk (8
// K-columns) of row r sits at sw128_offset(r % kImgRows, 8 * chunk).
constexpr int kImgRows = 128, kImgK = 64;
constexpr uint32_t kImgTileBytes = kImgRows * kImgK * 2;
size_t bf16_image_bytes(int64_t rows, int64_t K);
// Both images of src, FP32 [R][C] row major with leading dimension ld, in
// one pass: img_direct the image of src (rows R, K = C), img_transposed the
// image of src^T (rows C, K = R).
cudaError_t to_bf16_images(const float *src, int64_t R, int64_t C, int64_t ld, uint8_t *img_direct,
                           uint8_t *img_transposed, cudaStream_t stream);
// C[M][N] (row major, ld N) = A B^T from the images of A [M][K] and B [N][K];
// accumulate: atomically added to C (K split across CTAs); otherwise stored,
// with bias[n] added to the rows m % 5 == 0 when bias is not null.
cudaError_t tc_gemm(const uint8_t *a_img, const uint8_t *b_img, int64_t M, int64_t N, int64_t K, float *C,
                    const float *bias, bool accumulate, cudaStream_t stream);

}  // namespace spo_detail
