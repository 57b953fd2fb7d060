// Learned surrogate of an orbital set: periodic multiresolution hashed grid
// + softplus perceptron, with value / gradient / Laplacian carried through
// the network as five channels (the function is specified in include/spo.h).
//
// Training (FP32 master parameters): each step samples uniform positions,
// asks the spline (the teacher) for their VGL, runs the forward pass with
// channels, the loss, the hand-derived backward (encode, GEMMs, softplus
// jets) and one Adam step.  The layers' products run by default on the
// tcgen05 tensor cores with BF16 operands and FP32 accumulation
// (spo_tc_gemm.cu); spo_surrogate_set_train_precision(0) runs them in FP32
// on the CUDA cores instead.  Inference (precision 1) uses an FP16
// grid and BF16 weights; its perceptron runs on the tcgen05 tensor cores
// (spo_surrogate_mma.cu); precision 0 evaluates the FP32 master parameters.
//
// Activations are stored as [P][5][width] (row = position x channel), so a
// linear layer is one GEMM over 5 P rows with the bias added to the value
// rows only.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "spo.h"
#include "spo_host.h"
#include "spo_internal.h"
#include "spo_surrogate.h"
#include "spo_surrogate_enc.cuh"
#include "spo_umma.cuh"

namespace {

using spo_detail::cuda_fail;
using spo_detail::DeviceGuard;
using spo_detail::fail;
using spo_detail::SurrLevels;
using spo_dev::level_corners;
using spo_dev::div_index;

constexpr int kMaxLayers = 8;   // weight matrices (hidden layers + output)

// ---------------------------------------------------------------------------
// encoding (level geometry and corner weights: spo_surrogate_enc.cuh)
// ---------------------------------------------------------------------------
template <typename TG>
__device__ __forceinline__ float grid_val(const TG *g, size_t i);
template <>
__device__ __forceinline__ float grid_val<float>(const float *g, size_t i) { return __ldg(g + i); }
template <>
__device__ __forceinline__ float grid_val<__half>(const __half *g, size_t i) { return __half2float(g[i]); }

// e[p][ch][l F + f]; one thread per (position, level)
template <typename TG>
__global__ void encode_fwd_kernel(const TG *__restrict__ grid, SurrLevels lv, const float *__restrict__ pos,
                                  int64_t P, float *__restrict__ e) {
    const int L = lv.levels, F = lv.features;
    const int W = L * F;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P * L;
         it += (int64_t)gridDim.x * blockDim.x) {
        int l;
        const int64_t p = div_index(it, L, l);
        float r[3] = {__ldg(pos + 3 * p), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2)};
        uint32_t slot[8];
        float cw[5][8];
        level_corners(r, lv.R[l], lv.dense[l] != 0, lv.mask, slot, cw);
        const TG *gl = grid + (size_t)l * lv.table * F;
        for (int f = 0; f < F; ++f) {
            float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float th = grid_val<TG>(gl, (size_t)slot[q] * F + f);
#pragma unroll
                for (int ch = 0; ch < 5; ++ch) acc[ch] = fmaf(cw[ch][q], th, acc[ch]);
            }
#pragma unroll
            for (int ch = 0; ch < 5; ++ch) e[(p * 5 + ch) * W + l * F + f] = acc[ch];
        }
    }
}

// g_grid[l][slot][f] += sum_ch cw[ch][q] ge[p][ch][l F + f]
__global__ void encode_bwd_kernel(SurrLevels lv, const float *__restrict__ pos, int64_t P,
                                  const float *__restrict__ ge, float *__restrict__ g_grid) {
    const int L = lv.levels, F = lv.features;
    const int W = L * F;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P * L;
         it += (int64_t)gridDim.x * blockDim.x) {
        int l;
        const int64_t p = div_index(it, L, l);
        float r[3] = {__ldg(pos + 3 * p), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2)};
        uint32_t slot[8];
        float cw[5][8];
        level_corners(r, lv.R[l], lv.dense[l] != 0, lv.mask, slot, cw);
        float *gl = g_grid + (size_t)l * lv.table * F;
        for (int f = 0; f < F; ++f) {
            float g[5];
#pragma unroll
            for (int ch = 0; ch < 5; ++ch) g[ch] = __ldg(ge + (p * 5 + ch) * W + l * F + f);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float v = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 5; ++ch) v = fmaf(cw[ch][q], g[ch], v);
                atomicAdd(gl + (size_t)slot[q] * F + f, v);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 tiled GEMMs (CUDA cores): C[i][j] = sum_k A(i, k) B(k, j)
// ---------------------------------------------------------------------------
constexpr int TM = 64, TN = 64, TK = 16;

// mode 0 (forward):   A(i,k) = X[i][k] (ld K),  B(k,j) = Wt[j][k] (ld K);  C[i][j] (ld N) = . + bias on value rows
// mode 1 (back data): A(i,k) = G[i][k] (ld K),  B(k,j) = Wt[k][j] (ld N);  C[i][j]
// mode 2 (weights):   A(i,k) = G[k][i] (ld M),  B(k,j) = X[k][j] (ld N);  C[i][j] += (split-K, atomics)
// BF16 (mode 0 only): A rounded to BF16, B read as BF16.
template <int MODE, bool BF16>
__global__ void __launch_bounds__(256)
gemm_kernel(const float *__restrict__ A, const void *__restrict__ Bv, float *__restrict__ C,
            const float *__restrict__ bias, int M, int N, int K, int lda, int ldb, int k_chunk) {
    __shared__ float As[TK][TM + 1];
    __shared__ float Bs[TK][TN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;   // row tiles on x: 5 P rows can exceed 65535 tiles
    const int kbeg = blockIdx.z * k_chunk, kend = min(K, kbeg + k_chunk);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int ii = e / TK, kk = e % TK;   // (used by modes 0 and 1)
            int i, k;
            float v = 0.0f;
            if (MODE == 2) {
                const int ii2 = e % TM, kk2 = e / TM;
                i = i0 + ii2;
                k = k0 + kk2;
                if (i < M && k < kend) v = __ldg(A + (int64_t)k * lda + i);
                As[kk2][ii2] = v;
            } else {
                i = i0 + ii;
                k = k0 + kk;
                if (i < M && k < kend) v = __ldg(A + (int64_t)i * lda + k);
                if (BF16) v = __bfloat162float(__float2bfloat16_rn(v));
                As[kk][ii] = v;
            }
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            float v = 0.0f;
            if (MODE == 0) {
                const int jj = e / TK, kk = e % TK;
                const int j = j0 + jj, k = k0 + kk;
                if (j < N && k < kend)
                    v = BF16 ? __bfloat162float(static_cast<const __nv_bfloat16 *>(Bv)[(int64_t)j * ldb + k])
                             : __ldg(static_cast<const float *>(Bv) + (int64_t)j * ldb + k);
                Bs[kk][jj] = v;
            } else {
                const int jj = e % TN, kk = e / TN;
                const int j = j0 + jj, k = k0 + kk;
                if (j < N && k < kend) v = __ldg(static_cast<const float *>(Bv) + (int64_t)k * ldb + j);
                Bs[kk][jj] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = Bs[kk][tx * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty * 4 + u;
        if (i >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = j0 + tx * 4 + v;
            if (j >= N) continue;
            if (MODE == 2) {
                atomicAdd(C + (int64_t)i * N + j, acc[u][v]);
            } else {
                float r = acc[u][v];
                if (MODE == 0 && bias && i % 5 == 0) r += __ldg(bias + j);
                C[(int64_t)i * N + j] = r;
            }
        }
    }
}

// The same three products with 128 x 64 CTA tiles, 8 x 4 outputs per thread,
// 16-byte global and shared-memory accesses and packed FP32x2 FMA; used when
// every row length and leading dimension is a multiple of 4 floats and the
// pointers are 16-byte aligned (the scalar kernel above takes the rest).
constexpr int VM = 128, VN = 64, VK = 16;

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

template <int MODE>
__global__ void __launch_bounds__(256)
gemm_v4_kernel(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C,
               const float *__restrict__ bias, int M, int N, int K, int lda, int ldb, int k_chunk) {
    __shared__ __align__(16) float As[VK][VM + 4];
    __shared__ __align__(16) float Bs[VK][VN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;   // columns tx*4 .. +3, rows ty*8 .. +7
    const int i0 = blockIdx.x * VM, j0 = blockIdx.y * VN;
    const int kbeg = blockIdx.z * k_chunk, kend = min(K, kbeg + k_chunk);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 acc[8][2];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u][0] = acc[u][1] = make_float2(0.f, 0.f);
    for (int k0 = kbeg; k0 < kend; k0 += VK) {
        if (MODE == 2) {   // A[k][i]: rows along i
            for (int e = tid; e < VK * VM / 4; e += 256) {
                const int kk = e / (VM / 4), iq = e - kk * (VM / 4);
                const int k = k0 + kk, i = i0 + 4 * iq;
                const float4 v = (k < kend && i < M) ? ldg4(A + (int64_t)k * lda + i) : zero;
                *reinterpret_cast<float4 *>(&As[kk][4 * iq]) = v;
            }
        } else {           // A[i][k]: rows along k, stored transposed
            for (int e = tid; e < VM * VK / 4; e += 256) {
                const int ii = e / (VK / 4), kq = e - ii * (VK / 4);
                const int i = i0 + ii, k = k0 + 4 * kq;
                const float4 v = (i < M && k < kend) ? ldg4(A + (int64_t)i * lda + k) : zero;
                As[4 * kq + 0][ii] = v.x;
                As[4 * kq + 1][ii] = v.y;
                As[4 * kq + 2][ii] = v.z;
                As[4 * kq + 3][ii] = v.w;
            }
        }
        if (MODE == 0) {   // B[j][k]: rows along k, stored transposed
            for (int e = tid; e < VN * VK / 4; e += 256) {
                const int jj = e / (VK / 4), kq = e - jj * (VK / 4);
                const int j = j0 + jj, k = k0 + 4 * kq;
                const float4 v = (j < N && k < kend) ? ldg4(B + (int64_t)j * ldb + k) : zero;
                Bs[4 * kq + 0][jj] = v.x;
                Bs[4 * kq + 1][jj] = v.y;
                Bs[4 * kq + 2][jj] = v.z;
                Bs[4 * kq + 3][jj] = v.w;
            }
        } else {           // B[k][j]: rows along j
            for (int e = tid; e < VK * VN / 4; e += 256) {
                const int kk = e / (VN / 4), jq = e - kk * (VN / 4);
                const int k = k0 + kk, j = j0 + 4 * jq;
                const float4 v = (k < kend && j < N) ? ldg4(B + (int64_t)k * ldb + j) : zero;
                *reinterpret_cast<float4 *>(&Bs[kk][4 * jq]) = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < VK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][8 * ty]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][8 * ty + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float2 au = make_float2(a[u], a[u]);
                acc[u][0] = __ffma2_rn(au, b01, acc[u][0]);
                acc[u][1] = __ffma2_rn(au, b23, acc[u][1]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = i0 + 8 * ty + u;
        if (i >= M) continue;
        const float r[4] = {acc[u][0].x, acc[u][0].y, acc[u][1].x, acc[u][1].y};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = j0 + 4 * tx + v;
            if (j >= N) continue;
            if (MODE == 2) {
                atomicAdd(C + (int64_t)i * N + j, r[v]);
            } else {
                float x = r[v];
                if (MODE == 0 && bias && i % 5 == 0) x += __ldg(bias + j);
                C[(int64_t)i * N + j] = x;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// softplus with channels
// ---------------------------------------------------------------------------
// softplus(z) and its first three derivatives: sigma, sigma (1 - sigma),
// sigma (1 - sigma) (1 - 2 sigma).  One exponential e = exp(-|z|) serves the
// softplus and both tails of the sigmoid: with r = 1 / (1 + e), sigma is r
// for z >= 0 and e r below, and 1 - sigma the other one (so 1 - sigma is
// formed without cancellation for large z).
__device__ __forceinline__ void softplus_d(float z, float &sp, float &d1, float &d2, float &d3) {
    const float e = expf(-fabsf(z));
    const float r = 1.0f / (1.0f + e), er = e * r;
    sp = fmaxf(z, 0.0f) + log1pf(e);
    const float s1 = z >= 0.0f ? r : er, s0 = z >= 0.0f ? er : r;
    d1 = s1;
    d2 = s1 * s0;
    d3 = d2 * (s0 - s1);
}

// h = the five channels of softplus(z) for one unit: value, gradient, Laplacian
__device__ __forceinline__ void act_fwd_one(const float *zp, int64_t W, float (&h)[5]) {
    float sp, d1, d2, d3;
    softplus_d(zp[0], sp, d1, d2, d3);
    const float gx = zp[W], gy = zp[2 * W], gz = zp[3 * W], lz = zp[4 * W];
    h[0] = sp;
    h[1] = d1 * gx;
    h[2] = d1 * gy;
    h[3] = d1 * gz;
    h[4] = d2 * (gx * gx + gy * gy + gz * gz) + d1 * lz;
}

// o = d loss / d z for one unit, from z and g = d loss / d h
__device__ __forceinline__ void act_bwd_one(const float *zp, const float *gp, int64_t W, float (&o)[5]) {
    float sp, d1, d2, d3;
    softplus_d(zp[0], sp, d1, d2, d3);
    const float zx = zp[W], zy = zp[2 * W], zz = zp[3 * W], zl = zp[4 * W];
    const float g0 = gp[0], gxv = gp[W], gyv = gp[2 * W], gzv = gp[3 * W], gl = gp[4 * W];
    const float g2 = zx * zx + zy * zy + zz * zz;
    o[0] = g0 * d1 + (gxv * zx + gyv * zy + gzv * zz) * d2 + gl * (d3 * g2 + d2 * zl);
    o[1] = gxv * d1 + 2.0f * gl * d2 * zx;
    o[2] = gyv * d1 + 2.0f * gl * d2 * zy;
    o[3] = gzv * d1 + 2.0f * gl * d2 * zz;
    o[4] = gl * d1;
}

__global__ void act_fwd_kernel(const float *__restrict__ z, float *__restrict__ h, int64_t P, int W) {
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P * W;
         it += (int64_t)gridDim.x * blockDim.x) {
        int j;
        const int64_t p = div_index(it, W, j);
        float o[5];
        act_fwd_one(z + p * 5 * W + j, W, o);
        float *hp = h + p * 5 * W + j;
#pragma unroll
        for (int c = 0; c < 5; ++c) hp[c * W] = o[c];
    }
}

__global__ void act_bwd_kernel(const float *__restrict__ z, const float *__restrict__ g,
                               float *__restrict__ gz, int64_t P, int W) {
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P * W;
         it += (int64_t)gridDim.x * blockDim.x) {
        int j;
        const int64_t p = div_index(it, W, j);
        float o[5];
        act_bwd_one(z + p * 5 * W + j, g + p * 5 * W + j, W, o);
        float *op = gz + p * 5 * W + j;
#pragma unroll
        for (int c = 0; c < 5; ++c) op[c * W] = o[c];
    }
}

struct ChannelWeights {
    float w[5];
};

// Fused forms for the tensor-core training, over a block of 16 positions
// (80 rows of [5 P][W]) x 64 units: MODE kActFwd, the activation of z;
// kActBwd, its backward from z and g = d loss / d h; kLoss, the loss
// gradient 2 w_c (z - g) / (P W) of the network output z against the target
// g, with the loss sum_c w_c mean((z - g)^2) added to *loss.  The block's
// result is staged in shared memory and written straight out as both BF16
// operand images (direct: rows = the 5 P rows, K = units; transposed: rows =
// units, K = the 5 P rows), with the zero padding of both images; the FP32
// result is not stored.  kActBwd and kLoss also add the block's column sums
// of the value rows to the bias gradient gb.  Blocks cover the rows
// padded to a multiple of 128 (rows past 5 P are zero) and the units padded
// to a multiple of 128 (the transposed image's rows); nbc column blocks per
// row of blocks, linear block index.
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

constexpr int kActFwd = 0, kActBwd = 1, kLoss = 2;

template <int MODE>
__global__ void __launch_bounds__(256) act_images_kernel(const float *__restrict__ z, const float *__restrict__ g,
                                                         int64_t P, int W, int64_t nbc, int64_t nblocks,
                                                         int64_t rows_pad_d, int64_t kc_n_d,
                                                         uint8_t *__restrict__ img_d, int64_t rows_pad_t,
                                                         int64_t kc_n_t, uint8_t *__restrict__ img_t,
                                                         float *__restrict__ gb, ChannelWeights cw, double *loss) {
    using spo_detail::kImgRows;
    using spo_detail::kImgTileBytes;
    __shared__ float h[80][65];
    __shared__ double red[256];
    const double inv = 1.0 / ((double)P * (double)W);
    float local = 0.0f;
    // the CTA takes blocks blockIdx.x, blockIdx.x + gridDim.x, ...
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        const int64_t br = blk / nbc;
        const int64_t p0 = br * 16, r0 = br * 80, c0 = (blk - br * nbc) * 64;
        // 16 x 64 (position, unit) pairs, 4 per thread: all their loads are
        // issued before any of their arithmetic
        float zin[4][5], gin[4][5];
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int e = threadIdx.x + 256 * it;
            const int64_t p = p0 + (e >> 6), j = c0 + (e & 63);
            const bool ok = p < P && j < W;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const int64_t at = (p * 5 + c) * W + j;
                zin[it][c] = ok ? __ldg(z + at) : 0.0f;
                if constexpr (MODE != kActFwd) gin[it][c] = ok ? __ldg(g + at) : 0.0f;
            }
        }
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int e = threadIdx.x + 256 * it;
            const int pl = e >> 6, cj = e & 63;
            const bool ok = p0 + pl < P && c0 + cj < W;
            float o[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (ok) {
                if constexpr (MODE == kActBwd) {
                    act_bwd_one(zin[it], gin[it], 1, o);
                } else if constexpr (MODE == kLoss) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) {
                        const float d = zin[it][c] - gin[it][c];
                        o[c] = (float)(2.0 * cw.w[c] * inv) * d;
                        local = fmaf(cw.w[c] * d, d, local);
                    }
                } else {
                    act_fwd_one(zin[it], 1, o);
                }
            }
#pragma unroll
            for (int c = 0; c < 5; ++c) h[pl * 5 + c][cj] = o[c];
        }
        __syncthreads();
        if constexpr (MODE != kActFwd) {
            if (threadIdx.x < 64 && c0 + threadIdx.x < W) {
                float sb = 0.0f;
                for (int pl = 0; pl < 16; ++pl) sb += h[pl * 5][threadIdx.x];
                atomicAdd(gb + c0 + threadIdx.x, sb);
            }
        }
        const int64_t KBd = kc_n_d / 8, KBt = kc_n_t / 8;
        for (int e = threadIdx.x; e < 80 * 8; e += 256) {   // direct: row r0 + r, K columns c0 + 8q ..
            const int r = e >> 3, q = e & 7;
            const int64_t row = r0 + r, kc = c0 / 8 + q;
            if (row < rows_pad_d && kc < kc_n_d) {
                const float *v = &h[r][8 * q];
                uint8_t *t = img_d + (size_t)((row / kImgRows) * KBd + kc / 8) * kImgTileBytes;
                *reinterpret_cast<uint4 *>(t + spo_dev::sw128_offset((int)(row % kImgRows), q * 8)) =
                    make_uint4(bf16x2_rn(v[0], v[1]), bf16x2_rn(v[2], v[3]), bf16x2_rn(v[4], v[5]),
                               bf16x2_rn(v[6], v[7]));
            }
        }
        for (int e = threadIdx.x; e < 64 * 10; e += 256) {   // transposed: row c0 + cc, K rows r0 + 8q ..
            const int cc = e & 63, q = e >> 6;
            const int64_t row = c0 + cc, kc = r0 / 8 + q;
            if (row < rows_pad_t && kc < kc_n_t) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = h[8 * q + k][cc];
                uint8_t *t = img_t + (size_t)((row / kImgRows) * KBt + kc / 8) * kImgTileBytes;
                *reinterpret_cast<uint4 *>(t + spo_dev::sw128_offset((int)(row % kImgRows), (int)(kc % 8) * 8)) =
                    make_uint4(bf16x2_rn(v[0], v[1]), bf16x2_rn(v[2], v[3]), bf16x2_rn(v[4], v[5]),
                               bf16x2_rn(v[6], v[7]));
            }
        }
        __syncthreads();   // h is refilled by the next block
    }
    if constexpr (MODE == kLoss) {
        red[threadIdx.x] = (double)local * inv;
        __syncthreads();
        for (int k = 128; k > 0; k >>= 1) {
            if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(loss, red[0]);
    }
}

// Both images of act_images_kernel<mode>'s result over [5 P][W]; gb: the
// bias gradient (kActBwd, kLoss); cw, loss: the loss (kLoss).
cudaError_t act_images(int mode, const float *z, const float *g, int64_t P, int W, uint8_t *img_d,
                       uint8_t *img_t, float *gb, cudaStream_t st, ChannelWeights cw = {},
                       double *loss = nullptr) {
    const int64_t M = 5 * P;
    const int64_t rp_d = (M + 127) / 128 * 128, kc_d = ((int64_t)W + 63) / 64 * 8;
    const int64_t rp_t = ((int64_t)W + 127) / 128 * 128, kc_t = (M + 63) / 64 * 8;
    const int64_t nbr = (rp_d + 79) / 80, nbc = rp_t / 64;
    const int64_t nblocks = nbr * nbc;
    const unsigned grid = (unsigned)std::min<int64_t>(nblocks, 152 * 8);
    if (mode == kActBwd)
        act_images_kernel<kActBwd><<<grid, 256, 0, st>>>(z, g, P, W, nbc, nblocks, rp_d, kc_d, img_d, rp_t, kc_t,
                                                         img_t, gb, cw, loss);
    else if (mode == kLoss)
        act_images_kernel<kLoss><<<grid, 256, 0, st>>>(z, g, P, W, nbc, nblocks, rp_d, kc_d, img_d, rp_t, kc_t,
                                                       img_t, gb, cw, loss);
    else
        act_images_kernel<kActFwd><<<grid, 256, 0, st>>>(z, nullptr, P, W, nbc, nblocks, rp_d, kc_d, img_d, rp_t,
                                                         kc_t, img_t, nullptr, cw, loss);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// loss, bias gradient, Adam, sampling, quantisation
// ---------------------------------------------------------------------------

// g = 2 w_c (out - target) / (P N) in FP32; the loss sum_c w_c mean(d^2)
// is summed per thread in FP32, per block and across blocks in FP64.
// blockIdx.y is the channel c; blocks stride over positions, threads over
// the orbitals of row (p, c).
__global__ void loss_kernel(const float *__restrict__ out, const float *__restrict__ target, int64_t P,
                            int64_t N, ChannelWeights cw, float *__restrict__ g, double *loss, int vec) {
    __shared__ double red[256];
    const int ch = blockIdx.y;
    const double inv = 1.0 / ((double)P * (double)N);
    const float w = cw.w[ch], gs = (float)(2.0 * cw.w[ch] * inv);
    float local = 0.0f;
    // the elements of channel ch, flattened over (position, orbital); with
    // vec (N % 4 == 0, 16-byte aligned buffers) four at a time
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (vec) {
        const int64_t n4 = N / 4, total = P * n4;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
            const int64_t p = e / n4;
            const int64_t at = (p * 5 + ch) * N + (e - p * n4) * 4;
            const float4 o = __ldg(reinterpret_cast<const float4 *>(out + at));
            const float4 t = __ldg(reinterpret_cast<const float4 *>(target + at));
            const float d0 = o.x - t.x, d1 = o.y - t.y, d2 = o.z - t.z, d3 = o.w - t.w;
            *reinterpret_cast<float4 *>(g + at) = make_float4(gs * d0, gs * d1, gs * d2, gs * d3);
            local = fmaf(w * d0, d0, local);
            local = fmaf(w * d1, d1, local);
            local = fmaf(w * d2, d2, local);
            local = fmaf(w * d3, d3, local);
        }
    } else {
        const int64_t total = P * N;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
            const int64_t p = e / N;
            const int64_t at = (p * 5 + ch) * N + (e - p * N);
            const float d = out[at] - target[at];
            g[at] = gs * d;
            local = fmaf(w * d, d, local);
        }
    }
    red[threadIdx.x] = (double)local * inv;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// sums of target_c^2 over positions and orbitals, per channel (pw[0..4])
__global__ void channel_power_kernel(const float *__restrict__ target, int64_t P, int64_t N,
                                     double *pw) {
    __shared__ double red[5][256];
    double local[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t row = blockIdx.x; row < P * 5; row += gridDim.x) {
        const int ch = (int)(row % 5);
        const float *t = target + row * N;
        float acc = 0.0f;
        for (int64_t j = threadIdx.x; j < N; j += blockDim.x) acc = fmaf(t[j], t[j], acc);
#pragma unroll
        for (int c = 0; c < 5; ++c)
            if (c == ch) local[c] += acc;
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) red[c][threadIdx.x] = local[c];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int c = 0; c < 5; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) atomicAdd(pw + threadIdx.x, red[threadIdx.x][0]);
}

// gb[j] += sum_p gz[p][0][j]; blockIdx.y takes a slice of the positions
__global__ void bias_grad_kernel(const float *__restrict__ gz, int64_t P, int W, float *__restrict__ gb) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= W) return;
    const int64_t per = (P + gridDim.y - 1) / gridDim.y;
    const int64_t p0 = (int64_t)blockIdx.y * per, p1 = min(P, p0 + per);
    float s = 0.0f;
    for (int64_t p = p0; p < p1; ++p) s += __ldg(gz + p * 5 * W + j);
    atomicAdd(gb + j, s);
}

__device__ __forceinline__ void adam_one(float &p, float &g, float &m, float &v, float lr, float b1, float b2,
                                         float eps, float c1, float c2) {
    const float mi = b1 * m + (1.0f - b1) * g;
    const float vi = b2 * v + (1.0f - b2) * g * g;
    m = mi;
    v = vi;
    p -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g = 0.0f;
}

// Device-side state of a training call: the learning rate, Adam's step
// count and bias corrections, and the index of the current step within the
// run of samples drawn together.  Kept on the device so that one captured
// step (a CUDA graph) serves every step of the call.
struct TrainState {
    float lr;     // the call's learning rate
    float c1, c2; // 1 - beta1^t, 1 - beta2^t of the current step
    int64_t j;    // step within the call
    int64_t k;    // step within the current run of samples
};

__global__ void train_begin_kernel(TrainState *ts, float lr) {
    ts->lr = lr;
    ts->j = 0;
    ts->k = 0;
}

// Copies the samples and spline values of step k of the run into the
// step's fixed buffers.
__global__ void stage_step_kernel(const TrainState *__restrict__ ts, const float *__restrict__ tpos,
                                  const float *__restrict__ ttarget, int64_t npos, int64_t ntgt,
                                  float *__restrict__ pos, float *__restrict__ target) {
    const int64_t k = ts->k;
    const float *sp = tpos + k * npos, *sg = ttarget + k * ntgt;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ntgt % 4 == 0 && ((reinterpret_cast<uintptr_t>(sg) | reinterpret_cast<uintptr_t>(target)) & 15u) == 0;
    if (vec) {
        for (int64_t i = i0; i < ntgt / 4; i += stride)
            reinterpret_cast<float4 *>(target)[i] = reinterpret_cast<const float4 *>(sg)[i];
    } else {
        for (int64_t i = i0; i < ntgt; i += stride) target[i] = sg[i];
    }
    for (int64_t i = i0; i < npos; i += stride) pos[i] = sp[i];
}

// The next step: its bias corrections from the call's table (formed on the
// host, in double, rounded once to float), and the next indices.
__global__ void train_tick_kernel(TrainState *ts, const float2 *__restrict__ corr) {
    const float2 c = corr[ts->j];
    ts->c1 = c.x;
    ts->c2 = c.y;
    ts->j += 1;
    ts->k += 1;
}

// One Adam step over n parameters (the gradient is zeroed for the next
// step); four per thread when the arrays are 16-byte aligned.  The rate is
// (the call's rate x lr_mult) x lr_scale, the bias corrections those of the
// step state.  lazy: a parameter whose gradient is zero in this step keeps
// its value and both moments (the sparse form for the hash grid, whose
// entries a batch touches only a few of), and a group of four such
// parameters is not read past its gradients.
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, const TrainState *__restrict__ ts, float lr_mult,
                            float lr_scale, float b1, float b2, float eps, int lazy) {
    const float lr = ts->lr * lr_mult * lr_scale, c1 = ts->c1, c2 = ts->c2;
    const bool vec = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                       reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15u) == 0;
    const int64_t n4 = vec ? n / 4 : 0;
    auto step = [&](float &pp, float &gg, float &mm, float &vv) {
        if (!lazy || gg != 0.0f) adam_one(pp, gg, mm, vv, lr, b1, b2, eps, c1, c2);
    };
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 G4 = reinterpret_cast<float4 *>(g)[i];
        if (lazy && G4.x == 0.0f && G4.y == 0.0f && G4.z == 0.0f && G4.w == 0.0f) continue;
        float4 P4 = reinterpret_cast<float4 *>(p)[i];
        float4 M4 = reinterpret_cast<float4 *>(m)[i], V4 = reinterpret_cast<float4 *>(v)[i];
        step(P4.x, G4.x, M4.x, V4.x);
        step(P4.y, G4.y, M4.y, V4.y);
        step(P4.z, G4.z, M4.z, V4.z);
        step(P4.w, G4.w, M4.w, V4.w);
        reinterpret_cast<float4 *>(p)[i] = P4;
        reinterpret_cast<float4 *>(g)[i] = G4;
        reinterpret_cast<float4 *>(m)[i] = M4;
        reinterpret_cast<float4 *>(v)[i] = V4;
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        step(p[i], g[i], m[i], v[i]);
}

// uniform positions in the unit cube, splitmix64 on (seed, counter)
// Uniform samples of a run of steps; also restarts the step state's sample
// index.
__global__ void sample_kernel(float *pos, int64_t n3, unsigned long long seed, unsigned long long base,
                              TrainState *ts) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ts->k = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (base + (unsigned long long)i + 1ull) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        pos[i] = (float)(z >> 40) * (1.0f / 16777216.0f);
    }
}

__global__ void to_half_kernel(const float *__restrict__ a, __half *__restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2half_rn(a[i]);
}

__global__ void to_bf16_kernel(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// a[i] = (2 u_i - 1) * mul (div == 0) or (2 u_i - 1) / div, u_i the 53-bit
// uniform of splitmix64(seed, counter i + 1), in FP64 rounded once to FP32
__global__ void uniform_init_kernel(float *a, int64_t n, unsigned long long seed, double mul, double div) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double v = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        a[i] = (float)(div != 0.0 ? v / div : v * mul);
    }
}

int blocks_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 16));
}

}  // namespace

// ---------------------------------------------------------------------------
// the object
// ---------------------------------------------------------------------------
struct spo_surrogate {
    int device = 0;
    spo_surrogate_spec spec{};
    int nl = 0;                      // weight matrices
    int widths[kMaxLayers + 1] = {};
    SurrLevels lv{};
    int64_t grid_n = 0;              // levels * T * F

    // FP32 master parameters, gradients and Adam moments: one flat buffer
    // each, [grid | W0 | b0 | W1 | b1 | ...]
    float *param = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t nparam = 0;
    int64_t w_off[kMaxLayers] = {}, b_off[kMaxLayers] = {};
    int64_t adam_t = 0;
    float beta1 = 0.9f, beta2 = 0.99f, eps = 1e-15f;
    float grid_lr_mult = 1.0f;   // the grid's learning rate relative to the perceptron's
    float level_lr_power = 0.0f; // level l's grid rate is further scaled by (R_0 / R_l)^power

    // inference copies
    __half *grid16 = nullptr;
    __nv_bfloat16 *w16 = nullptr;    // all weight matrices back to back
    int64_t w16_off[kMaxLayers] = {};
    int64_t w16_n = 0;

    // scratch (grown): positions, targets, per-layer activations and
    // pre-activations, two gradient buffers
    float *pos = nullptr, *target = nullptr;
    float *act[kMaxLayers + 1] = {}, *pre[kMaxLayers] = {};
    float *gbuf[2] = {};
    double *dacc = nullptr;          // loss and channel powers
    int64_t cap_P = 0;

    bool use_tc = false;   // the fused tensor-core kernel serves precision 1
    int num_sms = 0;
    spo_detail::SurrImagePlan plan{};   // its weight image
    uint8_t *wimg = nullptr;
    uint8_t *feat = nullptr;            // its encoded-feature images (grown on demand)
    size_t feat_cap = 0;

    int train_precision = 1;            // 1: training GEMMs on the tensor cores (BF16), 0: FP32
    // BF16 operand images of the tensor-core training, carved from one arena:
    // ia, ib (A-side scratch of one product), and per layer xt (X^T, kept
    // from the forward pass to the weight gradient), wd (W) and wt (W^T)
    uint8_t *img = nullptr;
    size_t img_cap = 0;
    uint8_t *ia = nullptr, *ib = nullptr;
    uint8_t *xt[kMaxLayers] = {}, *wd[kMaxLayers] = {}, *wt[kMaxLayers] = {};
    int64_t img_M = 0;                  // rows the carve-up was made for

    // samples and spline values of a run of training steps, drawn and
    // evaluated together (grown)
    float *tpos = nullptr, *ttarget = nullptr;
    int64_t tcap = 0;

    // one training step captured as a CUDA graph, replayed for every step
    // whose inputs (sizes, buffers, settings: step_key) match the capture
    TrainState *tstate = nullptr;
    float2 *corr = nullptr;      // per step of a call: 1 - beta1^t, 1 - beta2^t
    int64_t corr_cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    std::vector<uint64_t> step_key;
    bool graphs_off = false;   // a capture failed: steps run as plain launches
};

namespace {

void free_scratch(spo_surrogate *s) {
    cudaFree(s->pos);
    cudaFree(s->target);
    for (auto &a : s->act) { cudaFree(a); a = nullptr; }
    for (auto &a : s->pre) { cudaFree(a); a = nullptr; }
    for (auto &a : s->gbuf) { cudaFree(a); a = nullptr; }
    s->pos = s->target = nullptr;
    s->cap_P = 0;
    cudaFree(s->tpos);
    cudaFree(s->ttarget);
    s->tpos = s->ttarget = nullptr;
    s->tcap = 0;
}

// Room for the samples and spline values of n positions (a run of steps).
spo_status grow_teacher(spo_surrogate *s, int64_t n) {
    if (s->tcap >= n) return SPO_OK;
    cudaFree(s->tpos);
    cudaFree(s->ttarget);
    s->tpos = s->ttarget = nullptr;
    s->tcap = 0;
    cudaError_t e = cudaMalloc(&s->tpos, sizeof(float) * 3 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&s->ttarget, sizeof(float) * 5 * (size_t)n * s->spec.N);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->tpos);
        s->tpos = nullptr;
        return fail(SPO_ENOMEM, "training samples for %lld positions failed", (long long)n);
    }
    s->tcap = n;
    return SPO_OK;
}

spo_status grow_scratch(spo_surrogate *s, int64_t P) {
    if (s->cap_P >= P) return SPO_OK;
    free_scratch(s);
    const int wmax = *std::max_element(s->widths, s->widths + s->nl + 1);
    cudaError_t e = cudaMalloc(&s->pos, sizeof(float) * 3 * (size_t)P);
    if (e == cudaSuccess) e = cudaMalloc(&s->target, sizeof(float) * 5 * (size_t)P * s->spec.N);
    for (int l = 0; l <= s->nl && e == cudaSuccess; ++l)
        e = cudaMalloc(&s->act[l], sizeof(float) * 5 * (size_t)P * s->widths[l]);
    for (int l = 0; l < s->nl && e == cudaSuccess; ++l)
        e = cudaMalloc(&s->pre[l], sizeof(float) * 5 * (size_t)P * s->widths[l + 1]);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaMalloc(&s->gbuf[k], sizeof(float) * 5 * (size_t)P * wmax);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_scratch(s);
        return fail(SPO_ENOMEM, "surrogate scratch for %lld positions failed", (long long)P);
    }
    s->cap_P = P;
    return SPO_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cudaError_t gemm(int mode, bool bf16, const float *A, const void *B, float *C, const float *bias, int M,
                 int N, int K, int lda, int ldb, cudaStream_t st) {
    // vector forms: every row that is read four floats at a time is a
    // multiple of 4 long and starts 16-byte aligned
    const bool vec = !bf16 && aligned16(A) && aligned16(B) && lda % 4 == 0 && ldb % 4 == 0 &&
                     (mode == 2 ? (M % 4 == 0 && N % 4 == 0) : (K % 4 == 0 && (mode == 0 || N % 4 == 0)));
    if (vec) {
        const float *Bf = static_cast<const float *>(B);
        if (mode == 2) {
            const int tiles = ((M + VM - 1) / VM) * ((N + VN - 1) / VN);
            const int chunks = std::max(1, std::min(std::max(1, K / 256), (4 * 152 + tiles - 1) / tiles));
            const int k_chunk = ((K + chunks - 1) / chunks + VK - 1) / VK * VK;
            dim3 g((M + VM - 1) / VM, (N + VN - 1) / VN, (K + k_chunk - 1) / k_chunk);
            gemm_v4_kernel<2><<<g, 256, 0, st>>>(A, Bf, C, bias, M, N, K, lda, ldb, k_chunk);
        } else {
            dim3 g((M + VM - 1) / VM, (N + VN - 1) / VN, 1);
            if (mode == 0)
                gemm_v4_kernel<0><<<g, 256, 0, st>>>(A, Bf, C, bias, M, N, K, lda, ldb, K);
            else
                gemm_v4_kernel<1><<<g, 256, 0, st>>>(A, Bf, C, bias, M, N, K, lda, ldb, K);
        }
        return cudaGetLastError();
    }
    if (mode == 2) {
        // C[M][N] += sum over the K rows of the activations: split that range
        // across CTAs so that about four CTAs per SM run (152 SMs)
        const int tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
        const int chunks = std::max(1, std::min(std::max(1, K / 256), (4 * 152 + tiles - 1) / tiles));
        const int k_chunk = ((K + chunks - 1) / chunks + TK - 1) / TK * TK;
        dim3 g((M + TM - 1) / TM, (N + TN - 1) / TN, (K + k_chunk - 1) / k_chunk);
        gemm_kernel<2, false><<<g, 256, 0, st>>>(A, B, C, bias, M, N, K, lda, ldb, k_chunk);
    } else {
        dim3 g((M + TM - 1) / TM, (N + TN - 1) / TN, 1);
        if (mode == 0 && bf16)
            gemm_kernel<0, true><<<g, 256, 0, st>>>(A, B, C, bias, M, N, K, lda, ldb, K);
        else if (mode == 0)
            gemm_kernel<0, false><<<g, 256, 0, st>>>(A, B, C, bias, M, N, K, lda, ldb, K);
        else
            gemm_kernel<1, false><<<g, 256, 0, st>>>(A, B, C, bias, M, N, K, lda, ldb, K);
    }
    return cudaGetLastError();
}

// Operand images for the tensor-core form of the three products of each
// layer over M = 5 P rows: forward (X [M][in] and W [o][in]), weight
// gradient (gz^T and X^T, K = M) and data gradient (gz [M][o] and W^T).
cudaError_t ensure_images(spo_surrogate *s, int64_t M) {
    if (s->img_M == M && s->img) return cudaSuccess;
    auto al = [](size_t b) { return (b + 1023) & ~size_t(1023); };
    size_t a = 0, b = 0, per[kMaxLayers][3] = {};
    size_t total = 0;
    for (int l = 0; l < s->nl; ++l) {
        const int64_t in = s->widths[l], o = s->widths[l + 1];
        a = std::max({a, al(spo_detail::bf16_image_bytes(M, in)), al(spo_detail::bf16_image_bytes(o, M))});
        b = std::max(b, al(spo_detail::bf16_image_bytes(M, o)));
        per[l][0] = al(spo_detail::bf16_image_bytes(in, M));
        per[l][1] = al(spo_detail::bf16_image_bytes(o, in));
        per[l][2] = al(spo_detail::bf16_image_bytes(in, o));
        total += per[l][0] + per[l][1] + per[l][2];
    }
    total += a + b;
    if (s->img_cap < total) {
        cudaFree(s->img);
        s->img = nullptr;
        s->img_cap = 0;
        s->img_M = 0;
        const cudaError_t e = cudaMalloc(&s->img, total);
        if (e != cudaSuccess) return e;
        s->img_cap = total;
    }
    uint8_t *p = s->img;
    s->ia = p;
    p += a;
    s->ib = p;
    p += b;
    for (int l = 0; l < s->nl; ++l) {
        s->xt[l] = p;
        p += per[l][0];
        s->wd[l] = p;
        p += per[l][1];
        s->wt[l] = p;
        p += per[l][2];
    }
    s->img_M = M;
    return cudaSuccess;
}

// Z [M][o] = X [M][in] W_l^T, plus b_l on the value rows (FP32 products on
// the CUDA cores).
cudaError_t lin_forward(spo_surrogate *s, const float *X, int l, float *Z, int64_t M, cudaStream_t st) {
    const int in = s->widths[l], o = s->widths[l + 1];
    const float *W = s->param + s->w_off[l], *b = s->param + s->b_off[l];
    return gemm(0, false, X, W, Z, b, (int)M, o, in, in, in, st);
}

// dW_l [o][in] += gz [M][o]^T X [M][in] and G [M][in] = gz [M][o] W_l [o][in]
// (FP32 products on the CUDA cores).
cudaError_t lin_backward(spo_surrogate *s, const float *gz, const float *X, int l, float *G, int64_t M,
                         cudaStream_t st) {
    const int in = s->widths[l], o = s->widths[l + 1];
    float *dW = s->grad + s->w_off[l];
    const float *W = s->param + s->w_off[l];
    cudaError_t e = gemm(2, false, gz, X, dW, nullptr, o, in, (int)M, o, in, st);
    if (e == cudaSuccess) e = gemm(1, false, gz, W, G, nullptr, (int)M, in, o, o, in, st);
    return e;
}

// Forward pass with the FP32 master parameters over P positions, leaving
// activations in s->act / s->pre; the output goes to `out`.  tc: the
// layers' products on the tensor cores (BF16 operands, FP32 accumulation).
cudaError_t forward_train(spo_surrogate *s, const float *pos, int64_t P, float *out, cudaStream_t st, bool tc) {
    cudaError_t e;
    encode_fwd_kernel<float><<<blocks_for(P * s->lv.levels), 256, 0, st>>>(s->param, s->lv, pos, P,
                                                                             s->act[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (tc && (e = ensure_images(s, 5 * P)) != cudaSuccess) return e;
    for (int l = 0; l < s->nl && tc; ++l) {   // W and W^T of every layer
        const int in = s->widths[l], o = s->widths[l + 1];
        e = spo_detail::to_bf16_images(s->param + s->w_off[l], o, in, in, s->wd[l], s->wt[l], st);
        if (e != cudaSuccess) return e;
    }
    for (int l = 0; l < s->nl; ++l) {
        const int in = s->widths[l], o = s->widths[l + 1];
        float *z = (l == s->nl - 1 && out) ? out : s->pre[l];
        if (tc) {
            // layer l's input images: the encoder output's made here, the
            // others by the previous layer's fused activation
            if (l == 0) e = spo_detail::to_bf16_images(s->act[0], 5 * P, in, in, s->ia, s->xt[0], st);
            else e = cudaSuccess;
            if (e == cudaSuccess)
                e = spo_detail::tc_gemm(s->ia, s->wd[l], 5 * P, o, in, z, s->param + s->b_off[l], false, st);
            if (e == cudaSuccess && l < s->nl - 1)
                e = act_images(kActFwd, z, nullptr, P, o, s->ia, s->xt[l + 1], nullptr, st);
            if (e != cudaSuccess) return e;
            continue;
        }
        e = lin_forward(s, s->act[l], l, z, 5 * P, st);
        if (e != cudaSuccess) return e;
        if (l < s->nl - 1) {
            act_fwd_kernel<<<blocks_for(P * o), 256, 0, st>>>(z, s->act[l + 1], P, o);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t forward_fp32(spo_surrogate *s, const float *pos, int64_t P, float *out, cudaStream_t st) {
    return forward_train(s, pos, P, out, st, false);
}

spo_detail::SurrMlpView mlp_view(const spo_surrogate *s) {
    spo_detail::SurrMlpView v;
    v.nl = s->nl;
    for (int l = 0; l <= s->nl; ++l) v.widths[l] = s->widths[l];
    for (int l = 0; l < s->nl; ++l) {
        v.W[l] = s->w16 + s->w16_off[l];
        v.b[l] = s->param + s->b_off[l];
    }
    return v;
}

// FP16 grid, BF16 weights and (for the fused kernel) the weight image from
// the FP32 master parameters.
void refresh_inference(spo_surrogate *s, cudaStream_t st) {
    to_half_kernel<<<blocks_for(s->grid_n), 256, 0, st>>>(s->param, s->grid16, s->grid_n);
    for (int l = 0; l < s->nl; ++l) {
        const int64_t n = (int64_t)s->widths[l] * s->widths[l + 1];
        to_bf16_kernel<<<blocks_for(n), 256, 0, st>>>(s->param + s->w_off[l], s->w16 + s->w16_off[l], n);
    }
    if (s->use_tc) spo_detail::surrogate_write_image(mlp_view(s), s->plan, s->wimg, st);
}

// Channel weights of the loss: given, else 1 / mean(target_c^2) of `target`.
cudaError_t channel_weights_for(spo_surrogate *s, const float *target, int64_t P, const float *given,
                                ChannelWeights &cw, cudaStream_t st) {
    if (given) {
        for (int c = 0; c < 5; ++c) cw.w[c] = given[c];
        return cudaSuccess;
    }
    const int64_t N = s->spec.N;
    cudaError_t e = cudaMemsetAsync(s->dacc, 0, sizeof(double) * 8, st);
    if (e != cudaSuccess) return e;
    channel_power_kernel<<<(unsigned)std::min<int64_t>(P * 5, 152 * 8), 256, 0, st>>>(target, P, N, s->dacc);
    double pw[8];
    e = cudaMemcpyAsync(pw, s->dacc, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int c = 0; c < 5; ++c) {
        const double mean = pw[c] / ((double)P * N);
        cw.w[c] = mean > 0 ? (float)(1.0 / mean) : 1.0f;
    }
    return e;
}

// Forward, loss (into dacc[0]) and backward over P positions; the gradient
// is added to s->grad.
cudaError_t backward(spo_surrogate *s, const float *pos, const float *target, int64_t P,
                     const ChannelWeights &cw, cudaStream_t st, bool tc) {
    const int64_t N = s->spec.N;
    const int64_t M = 5 * P;
    float *out = s->gbuf[0];   // network output [P][5][N] (gbuf holds max width >= N columns)
    cudaError_t e = forward_train(s, pos, P, out, st, tc);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dacc, 0, sizeof(double), st);
    if (e == cudaSuccess && !tc) {
        const int vec = (N % 4 == 0 && aligned16(out) && aligned16(target) && aligned16(s->gbuf[1])) ? 1 : 0;
        const int64_t per_ch = vec ? P * (N / 4) : P * N;
        const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((per_ch + 255) / 256, 152 * 2));
        loss_kernel<<<dim3(bx, 5), 256, 0, st>>>(out, target, P, N, cw, s->gbuf[1], s->dacc, vec);
        e = cudaGetLastError();
    }
    // g = gbuf[gi] is d loss / d output of layer l; the two buffers alternate
    int gi = 1;
    for (int l = s->nl - 1; l >= 0 && e == cudaSuccess && tc; --l) {
        // tensor-core form: gz's two images come from the fused backward of
        // layer l's activation (which also adds the bias gradient), or, for
        // the output layer, from the loss gradient
        const int in = s->widths[l], o = s->widths[l + 1];
        float *gb = s->grad + s->b_off[l];
        if (l < s->nl - 1)
            e = act_images(kActBwd, s->pre[l], s->gbuf[gi], P, o, s->ib, s->ia, gb, st);
        else   // the output layer: loss, its gradient and the bias gradient in one pass
            e = act_images(kLoss, out, target, P, o, s->ib, s->ia, gb, st, cw, s->dacc);
        if (e == cudaSuccess)
            e = spo_detail::tc_gemm(s->ia, s->xt[l], o, in, M, s->grad + s->w_off[l], nullptr, true, st);
        if (e == cudaSuccess)   // d loss / d input of layer l
            e = spo_detail::tc_gemm(s->ib, s->wt[l], M, in, o, s->gbuf[1 - gi], nullptr, false, st);
        gi = 1 - gi;
    }
    for (int l = s->nl - 1; l >= 0 && e == cudaSuccess && !tc; --l) {
        const int o = s->widths[l + 1];
        float *gz = s->gbuf[gi];
        if (l < s->nl - 1) {   // through the softplus of layer l
            gz = s->gbuf[1 - gi];
            act_bwd_kernel<<<blocks_for(P * o), 256, 0, st>>>(s->pre[l], s->gbuf[gi], gz, P, o);
            e = cudaGetLastError();
            gi = 1 - gi;
        }
        if (e == cudaSuccess) {
            bias_grad_kernel<<<dim3((o + 127) / 128, (unsigned)std::min<int64_t>(P, 256)), 128, 0, st>>>(
                gz, P, o, s->grad + s->b_off[l]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {   // weight gradient and d loss / d input of layer l
            e = lin_backward(s, gz, s->act[l], l, s->gbuf[1 - gi], M, st);
            gi = 1 - gi;
        }
    }
    if (e == cudaSuccess) {
        encode_bwd_kernel<<<blocks_for(P * s->lv.levels), 256, 0, st>>>(s->lv, pos, P, s->gbuf[gi], s->grad);
        e = cudaGetLastError();
    }
    return e;
}

// One training step over the batch of P samples: stage step k's samples,
// forward, loss and backward, advance the step state, then Adam (the grid,
// level by level when the levels take different rates, sparse: only the
// entries the batch touched; and the perceptron, dense).
cudaError_t enqueue_step(spo_surrogate *s, int64_t P, const ChannelWeights &cw, cudaStream_t st, bool tc) {
    const int64_t npos = 3 * P, ntgt = 5 * P * s->spec.N;
    stage_step_kernel<<<blocks_for(ntgt / 4 + 1), 256, 0, st>>>(s->tstate, s->tpos, s->ttarget, npos, ntgt,
                                                                 s->pos, s->target);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = backward(s, s->pos, s->target, P, cw, st, tc);
    if (e != cudaSuccess) return e;
    train_tick_kernel<<<1, 1, 0, st>>>(s->tstate, s->corr);
    const float b1 = s->beta1, b2 = s->beta2;
    if (s->level_lr_power == 0.0f) {
        adam_kernel<<<blocks_for(s->grid_n), 256, 0, st>>>(s->param, s->grad, s->m1, s->m2, s->grid_n, s->tstate,
                                                           s->grid_lr_mult, 1.0f, b1, b2, s->eps, 1);
    } else {
        const int64_t nlev = (int64_t)s->lv.table * s->lv.features;
        for (int l = 0; l < s->lv.levels; ++l) {
            const float scale = (float)std::pow((double)s->lv.R[0] / s->lv.R[l], (double)s->level_lr_power);
            const int64_t o = l * nlev;
            adam_kernel<<<blocks_for(nlev), 256, 0, st>>>(s->param + o, s->grad + o, s->m1 + o, s->m2 + o, nlev,
                                                          s->tstate, s->grid_lr_mult, scale, b1, b2, s->eps, 1);
        }
    }
    const int64_t nm = s->nparam - s->grid_n;
    adam_kernel<<<blocks_for(nm), 256, 0, st>>>(s->param + s->grid_n, s->grad + s->grid_n, s->m1 + s->grid_n,
                                                s->m2 + s->grid_n, nm, s->tstate, 1.0f, 1.0f, b1, b2, s->eps, 0);
    return cudaGetLastError();
}

// Everything a captured step depends on: sizes, settings and the buffers
// its launches name.  A different key means a new capture.
std::vector<uint64_t> step_key(const spo_surrogate *s, int64_t P, const ChannelWeights &cw, bool tc) {
    auto bits = [](float f) { uint32_t u; memcpy(&u, &f, 4); return (uint64_t)u; };
    auto ptr = [](const void *p) { return (uint64_t)reinterpret_cast<uintptr_t>(p); };
    std::vector<uint64_t> k = {(uint64_t)P, (uint64_t)tc, bits(s->beta1), bits(s->beta2), bits(s->eps),
                               bits(s->grid_lr_mult), bits(s->level_lr_power), (uint64_t)s->img_M,
                               ptr(s->pos), ptr(s->target), ptr(s->tpos), ptr(s->ttarget), ptr(s->tstate),
                               ptr(s->param), ptr(s->grad), ptr(s->m1), ptr(s->m2), ptr(s->dacc), ptr(s->img), ptr(s->corr),
                               ptr(s->ia), ptr(s->ib), ptr(s->gbuf[0]), ptr(s->gbuf[1])};
    for (int c = 0; c < 5; ++c) k.push_back(bits(cw.w[c]));
    for (int l = 0; l <= s->nl; ++l) k.push_back(ptr(s->act[l]));
    for (int l = 0; l < s->nl; ++l) {
        k.push_back(ptr(s->pre[l]));
        k.push_back(ptr(s->xt[l]));
        k.push_back(ptr(s->wd[l]));
        k.push_back(ptr(s->wt[l]));
    }
    return k;
}

// Runs one training step: a replay of the captured step when it matches
// (capturing it first when it does not), plain launches when capture is
// not possible.
cudaError_t run_step(spo_surrogate *s, int64_t P, const ChannelWeights &cw, cudaStream_t st, bool tc,
                     bool replay) {
    if (!replay || s->graphs_off) return enqueue_step(s, P, cw, st, tc);
    std::vector<uint64_t> key = step_key(s, P, cw, tc);
    if (!s->step_exec || key != s->step_key) {
        if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
        s->step_exec = nullptr;
        if (!s->cap_stream && cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s->graphs_off = true;
            return enqueue_step(s, P, cw, st, tc);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t eq = enqueue_step(s, P, cw, s->cap_stream, tc);
            e = cudaStreamEndCapture(s->cap_stream, &g);
            if (e == cudaSuccess) e = eq;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->step_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {   // not capturable here: plain launches from now on
            cudaGetLastError();
            s->step_exec = nullptr;
            s->graphs_off = true;
            return enqueue_step(s, P, cw, st, tc);
        }
        s->step_key = std::move(key);
    }
    return cudaGraphLaunch(s->step_exec, st);
}



}  // namespace

namespace spo_detail {

// Inference forward on the CUDA cores (FP16 grid, BF16 weights and layer
// inputs, FP32 accumulation): the reading the fused tensor-core kernel
// follows, used for networks that kernel does not serve.
cudaError_t surrogate_forward_inference(spo_surrogate *s, const float *pos, int64_t P, float *out,
                                        cudaStream_t st) {
    cudaError_t e;
    encode_fwd_kernel<__half><<<blocks_for(P * s->lv.levels), 256, 0, st>>>(s->grid16, s->lv, pos, P,
                                                                              s->act[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int M = (int)(5 * P);
    for (int l = 0; l < s->nl; ++l) {
        const int in = s->widths[l], o = s->widths[l + 1];
        float *z = (l == s->nl - 1) ? out : s->pre[l];
        e = gemm(0, true, s->act[l], s->w16 + s->w16_off[l], z, s->param + s->b_off[l], M, o, in, in, in, st);
        if (e != cudaSuccess) return e;
        if (l < s->nl - 1) {
            act_fwd_kernel<<<blocks_for(P * o), 256, 0, st>>>(z, s->act[l + 1], P, o);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}


}  // namespace spo_detail

extern "C" {

spo_status spo_surrogate_create(const spo_surrogate_spec *spec, uint64_t seed, spo_surrogate **out) {
    fail(SPO_OK, "");
    if (!spec || !out) return fail(SPO_EINVAL, "spec or out is NULL");
    *out = nullptr;
    if (spec->levels < 1 || spec->levels > spo_detail::kSurrMaxLevels || spec->log2_table < 4 ||
        spec->log2_table > 24 || spec->features < 1 || spec->features > 4 || spec->r_min < 2 ||
        spec->r_max < spec->r_min || spec->r_max > (1 << 20) || spec->hidden < 1 ||
        spec->hidden > 1024 || spec->layers < 1 || spec->layers > kMaxLayers - 1 || spec->N < 1 ||
        spec->N > 4096)
        return fail(SPO_EINVAL, "surrogate spec out of range");
    spo_surrogate *s = new (std::nothrow) spo_surrogate();
    if (!s) return fail(SPO_ENOMEM, "host allocation failed");
    cudaGetDevice(&s->device);
    s->spec = *spec;
    s->nl = spec->layers + 1;
    s->widths[0] = spec->levels * spec->features;
    for (int l = 1; l <= spec->layers; ++l) s->widths[l] = spec->hidden;
    s->widths[s->nl] = (int)spec->N;
    // level resolutions: floor(r_min b^l), b = (r_max / r_min)^(1 / (levels - 1))
    s->lv.levels = spec->levels;
    s->lv.features = spec->features;
    s->lv.table = 1 << spec->log2_table;
    s->lv.mask = (uint32_t)s->lv.table - 1u;
    const double b = spec->levels > 1 ? std::pow((double)spec->r_max / spec->r_min, 1.0 / (spec->levels - 1)) : 1.0;
    for (int l = 0; l < spec->levels; ++l) {
        const int R = (int)std::floor(spec->r_min * std::pow(b, l) + 1e-9);
        s->lv.R[l] = R;
        s->lv.dense[l] = (int64_t)R * R * R <= (int64_t)s->lv.table;
    }
    s->grid_n = (int64_t)spec->levels * s->lv.table * spec->features;
    int64_t off = s->grid_n, w16 = 0;
    for (int l = 0; l < s->nl; ++l) {
        s->w_off[l] = off;
        off += (int64_t)s->widths[l] * s->widths[l + 1];
        s->b_off[l] = off;
        off += s->widths[l + 1];
        s->w16_off[l] = w16;
        w16 += (int64_t)s->widths[l] * s->widths[l + 1];
    }
    s->nparam = off;
    s->w16_n = w16;
    {
        spo_detail::SurrMlpView v;
        v.nl = s->nl;
        for (int l = 0; l <= s->nl; ++l) v.widths[l] = s->widths[l];
        s->use_tc = spo_detail::surrogate_tc_supported(v, s->lv);
    }
    DeviceGuard guard(s->device);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    cudaError_t e = cudaMalloc(&s->param, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&s->grad, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&s->m1, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&s->m2, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&s->grid16, sizeof(__half) * s->grid_n);
    if (e == cudaSuccess) e = cudaMalloc(&s->w16, sizeof(__nv_bfloat16) * w16);
    if (e == cudaSuccess) e = cudaMalloc(&s->dacc, sizeof(double) * 8);
    if (e == cudaSuccess && s->use_tc) {
        spo_detail::SurrMlpView v;
        v.nl = s->nl;
        for (int l = 0; l <= s->nl; ++l) v.widths[l] = s->widths[l];
        s->plan = spo_detail::surrogate_image_plan(v);
        e = cudaMalloc(&s->wimg, s->plan.total);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->param); cudaFree(s->grad); cudaFree(s->m1); cudaFree(s->m2);
        cudaFree(s->grid16); cudaFree(s->w16); cudaFree(s->dacc); cudaFree(s->wimg);
        delete s;
        return fail(SPO_ENOMEM, "surrogate parameter allocation failed");
    }
    cudaStream_t st = nullptr;
    uniform_init_kernel<<<blocks_for(s->grid_n), 256, 0, st>>>(s->param, s->grid_n, seed, 1e-4, 0.0);
    for (int l = 0; l < s->nl; ++l) {
        const int64_t n = (int64_t)s->widths[l] * s->widths[l + 1];
        uniform_init_kernel<<<blocks_for(n), 256, 0, st>>>(s->param + s->w_off[l], n,
                                                            seed + 1 + (uint64_t)l, 0.0,
                                                            std::sqrt((double)s->widths[l]));
    }
    for (int l = 0; l < s->nl; ++l) cudaMemsetAsync(s->param + s->b_off[l], 0, sizeof(float) * s->widths[l + 1], st);
    cudaMemsetAsync(s->grad, 0, sizeof(float) * off, st);
    cudaMemsetAsync(s->m1, 0, sizeof(float) * off, st);
    cudaMemsetAsync(s->m2, 0, sizeof(float) * off, st);
    refresh_inference(s, st);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        spo_surrogate_destroy(s);
        return cuda_fail(e, "surrogate initialisation");
    }
    *out = s;
    return SPO_OK;
}

spo_status spo_surrogate_destroy(spo_surrogate *s) {
    if (!s) return SPO_OK;
    DeviceGuard guard(s->device);
    cudaDeviceSynchronize();
    free_scratch(s);
    cudaFree(s->param); cudaFree(s->grad); cudaFree(s->m1); cudaFree(s->m2);
    cudaFree(s->grid16); cudaFree(s->w16); cudaFree(s->dacc); cudaFree(s->wimg);
    cudaFree(s->feat);
    cudaFree(s->img);
    cudaFree(s->tstate);
    cudaFree(s->corr);
    if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
    return SPO_OK;
}

spo_status spo_surrogate_footprint(const spo_surrogate *s, size_t *bytes) {
    if (!s || !bytes) return fail(SPO_EINVAL, "surrogate or bytes is NULL");
    int64_t biases = 0;
    for (int l = 0; l < s->nl; ++l) biases += s->widths[l + 1];
    *bytes = sizeof(__half) * s->grid_n + sizeof(__nv_bfloat16) * s->w16_n + sizeof(float) * biases;
    return SPO_OK;
}

spo_status spo_surrogate_params(spo_surrogate *s, float *grid, float *const *W, float *const *b,
                                int to_device) {
    fail(SPO_OK, "");
    if (!s || !grid || !W || !b) return fail(SPO_EINVAL, "NULL argument");
    DeviceGuard guard(s->device);
    const cudaMemcpyKind k = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    auto cp = [&](float *dev, float *host, int64_t n) {
        return to_device ? cudaMemcpy(dev, host, sizeof(float) * n, k)
                         : cudaMemcpy(host, dev, sizeof(float) * n, k);
    };
    cudaError_t e = cp(s->param, grid, s->grid_n);
    for (int l = 0; l < s->nl && e == cudaSuccess; ++l) {
        e = cp(s->param + s->w_off[l], W[l], (int64_t)s->widths[l] * s->widths[l + 1]);
        if (e == cudaSuccess) e = cp(s->param + s->b_off[l], b[l], s->widths[l + 1]);
    }
    if (e == cudaSuccess && to_device) {
        refresh_inference(s, nullptr);
        e = cudaDeviceSynchronize();
    }
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "parameter copy");
}

spo_status spo_surrogate_eval(spo_surrogate *s, spo_kind kind, const float *pos, int64_t P, float *out,
                              int precision, void *stream) {
    fail(SPO_OK, "");
    if (!s) return fail(SPO_EINVAL, "surrogate is NULL");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL)
        return fail(SPO_EUNSUPPORTED, "the surrogate gives V or VGL");
    if (P < 0 || P > (INT64_C(1) << 26)) return fail(SPO_EINVAL, "P out of range");
    if (P == 0) return SPO_OK;
    if (!pos || !out) return fail(SPO_EINVAL, "pos or out is NULL");
    if (precision != 0 && precision != 1) return fail(SPO_EINVAL, "precision must be 0 or 1");
    DeviceGuard guard(s->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == 1 && s->use_tc) {   // encoding kernel + one fused launch
        // the fused kernel writes 32-byte vectors (N is a multiple of 16)
        if (reinterpret_cast<uintptr_t>(out) & 31u)
            return fail(SPO_EINVAL, "precision 1 needs out 32-byte aligned");
        const bool vo = kind == SPO_KIND_V;
        const size_t need = spo_detail::surrogate_feature_bytes(P, vo, s->num_sms);
        if (need > s->feat_cap) {
            cudaStreamSynchronize(st);   // the old buffer may still be read
            cudaFree(s->feat);
            s->feat = nullptr;
            s->feat_cap = 0;
            if (cudaMalloc(&s->feat, need) != cudaSuccess) {
                cudaGetLastError();
                return fail(SPO_ENOMEM, "feature buffer of %zu bytes", need);
            }
            s->feat_cap = need;
        }
        const cudaError_t e = spo_detail::surrogate_fused_tc(mlp_view(s), s->wimg, s->plan, s->grid16, s->lv, pos,
                                                             P, out, vo, s->num_sms, s->feat, st);
        return e == cudaSuccess ? SPO_OK : cuda_fail(e, "fused surrogate evaluation");
    }
    // evaluate in chunks of at most 65536 positions (bounded scratch)
    const int64_t chunk = std::min<int64_t>(P, 65536);
    spo_status rs = grow_scratch(s, chunk);
    if (rs != SPO_OK) return rs;
    const int64_t N = s->spec.N;
    cudaError_t e = cudaSuccess;
    for (int64_t p0 = 0; p0 < P && e == cudaSuccess; p0 += chunk) {
        const int64_t np = std::min(chunk, P - p0);
        float *dst = kind == SPO_KIND_VGL ? out + p0 * 5 * N : s->target;
        e = precision == 0 ? forward_fp32(s, pos + 3 * p0, np, dst, st)
                           : spo_detail::surrogate_forward_inference(s, pos + 3 * p0, np, dst, st);
        if (e == cudaSuccess && kind == SPO_KIND_V)   // value rows only
            e = cudaMemcpy2DAsync(out + p0 * N, sizeof(float) * N, s->target, sizeof(float) * 5 * N,
                                  sizeof(float) * N, np, cudaMemcpyDeviceToDevice, st);
    }
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "surrogate evaluation");
}

spo_status spo_surrogate_grad(spo_surrogate *s, const float *pos, const float *target, int64_t P,
                              const float *channel_weights, int precision, float *loss, float *grid,
                              float *const *W, float *const *b, void *stream) {
    fail(SPO_OK, "");
    if (!s || !pos || !target || !grid || !W || !b) return fail(SPO_EINVAL, "NULL argument");
    if (precision != 0 && precision != 1) return fail(SPO_EINVAL, "precision must be 0 or 1");
    if (P < 1 || P > (1 << 20)) return fail(SPO_EINVAL, "need 1 <= P <= 2^20");
    DeviceGuard guard(s->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    spo_status rs = grow_scratch(s, P);
    if (rs != SPO_OK) return rs;
    ChannelWeights cw{};
    cudaError_t e = channel_weights_for(s, target, P, channel_weights, cw, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->grad, 0, sizeof(float) * s->nparam, st);
    if (e == cudaSuccess) e = backward(s, pos, target, P, cw, st, precision == 1);
    double loss_h = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss_h, s->dacc, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grid, s->grad, sizeof(float) * s->grid_n, cudaMemcpyDeviceToHost, st);
    for (int l = 0; l < s->nl && e == cudaSuccess; ++l) {
        e = cudaMemcpyAsync(W[l], s->grad + s->w_off[l], sizeof(float) * s->widths[l] * s->widths[l + 1],
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b[l], s->grad + s->b_off[l], sizeof(float) * s->widths[l + 1],
                                cudaMemcpyDeviceToHost, st);
    }
    // training expects the gradient buffer zeroed between steps
    if (e == cudaSuccess) e = cudaMemsetAsync(s->grad, 0, sizeof(float) * s->nparam, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (loss) *loss = (float)loss_h;
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "surrogate gradient");
}

spo_status spo_surrogate_train(spo_surrogate *s, const spo_set *teacher, int64_t steps, int64_t batch,
                               float lr, const float *channel_weights, uint64_t seed, void *stream,
                               float *last_loss) {
    fail(SPO_OK, "");
    if (!s || !teacher) return fail(SPO_EINVAL, "surrogate or teacher is NULL");
    if (teacher->N != s->spec.N) return fail(SPO_EINVAL, "teacher has N = %lld, surrogate %lld",
                                             (long long)teacher->N, (long long)s->spec.N);
    if (steps < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0.0f))
        return fail(SPO_EINVAL, "need steps >= 0, 1 <= batch <= 2^20, lr > 0");
    DeviceGuard guard(s->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    spo_status rs = grow_scratch(s, batch);
    if (rs != SPO_OK) return rs;
    const int64_t P = batch;
    // The samples of `run` consecutive steps are drawn at once (the same
    // counter-based stream as one step at a time) and the spline's VGL at
    // all of them is one evaluation: about 32 positions per brick of the
    // teacher's binning instead of the few of one batch, at most 1 GiB of
    // spline values.
    const int64_t nbins = (int64_t)teacher->nbx * teacher->nby * teacher->nbz;
    const int64_t per_step = (int64_t)5 * P * s->spec.N * (int64_t)sizeof(float);
    int64_t run = std::max<int64_t>(1, (32 * nbins + P - 1) / P);
    run = std::min<int64_t>(run, std::max<int64_t>(1, (INT64_C(1) << 30) / per_step));
    run = std::max<int64_t>(1, std::min<int64_t>(run, steps));
    rs = grow_teacher(s, run * P);
    if (rs != SPO_OK) return rs;
    if (!s->tstate && cudaMalloc(&s->tstate, sizeof(TrainState)) != cudaSuccess) {
        cudaGetLastError();
        s->tstate = nullptr;
        return fail(SPO_ENOMEM, "training step state");
    }
    // Adam's bias corrections of the call's steps, as the host computes them
    if (s->corr_cap < steps) {
        cudaFree(s->corr);
        s->corr = nullptr;
        s->corr_cap = 0;
        if (cudaMalloc(&s->corr, sizeof(float2) * (size_t)std::max<int64_t>(steps, 64)) != cudaSuccess) {
            cudaGetLastError();
            return fail(SPO_ENOMEM, "training step table");
        }
        s->corr_cap = std::max<int64_t>(steps, 64);
    }
    std::vector<float2> corr((size_t)steps);
    for (int64_t j = 0; j < steps; ++j) {
        const double t = (double)(s->adam_t + j + 1);
        corr[(size_t)j] = make_float2((float)(1.0 - std::pow((double)s->beta1, t)),
                                      (float)(1.0 - std::pow((double)s->beta2, t)));
    }
    ChannelWeights cw{};
    double loss_h = 0.0;
    cudaError_t e = steps > 0 ? cudaMemcpyAsync(s->corr, corr.data(), sizeof(float2) * (size_t)steps,
                                                cudaMemcpyHostToDevice, st)
                              : cudaSuccess;
    train_begin_kernel<<<1, 1, 0, st>>>(s->tstate, lr);
    if (e == cudaSuccess) e = cudaGetLastError();
    for (int64_t step = 0; step < steps && e == cudaSuccess; ++step) {
        const int64_t k = step % run;
        if (k == 0) {   // the next run's samples and their spline values (restarts the sample index)
            const int64_t n = std::min<int64_t>(run, steps - step) * P;
            sample_kernel<<<blocks_for(3 * n), 256, 0, st>>>(s->tpos, 3 * n, seed,
                                                               (unsigned long long)step * 3 * P, s->tstate);
            const spo_status es = spo_detail::eval_queue(teacher, SPO_KIND_VGL, s->tpos, n, s->ttarget, st,
                                                         SPO_ALGO_AUTO);
            if (es != SPO_OK) {   // keep the inference copies in step with the parameters taken so far
                refresh_inference(s, st);
                cudaStreamSynchronize(st);
                return es;
            }
        }
        if (step == 0)
            e = channel_weights_for(s, s->ttarget, P, channel_weights, cw, st);
        // the first step of a call runs as plain launches (it grows the
        // scratch the captured step then names); the others replay it
        if (e == cudaSuccess) e = run_step(s, P, cw, st, s->train_precision == 1, step > 0);
        if (e == cudaSuccess) ++s->adam_t;
        if (e == cudaSuccess && step == steps - 1) {
            e = cudaMemcpyAsync(&loss_h, s->dacc, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    if (e == cudaSuccess) {
        refresh_inference(s, st);
        e = cudaStreamSynchronize(st);
    }
    if (last_loss) *last_loss = (float)loss_h;
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "surrogate training");
}

spo_status spo_surrogate_set_optimizer(spo_surrogate *s, float beta1, float beta2, float eps,
                                       float grid_lr_mult) {
    fail(SPO_OK, "");
    if (!s) return fail(SPO_EINVAL, "surrogate is NULL");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) ||
        !(grid_lr_mult > 0.0f))
        return fail(SPO_EINVAL, "need 0 <= beta1, beta2 < 1, eps > 0 and grid_lr_mult > 0");
    s->beta1 = beta1;
    s->beta2 = beta2;
    s->eps = eps;
    s->grid_lr_mult = grid_lr_mult;
    return SPO_OK;
}

spo_status spo_surrogate_set_level_lr(spo_surrogate *s, float power) {
    fail(SPO_OK, "");
    if (!s) return fail(SPO_EINVAL, "surrogate is NULL");
    if (!(power >= 0.0f && power <= 4.0f)) return fail(SPO_EINVAL, "need 0 <= power <= 4");
    s->level_lr_power = power;
    return SPO_OK;
}

spo_status spo_surrogate_set_train_precision(spo_surrogate *s, int precision) {
    fail(SPO_OK, "");
    if (!s) return fail(SPO_EINVAL, "surrogate is NULL");
    if (precision != 0 && precision != 1) return fail(SPO_EINVAL, "precision must be 0 or 1");
    s->train_precision = precision;
    return SPO_OK;
}

spo_status spo_surrogate_nparams(const spo_surrogate *s, int64_t *n) {
    if (!s || !n) return fail(SPO_EINVAL, "surrogate or n is NULL");
    *n = s->nparam;
    return SPO_OK;
}

spo_status spo_surrogate_state(spo_surrogate *s, float *params, float *m, float *v, int64_t *step,
                               int restore) {
    fail(SPO_OK, "");
    if (!s || !params || !m || !v || !step) return fail(SPO_EINVAL, "NULL argument");
    if (restore && *step < 0) return fail(SPO_EINVAL, "step must be >= 0");
    DeviceGuard guard(s->device);
    const size_t bytes = sizeof(float) * (size_t)s->nparam;
    cudaError_t e;
    if (restore) {
        e = cudaMemcpy(s->param, params, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->m1, m, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->m2, v, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            s->adam_t = *step;
            refresh_inference(s, nullptr);
            e = cudaDeviceSynchronize();
        }
    } else {
        e = cudaMemcpy(params, s->param, bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(m, s->m1, bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(v, s->m2, bytes, cudaMemcpyDeviceToHost);
        *step = s->adam_t;
    }
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "surrogate state copy");
}

}  // extern "C"
