// Fused inference of the surrogate on the tcgen05 tensor cores: hashed-grid
// encoding (FP16 grid) and the whole perceptron (BF16 weights, FP32
// accumulation in tensor memory) with the value / gradient / Laplacian
// channels, in one persistent kernel.
//
// Tile: 128 MMA rows = 4 lane quarters x (6 positions x 5 channels + 2 pad
// rows), i.e. 24 positions.  Row 32 q + 5 i + c holds channel c of position
// 6 q + i of the tile, so a position's five channels sit in five adjacent
// lanes of one warp and the softplus jets exchange them with shuffles.
// Every linear layer is one GEMM over the 128 rows: D[128 x n] = A[128 x k]
// W^T, A from shared memory (BF16, 128-byte swizzle), W resident in shared
// memory for the kernel's lifetime, D in tensor memory.  The epilogue of a
// hidden layer reads D (tcgen05.ld), adds the bias to the value rows,
// applies h = sp(z0), h_d = sp'(z0) z_d, h_L = sp''(z0) |z_d|^2 + sp'(z0) z_L
// and writes BF16 A for the next layer; the output layer's epilogue adds the
// bias and stores FP32 rows [P][5][N] (or the value rows only, [P][N]).
//
// Shared memory: A0 (encoded features, one 64-column K-block) 16 KB, AH
// (hidden activations, two K-blocks) 32 KB, W0 16 KB, one 32 KB block per
// hidden-to-hidden layer, the output layer N x 256 bytes: 224 KB for the
// 32-128-128-128-384 network.  Tensor memory: 512 columns (the output layer
// needs N <= 384).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "spo_batch.h"
#include "spo_surrogate.h"
#include "spo_surrogate_enc.cuh"
#include "spo_tma.cuh"
#include "spo_umma.cuh"

namespace {

using namespace spo_dev;
using spo_detail::SurrLevels;

constexpr int kThreads = 256;        // 8 warps: two per lane quarter
constexpr int kPosPerQuarter = 6;
constexpr int kTilePos = 4 * kPosPerQuarter;
constexpr int kHidden = 128;
constexpr uint32_t kBlock = 128 * 128;   // one K-block of 128 rows x 64 BF16
constexpr uint32_t kTmemCols = 512;

struct FusedArgs {
    const __half2 *grid;   // [levels][table] feature pairs
    SurrLevels lv;
    const float *pos;
    int64_t P;
    const __nv_bfloat16 *W[spo_detail::kSurrMaxMats];
    const float *b[spo_detail::kSurrMaxMats];
    int nl;                // weight matrices (2..4)
    int K0;                // encoded features (16, 32, 48 or 64)
    int N;                 // outputs (multiple of 16, <= 384)
    int values_only;       // store the value rows only ([P][N])
    float *out;
    unsigned int *status;
};

struct Layout {
    uint32_t a0, ah, w0, wh, wl, bar, slot, bytes;
};

__host__ __device__ inline Layout layout_of(int nl, int N) {
    Layout L;
    L.a0 = 0;
    L.ah = L.a0 + kBlock;
    L.w0 = L.ah + 2 * kBlock;
    L.wh = L.w0 + kBlock;                               // hidden-to-hidden layers 1 .. nl-2
    L.wl = L.wh + (uint32_t)(nl - 2) * 2 * kBlock;      // output layer: two K-blocks of N rows
    L.bar = L.wl + (uint32_t)N * 256;
    L.slot = L.bar + 8;
    L.bytes = L.bar + 16;
    return L;
}

// Copies W [n][k] (row major, BF16) into K-blocks of the 128-byte swizzle
// layout: block kb holds columns 64 kb .. 64 kb + 63 of all n rows.
__device__ void stage_weights(uint8_t *dst, const __nv_bfloat16 *W, int n, int k) {
    const int chunks = k / 8;
    for (int i = threadIdx.x; i < n * chunks; i += kThreads) {
        const int r = i / chunks, kc = i - r * chunks;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(W + (size_t)r * k) + kc);
        const int kb = kc >> 3;
        *reinterpret_cast<uint4 *>(dst + (uint32_t)kb * (uint32_t)n * 128u + sw128_offset(r, (kc & 7) * 8)) = v;
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void softplus_jet(float z, float &sp, float &d1, float &d2) {
    const float e = __expf(-fabsf(z));
    sp = fmaxf(z, 0.0f) + __logf(1.0f + e);
    const float r = __frcp_rn(1.0f + e);
    d1 = z >= 0.0f ? r : e * r;
    d2 = d1 * (1.0f - d1);
}

// Encoded features of the tile's positions into A0 (BF16, rows as above).
__device__ void encode_tile(const FusedArgs &a, uint8_t *a0, int64_t tile) {
    const int L = a.lv.levels;
    for (int item = threadIdx.x; item < kTilePos * L; item += kThreads) {
        const int pi = item / L, l = item - pi * L;
        const int64_t p = tile * kTilePos + pi;
        float acc[5][2] = {};
        if (p < a.P) {
            const float r[3] = {__ldg(a.pos + 3 * p), __ldg(a.pos + 3 * p + 1), __ldg(a.pos + 3 * p + 2)};
            uint32_t slot[8];
            float cw[5][8];
            level_corners(r, a.lv.R[l], a.lv.dense[l] != 0, a.lv.mask, slot, cw);
            const __half2 *g = a.grid + (size_t)l * a.lv.table;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 th = __half22float2(g[slot[q]]);
#pragma unroll
                for (int ch = 0; ch < 5; ++ch) {
                    acc[ch][0] = fmaf(cw[ch][q], th.x, acc[ch][0]);
                    acc[ch][1] = fmaf(cw[ch][q], th.y, acc[ch][1]);
                }
            }
        }
        const int row0 = 32 * (pi / kPosPerQuarter) + 5 * (pi % kPosPerQuarter);
#pragma unroll
        for (int ch = 0; ch < 5; ++ch)
            *reinterpret_cast<uint32_t *>(a0 + sw128_offset(row0 + ch, 2 * l)) = pack_bf16(acc[ch][0], acc[ch][1]);
    }
}

// Issue one layer: D[128 x n] = A[128 x k] W^T from the K-blocks at a and w
// (w: blocks of n_rows rows), output columns n0 .. n0 + n - 1 (chunks of at
// most 128 columns).
__device__ void issue_layer(uint32_t tmem, uint32_t a, uint32_t w, int k, int n_rows, int n0, int n) {
    for (int c0 = 0; c0 < n; c0 += 128) {
        const int nn = min(128, n - c0);
        const uint32_t idesc = umma_idesc_bf16(128, nn);
        for (int kk = 0; kk < k / 16; ++kk) {
            const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
            umma_bf16(tmem + (uint32_t)(n0 + c0), umma_desc_sw128(a + kb * kBlock + ko),
                      umma_desc_sw128(w + kb * (uint32_t)n_rows * 128u + (uint32_t)(n0 + c0) * 128u + ko),
                      idesc, kk > 0);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) surrogate_fused_kernel(const __grid_constant__ FusedArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const Layout Lo = layout_of(a.nl, a.N);
    const uint32_t s0 = smem_addr(sm);
    const uint32_t bar = s0 + Lo.bar;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc(s0 + Lo.slot, kTmemCols);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero the activation blocks (pad rows and pad columns stay zero), stage the weights
    for (uint32_t i = threadIdx.x; i < 3 * kBlock / 16; i += kThreads)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    stage_weights(sm + Lo.w0, a.W[0], kHidden, a.K0);
    for (int l = 1; l < a.nl - 1; ++l) stage_weights(sm + Lo.wh + (uint32_t)(l - 1) * 2 * kBlock, a.W[l], kHidden, kHidden);
    stage_weights(sm + Lo.wl, a.W[a.nl - 1], a.N, kHidden);
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(sm + Lo.slot);

    const int wq = warp & 3, half = warp >> 2;
    const int qi = lane / 5, ch = lane - 5 * qi;
    const bool pad = lane >= 5 * kPosPerQuarter;
    const int base = pad ? lane : 5 * qi;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * wq) << 16);
    const int row = 32 * wq + lane;
    uint32_t phase = 0;
    bool failed = false;
    const int64_t ntiles = (a.P + kTilePos - 1) / kTilePos;

    auto wait_mma = [&]() -> bool {
        const bool ok = mbar_wait_bounded(bar, phase);
        const bool bad = __syncthreads_or(!ok) != 0;
        if (!bad) phase ^= 1u;
        tc_fence_after_sync();
        return !bad;
    };

    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        encode_tile(a, sm + Lo.a0, tile);
        fence_proxy_async_smem();
        tc_fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after_sync();
            issue_layer(tmem, s0 + Lo.a0, s0 + Lo.w0, a.K0, kHidden, 0, kHidden);
            umma_commit(bar);
        }
        if (!wait_mma()) { failed = true; break; }

        for (int l = 0; l < a.nl - 1; ++l) {
            // epilogue of hidden layer l: softplus jets into AH
            const float *bias = a.b[l];
            for (int c16 = half; c16 < kHidden / 16; c16 += 2) {
                float z[16];
                tmem_ld16(lane_addr + (uint32_t)(c16 * 16), z);
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    float h[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const float zj = z[j + u] + (ch == 0 ? __ldg(bias + c16 * 16 + j + u) : 0.0f);
                        const float z0 = __shfl_sync(0xffffffffu, zj, base);
                        const float sq = zj * zj;
                        const float s1 = __shfl_sync(0xffffffffu, sq, (base + 1) & 31);
                        const float s2 = __shfl_sync(0xffffffffu, sq, (base + 2) & 31);
                        const float s3 = __shfl_sync(0xffffffffu, sq, (base + 3) & 31);
                        float sp, d1, d2;
                        softplus_jet(z0, sp, d1, d2);
                        h[u] = ch == 0 ? sp : (ch < 4 ? d1 * zj : fmaf(d2, s1 + s2 + s3, d1 * zj));
                    }
                    pk[j / 2] = pack_bf16(h[0], h[1]);
                }
                if (!pad) {
                    uint8_t *blk = sm + Lo.ah + (uint32_t)(c16 >> 2) * kBlock;
                    const int k0 = (c16 & 3) * 16;
                    *reinterpret_cast<uint4 *>(blk + sw128_offset(row, k0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4 *>(blk + sw128_offset(row, k0 + 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
            fence_proxy_async_smem();
            tc_fence_before_sync();
            __syncthreads();
            if (threadIdx.x == 0) {
                tc_fence_after_sync();
                if (l + 1 < a.nl - 1)
                    issue_layer(tmem, s0 + Lo.ah, s0 + Lo.wh + (uint32_t)l * 2 * kBlock, kHidden, kHidden, 0, kHidden);
                else
                    issue_layer(tmem, s0 + Lo.ah, s0 + Lo.wl, kHidden, a.N, 0, a.N);
                umma_commit(bar);
            }
            if (!wait_mma()) { failed = true; break; }
        }
        if (failed) break;

        // output epilogue: bias on the value rows, FP32 stores
        const int64_t p = tile * kTilePos + kPosPerQuarter * wq + qi;
        const bool store = !pad && p < a.P && (!a.values_only || ch == 0);
        const float *bias = a.b[a.nl - 1];
        float *dst = a.values_only ? a.out + p * a.N : a.out + (p * 5 + ch) * a.N;
        for (int c16 = half; c16 < a.N / 16; c16 += 2) {
            float z[16];
            tmem_ld16(lane_addr + (uint32_t)(c16 * 16), z);
            if (store) {
                if (ch == 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) z[j] += __ldg(bias + c16 * 16 + j);
                }
                float4 *d4 = reinterpret_cast<float4 *>(dst + c16 * 16);
#pragma unroll
                for (int j = 0; j < 4; ++j) __stcs(d4 + j, make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]));
            }
        }
        tc_fence_before_sync();
        __syncthreads();
    }

    if (failed) {
        if (threadIdx.x == 0) atomicOr(a.status, 1u);
        // let the MMAs in flight finish (bounded) before the memory goes away
        mbar_wait_bounded(bar, phase);
        tc_fence_before_sync();
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

namespace spo_detail {

bool surrogate_tc_supported(const SurrMlpView &v, const SurrLevels &lv) {
    if (v.nl < 2 || v.nl > 4 || lv.features != 2 || lv.levels > kSurrMaxLevels) return false;
    const int K0 = v.widths[0], N = v.widths[v.nl];
    if (K0 % 16 != 0 || K0 < 16 || K0 > 64) return false;
    for (int l = 1; l < v.nl; ++l)
        if (v.widths[l] != kHidden) return false;
    return N % 16 == 0 && N >= 16 && N <= 384;
}

cudaError_t surrogate_fused_tc(const SurrMlpView &v, const __half *grid, const SurrLevels &lv,
                               const float *pos, int64_t P, float *out, bool values_only,
                               int num_sms, cudaStream_t stream) {
    if (P <= 0) return cudaSuccess;
    FusedArgs a{};
    a.grid = reinterpret_cast<const __half2 *>(grid);
    a.lv = lv;
    a.pos = pos;
    a.P = P;
    for (int l = 0; l < v.nl; ++l) {
        a.W[l] = v.W[l];
        a.b[l] = v.b[l];
    }
    a.nl = v.nl;
    a.K0 = v.widths[0];
    a.N = v.widths[v.nl];
    a.values_only = values_only ? 1 : 0;
    a.out = out;
    cudaError_t e = device_status_address(&a.status);
    if (e != cudaSuccess) return e;
    const Layout Lo = layout_of(a.nl, a.N);
    const size_t smem = Lo.bytes + 1024;   // slack for the 1024-byte alignment of the base
    e = cudaFuncSetAttribute(surrogate_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (P + kTilePos - 1) / kTilePos;
    const int grid_x = (int)std::min<int64_t>(ntiles, num_sms > 0 ? num_sms : 148);
    surrogate_fused_kernel<<<grid_x, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace spo_detail
