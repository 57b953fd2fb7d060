// BF16 GEMM on the tcgen05 tensor cores for the surrogate's training:
// C[M][N] = A B^T with A [M][K] and B [N][K] given as BF16 tile images,
// FP32 accumulation in tensor memory, FP32 output (stored, with an optional
// bias on the value rows, or added atomically for split-K sums).
//
// Image layout: tiles of 128 rows x 64 K-columns (16 KB), tile (mt, kb) at
// byte ((mt * KB + kb) * 16384), each tile in the 128-byte swizzle layout
// of a K-major MMA operand (row r at r * 128 bytes, its 16-byte chunks
// permuted by r mod 8); rows beyond M and columns beyond K are zero, so the
// MMAs may always run on whole tiles.  to_bf16_images writes both images of
// an FP32 row-major matrix (of it and of its transpose) in one pass.
//
// GEMM: one CTA (128 threads) per 128 x 128 output tile and K range.  One
// thread streams (A, B) tile pairs with bulk copies through 3 shared-memory
// stages and issues 4 MMAs (K = 16 each) per pair; a stage is refilled once
// the MMAs that read it have completed (tcgen05.commit on the stage's
// barrier).  The 4 warps then read the 128 x 128 accumulator (one lane
// quarter each) and write C.  Waits are bounded (device status bit 0).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "spo_batch.h"
#include "spo_surrogate.h"
#include "spo_tma.cuh"
#include "spo_umma.cuh"

namespace {

using namespace spo_dev;

constexpr int kRowsT = spo_detail::kImgRows, kColsT = spo_detail::kImgK;
constexpr uint32_t kTileBytes = spo_detail::kImgTileBytes;   // 16 KB
constexpr int kMaxStages = 3;
constexpr uint32_t kStageBytes = 2 * kTileBytes;       // A and B tiles
// shared memory of a CTA with `stages` stages: the stages, then full[3],
// empty[3], done and the tensor-memory slot (64 B), plus 1 KB of alignment
constexpr uint32_t smem_bytes(int stages) { return (uint32_t)stages * kStageBytes + 64 + 1024; }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Both images of an FP32 row-major R x C matrix in one pass: img_d with
// image rows = source rows (K = C) and img_t with image rows = source
// columns (K = R).  A CTA stages one 64 x 64 block through shared memory
// (blocks cover the source padded to multiples of 128 in both directions,
// so the zero padding of both images is written too) and writes its 16-byte
// chunks of each image; the block index is linear (nbc blocks per row of
// blocks).
__global__ void __launch_bounds__(256) to_image2_kernel(const float *__restrict__ src, int64_t R, int64_t C,
                                                        int64_t ld, int64_t nbc, int64_t rows_pad_d,
                                                        int64_t kc_n_d, uint8_t *__restrict__ img_d,
                                                        int64_t rows_pad_t, int64_t kc_n_t,
                                                        uint8_t *__restrict__ img_t) {
    __shared__ float tile[64][65];
    const int64_t br = (int64_t)blockIdx.x / nbc;
    const int64_t r0 = br * 64, c0 = ((int64_t)blockIdx.x - br * nbc) * 64;
    const int tcol = threadIdx.x & 63, trow = threadIdx.x >> 6;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int r = trow + 4 * k;
        const int64_t gr = r0 + r, gc = c0 + tcol;
        tile[r][tcol] = (gr < R && gc < C) ? __ldg(src + gr * ld + gc) : 0.0f;
    }
    __syncthreads();
    const int64_t KBd = kc_n_d / 8, KBt = kc_n_t / 8;
    // direct: chunk (r, q) = image row r0 + r, K columns c0 + 8q .. c0 + 8q + 7
    for (int e = threadIdx.x; e < 512; e += 256) {
        const int r = e >> 3, q = e & 7;
        const int64_t row = r0 + r, kc = c0 / 8 + q;
        if (row < rows_pad_d && kc < kc_n_d) {
            const float *v = &tile[r][8 * q];
            uint8_t *t = img_d + (size_t)((row / kRowsT) * KBd + kc / 8) * kTileBytes;
            *reinterpret_cast<uint4 *>(t + sw128_offset((int)(row % kRowsT), q * 8)) =
                make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
        }
    }
    // transposed: chunk (cc, q) = image row c0 + cc, K rows r0 + 8q .. r0 + 8q + 7
    for (int e = threadIdx.x; e < 512; e += 256) {
        const int cc = e & 63, q = e >> 6;
        const int64_t row = c0 + cc, kc = r0 / 8 + q;
        if (row < rows_pad_t && kc < kc_n_t) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = tile[8 * q + j][cc];
            uint8_t *t = img_t + (size_t)((row / kRowsT) * KBt + kc / 8) * kTileBytes;
            *reinterpret_cast<uint4 *>(t + sw128_offset((int)(row % kRowsT), q * 8)) =
                make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
        }
    }
}

struct GemmArgs {
    const uint8_t *a, *b;
    int64_t M, N;
    int KB;            // K-blocks of 64
    int kb_per;        // K-blocks per CTA (split-K)
    float *C;
    const float *bias; // added to rows i % 5 == 0 (stored form only)
    int accumulate;    // 1: atomically add into C
    int vec;           // N % 8 == 0 and C 32-byte aligned: 256-bit stores / 128-bit atomics
    int stages;        // shared-memory stages, min(3, kb_per): short K leaves room for more CTAs per SM
    unsigned int *status;
};

__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t s0 = smem_addr(sm);
    const int kStages = g.stages;
    const uint32_t full = s0 + (uint32_t)kStages * kStageBytes, empty = full + 8 * kMaxStages,
                   done = empty + 8 * kMaxStages;
    const uint32_t slot = done + 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool leader = threadIdx.x == 0;
    const int64_t mt = blockIdx.x, nt = blockIdx.y;
    const int kb0 = blockIdx.z * g.kb_per;
    const int nkb = max(0, min(g.KB, kb0 + g.kb_per) - kb0);

    if (warp == 0) tmem_alloc(slot, 128);
    if (leader) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(sm + (slot - s0));

    bool bad = false;
    if (leader) {
        auto load = [&](int i) {   // K-block kb0 + i into stage i % kStages
            const int s = i % kStages;
            const uint32_t bar = full + 8 * s;
            const size_t kb = (size_t)(kb0 + i);
            mbar_arrive_expect_tx(bar, kStageBytes);
            bulk_load(s0 + s * kStageBytes, g.a + ((size_t)mt * g.KB + kb) * kTileBytes, kTileBytes, bar);
            bulk_load(s0 + s * kStageBytes + kTileBytes, g.b + ((size_t)nt * g.KB + kb) * kTileBytes, kTileBytes,
                      bar);
        };
        int issued = 0, waited = 0;
        for (; issued < nkb && issued < kStages; ++issued) load(issued);
        const uint32_t idesc = umma_idesc_bf16(128, 128);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % kStages;
            const uint32_t ph = (uint32_t)((i / kStages) & 1);
            if (!mbar_wait_bounded(full + 8 * s, ph)) { bad = true; break; }
            waited = i + 1;
            tc_fence_after_sync();
            const uint32_t a = s0 + s * kStageBytes, b = a + kTileBytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                umma_bf16(tmem, umma_desc_sw128(a + 32 * kk), umma_desc_sw128(b + 32 * kk), idesc,
                          (i > 0 || kk > 0) ? 1u : 0u);
            umma_commit(empty + 8 * s);
            if (issued < nkb) {   // refill this stage once its MMAs are done
                if (!mbar_wait_bounded(empty + 8 * s, ph)) { bad = true; break; }
                load(issued++);
            }
        }
        umma_commit(done);   // every MMA issued so far
        if (bad) {
            atomicOr(g.status, 1u);
            for (int i = waited; i < issued; ++i)   // let the copies in flight land
                mbar_wait_bounded(full + 8 * (i % kStages), (uint32_t)((i / kStages) & 1));
        }
    }
    const bool ok = mbar_wait_bounded(done, 0);
    const bool failed = __syncthreads_or(!ok || bad) != 0;
    tc_fence_after_sync();
    if (!failed && nkb > 0) {
        const int64_t m = mt * kRowsT + 32 * warp + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c16 = 0; c16 < 8; ++c16) {
            float z[16];
            tmem_ld16(taddr + 16 * c16, z);
            if (m >= g.M) continue;
            const int64_t n0 = nt * 128 + 16 * c16;
            float *row = g.C + m * g.N;
            const bool brow = g.bias && !g.accumulate && m % 5 == 0;
            if (g.vec && n0 + 16 <= g.N) {
                if (brow) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) z[j] += __ldg(g.bias + n0 + j);
                }
                if (g.accumulate) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(row + n0 + 4 * q),
                                     "f"(z[4 * q]), "f"(z[4 * q + 1]), "f"(z[4 * q + 2]), "f"(z[4 * q + 3])
                                     : "memory");
                } else {
#pragma unroll
                    for (int q = 0; q < 2; ++q)
                        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(row + n0 + 8 * q),
                                     "f"(z[8 * q]), "f"(z[8 * q + 1]), "f"(z[8 * q + 2]), "f"(z[8 * q + 3]),
                                     "f"(z[8 * q + 4]), "f"(z[8 * q + 5]), "f"(z[8 * q + 6]), "f"(z[8 * q + 7])
                                     : "memory");
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t n = n0 + j;
                    if (n < g.N) {
                        if (g.accumulate) atomicAdd(row + n, z[j]);
                        else row[n] = brow ? z[j] + __ldg(g.bias + n) : z[j];
                    }
                }
            }
        }
    } else if (!ok && threadIdx.x == 0) {
        atomicOr(g.status, 1u);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 128);
    }
}

}  // namespace

namespace spo_detail {

size_t bf16_image_bytes(int64_t rows, int64_t K) {
    const int64_t rp = (rows + kRowsT - 1) / kRowsT, kb = (K + kColsT - 1) / kColsT;
    return (size_t)rp * (size_t)kb * kTileBytes;
}

cudaError_t to_bf16_images(const float *src, int64_t R, int64_t C, int64_t ld, uint8_t *img_direct,
                           uint8_t *img_transposed, cudaStream_t stream) {
    if (R <= 0 || C <= 0) return cudaSuccess;
    const int64_t rp_d = (R + kRowsT - 1) / kRowsT * kRowsT, kc_d = (C + kColsT - 1) / kColsT * 8;
    const int64_t rp_t = (C + kRowsT - 1) / kRowsT * kRowsT, kc_t = (R + kColsT - 1) / kColsT * 8;
    const int64_t nbr = rp_d / 64, nbc = rp_t / 64;   // 64 x 64 blocks over the padded source
    const int64_t blocks = nbr * nbc;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    to_image2_kernel<<<(unsigned)blocks, 256, 0, stream>>>(src, R, C, ld, nbc, rp_d, kc_d, img_direct, rp_t,
                                                           kc_t, img_transposed);
    return cudaGetLastError();
}

cudaError_t tc_gemm(const uint8_t *a_img, const uint8_t *b_img, int64_t M, int64_t N, int64_t K, float *C,
                    const float *bias, bool accumulate, cudaStream_t stream) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    GemmArgs g{};
    g.a = a_img;
    g.b = b_img;
    g.M = M;
    g.N = N;
    g.KB = (int)((K + kColsT - 1) / kColsT);
    g.C = C;
    g.bias = bias;
    g.accumulate = accumulate ? 1 : 0;
    g.vec = (N % 8 == 0 && (reinterpret_cast<uintptr_t>(C) & 31u) == 0) ? 1 : 0;
    cudaError_t e = device_status_address(&g.status);
    if (e != cudaSuccess) return e;
    const int64_t mts = (M + kRowsT - 1) / kRowsT, nts = (N + 127) / 128;
    // split K (accumulating form only) so that about two CTAs per SM run
    int splits = 1;
    if (accumulate) {
        const int64_t want = std::max<int64_t>(1, (2 * 152) / std::max<int64_t>(1, mts * nts));
        splits = (int)std::min<int64_t>(want, std::max(1, g.KB / 4));
    }
    g.kb_per = (g.KB + splits - 1) / splits;
    splits = std::max(1, (g.KB + g.kb_per - 1) / g.kb_per);
    g.stages = std::min(kMaxStages, std::max(1, g.kb_per));
    e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(kMaxStages));
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)mts, (unsigned)nts, (unsigned)splits);
    tc_gemm_kernel<<<grid, 128, smem_bytes(g.stages), stream>>>(g);
    return cudaGetLastError();
}

}  // namespace spo_detail
