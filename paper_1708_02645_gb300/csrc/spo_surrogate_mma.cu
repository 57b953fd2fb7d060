// Fused inference of the surrogate on the tcgen05 tensor cores: hashed-grid
// encoding (FP16 grid) and the whole perceptron (BF16 weights, FP32
// accumulation in tensor memory) with the value / gradient / Laplacian
// channels, in one persistent kernel.
//
// A tile is 128 positions, one per MMA row (tensor-memory lane).  Channel c
// of the activations is its own BF16 A operand H[c] [128 rows][128 K] in
// shared memory (128-byte swizzle), and every linear layer is one MMA group
// per channel, D_c[128 x n] = H[c] W^T, into its own tensor-memory column
// block.  A hidden layer runs in two phases so that five 128-column blocks
// never have to coexist in the 512 columns:
//   1. D_0..D_3 (value, gradient) into columns 0..511; the epilogue adds the
//      bias to D_0 and writes h0 = sp(z0), h_d = sp'(z0) z_d over H[0..3]
//      (already consumed), and parks T = sp''(z0) |z_d|^2 and sp'(z0) in
//      columns 128..383;
//   2. D_4 (Laplacian) into columns 0..127 from H[4]; the epilogue writes
//      h_L = T + sp'(z0) z_L over H[4].
// The output layer runs in chunks of 128 outputs with the operands swapped,
// D_c[128 outputs x positions] = W_chunk H[c]^T (one output per tensor-memory
// lane), the channels in rounds of as many as fit the 512 columns; a warp's
// store then writes 32 consecutive outputs of one position (128 bytes)
// instead of one 32-byte piece of 32 positions' rows.  Bias on the value
// channel.  Value-only evaluation carries channel 0 alone.
//
// Weights do not stay resident (H takes 160 KB): one thread streams them
// from an image pre-swizzled in global memory (one block per layer or output
// chunk, L2-resident) into two 32 KB stages with bulk copies, prefetching
// the next block while the current one is used.  The encoded features are
// written into K-block 0 of H[c] (the first layer's A operand).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "spo_batch.h"
#include "spo_surrogate.h"
#include "spo_surrogate_enc.cuh"
#include "spo_tma.cuh"
#include "spo_umma.cuh"

namespace {

using namespace spo_dev;
using spo_detail::SurrLevels;
using spo_detail::kSurrMaxLoads;

constexpr int kThreads = 512;        // 16 warps: 4 per tensor-memory lane quarter
constexpr int kTile = 128;           // positions per tile (MMA rows)
constexpr int kHidden = 128;
constexpr int kChunk = spo_detail::kSurrOutChunk;   // outputs per chunk (MMA rows)
static_assert(kChunk == 128, "an output chunk is one 128-row A operand");
constexpr uint32_t kBlock = 128 * 128;              // K-block: 128 rows x 64 BF16
constexpr uint32_t kChan = 2 * kBlock;              // one channel of H (K = 128)
constexpr uint32_t kStage = 2 * kBlock;             // one weight stage
constexpr uint32_t kOffStage = 5 * kChan;
constexpr uint32_t kOffBar = kOffStage + 2 * kStage;   // full[2], mma, tmem slot
constexpr uint32_t kSmemBytes = kOffBar + 64 + 1024;   // + alignment slack
constexpr uint32_t kTmemCols = 512;

struct FusedArgs {
    const __half2 *grid;   // [levels][table] feature pairs
    SurrLevels lv;
    const float *pos;
    int64_t P;
    const uint8_t *wimg;   // weight image: one block per load
    uint32_t load_off[kSurrMaxLoads], load_bytes[kSurrMaxLoads];
    int nloads;
    const float *b[spo_detail::kSurrMaxMats];
    int nl;                // weight matrices (2..4)
    int K0;                // encoded features (16..64, multiple of 16)
    int N;                 // outputs (multiple of 16, <= 384)
    int nch;               // channels carried: 5 (VGL) or 1 (V)
    int tile_pos;          // positions per tile (<= 128; the remaining MMA rows idle)
    const uint8_t *feat;   // encoded features: per (tile, channel) the 16 KB image of K-block 0
    float *out;
    unsigned int *status;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// 1 / x by the hardware approximation (x in [1, 2] here: no special cases);
// the activations it feeds are rounded to BF16.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void softplus_jet(float z, float &sp, float &d1, float &d2) {
    const float e = __expf(-fabsf(z));
    sp = fmaxf(z, 0.0f) + __logf(1.0f + e);
    const float r = rcp_approx(1.0f + e);
    d1 = z >= 0.0f ? r : e * r;
    d2 = d1 * (1.0f - d1);
}

// 8 BF16 (16 bytes) of row `row`, columns k .. k + 7 (k a multiple of 8) of
// channel block ch of H (shared-memory address sH).
__device__ __forceinline__ void store_h8(uint32_t sH, int ch, int row, int k, const float (&h)[8]) {
    const uint32_t addr = sH + (uint32_t)ch * kChan + (uint32_t)(k >> 6) * kBlock + sw128_offset(row, k & 63);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(pack_bf16(h[0], h[1])),
                 "r"(pack_bf16(h[2], h[3])), "r"(pack_bf16(h[4], h[5])), "r"(pack_bf16(h[6], h[7]))
                 : "memory");
}

// Encoded features of every position, written as the shared-memory images
// the fused kernel copies into K-block 0 of H[c]: per (tile, channel) 128
// rows of 128 bytes in the 128-byte swizzle layout, row = position within the
// tile, columns 2 l, 2 l + 1 = level l's two features (BF16).  One thread per
// (position, level); rows tile_pos .. 127 and columns >= 2 levels are never
// written (their MMA rows are never stored, their columns never read).
__global__ void encode_image_kernel(const __half2 *__restrict__ grid, SurrLevels lv, const float *__restrict__ pos,
                                    int64_t P, int tile_pos, int nch, uint8_t *__restrict__ img) {
    const int L = lv.levels;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P * L;
         it += (int64_t)gridDim.x * blockDim.x) {
        int l, row;
        const int64_t p = div_index(it, L, l);
        const int64_t tile = div_index(p, tile_pos, row);
        const float r[3] = {__ldg(pos + 3 * p), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2)};
        uint32_t slot[8];
        float cw[5][8];
        level_corners(r, lv.R[l], lv.dense[l] != 0, lv.mask, slot, cw);
        const __half2 *g = grid + (size_t)l * lv.table;
        float acc[5][2] = {};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float2 th = __half22float2(g[slot[q]]);
#pragma unroll
            for (int ch = 0; ch < 5; ++ch) {
                acc[ch][0] = fmaf(cw[ch][q], th.x, acc[ch][0]);
                acc[ch][1] = fmaf(cw[ch][q], th.y, acc[ch][1]);
            }
        }
        uint8_t *base = img + (size_t)tile * nch * kBlock;
#pragma unroll
        for (int ch = 0; ch < 5; ++ch)
            if (ch < nch)
                *reinterpret_cast<uint32_t *>(base + (uint32_t)ch * kBlock + sw128_offset(row, 2 * l)) =
                    pack_bf16(acc[ch][0], acc[ch][1]);
    }
    // the fused kernel may be scheduled once every block got here: the
    // block triggers after all its threads' writes
    __syncthreads();
    grid_dependents_launch();
}

__global__ void __launch_bounds__(kThreads, 1) surrogate_fused_kernel(const __grid_constant__ FusedArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t s0 = smem_addr(sm);
    const uint32_t sH = s0, sStage = s0 + kOffStage;
    const uint32_t full_bar = s0 + kOffBar;   // two barriers, 8 bytes apart
    const uint32_t mma_bar = s0 + kOffBar + 16;
    const uint32_t slot = s0 + kOffBar + 24;
    const uint32_t feat_bar = s0 + kOffBar + 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool leader = threadIdx.x == 0;

    const int64_t ntiles = (a.P + a.tile_pos - 1) / a.tile_pos;
    const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint64_t total_loads = (uint64_t)my_tiles * (uint64_t)a.nloads;
    uint64_t issued = 0, consumed = 0;   // weight loads (leader only)

    auto issue_load = [&](uint64_t g) {
        const int i = (int)(g % (uint64_t)a.nloads);
        const uint32_t bar = full_bar + 8u * (uint32_t)(g & 1);
        mbar_arrive_expect_tx(bar, a.load_bytes[i]);
        bulk_load(sStage + (uint32_t)(g & 1) * kStage, a.wimg + a.load_off[i], a.load_bytes[i], bar);
    };

    if (warp == 0) tmem_alloc(slot, kTmemCols);
    if (leader) {
        mbar_init(full_bar, 1);
        mbar_init(full_bar + 8, 1);
        mbar_init(mma_bar, 1);
        mbar_init(feat_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(sm + kOffBar + 24);
    if (leader)
        while (issued < total_loads && issued < 2) issue_load(issued++);
    // leader: copy a tile's encoded features into K-block 0 of H[c]
    auto issue_features = [&](int64_t tile) {
        const uint32_t bytes = (uint32_t)a.nch * kBlock;
        mbar_arrive_expect_tx(feat_bar, bytes);
        for (int c = 0; c < a.nch; ++c)
            bulk_load(sH + (uint32_t)c * kChan, a.feat + ((size_t)tile * a.nch + c) * kBlock, kBlock, feat_bar);
    };
    uint32_t feat_phase = 0;
    bool feat_pending = false;   // leader: a feature copy is in flight
    if (leader && blockIdx.x < ntiles) {
        grid_dependency_wait();   // the encoding kernel's images are complete
        issue_features(blockIdx.x);
        feat_pending = true;
    }

    const int wq = warp & 3, grp = warp >> 2;         // lane quarter, group within it
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * wq) << 16);
    const int row = 32 * wq + lane;                    // position within the tile
    uint32_t mma_phase = 0;
    bool failed = false;

    // Leader: wait for the weight block of load g (bounded).
    auto weights_ready = [&](uint64_t g) -> bool {
        return mbar_wait_bounded(full_bar + 8u * (uint32_t)(g & 1), (uint32_t)((g >> 1) & 1));
    };
    // All threads: wait for the MMA group just committed; a failure anywhere
    // (including the leader's weight wait, `leader_bad`) is seen by all.
    auto wait_mma = [&](bool leader_bad) -> bool {
        const bool ok = mbar_wait_bounded(mma_bar, mma_phase);
        const bool bad = __syncthreads_or(!ok || leader_bad) != 0;
        mma_phase ^= 1u;
        tc_fence_after_sync();
        return !bad;
    };
    // Leader: the stage of load g is free again; prefetch load g + 2 into it.
    auto release = [&](uint64_t g) {
        consumed = g + 1;
        if (g + 2 < total_loads && issued == g + 2) issue_load(issued++);
    };

    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
        {   // this tile's features (copy issued at the end of the previous tile)
            const bool ok = mbar_wait_bounded(feat_bar, feat_phase);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            feat_phase ^= 1u;
            if (leader) feat_pending = false;
        }

        for (int l = 0; l < a.nl && !failed; ++l) {
            const uint64_t g0 = (uint64_t)it * (uint64_t)a.nloads + (uint64_t)l;
            if (l < a.nl - 1) {
                // ---- hidden layer l: phase 1 (value and gradient channels)
                const int K = l == 0 ? a.K0 : kHidden;
                const uint32_t stage = sStage + (uint32_t)(g0 & 1) * kStage;
                bool bad = false;
                if (leader) {
                    tc_fence_after_sync();
                    bad = !weights_ready(g0);
                    if (!bad) {
                        for (int c = 0; c < min(a.nch, 4); ++c)
                            for (int kk = 0; kk < K / 16; ++kk) {
                                const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
                                umma_bf16(tmem + 128u * c, umma_desc_sw128(sH + c * kChan + kb * kBlock + ko),
                                          umma_desc_sw128(stage + kb * kBlock + ko), umma_idesc_bf16(128, kHidden),
                                          kk > 0);
                            }
                    }
                    umma_commit(mma_bar);
                }
                if (!wait_mma(bad)) { failed = true; break; }
                if (a.nch == 1 && leader) release(g0);

                const float *bias = a.b[l];
                for (int u = 0; u < 4; ++u) {
                    const int j0 = 32 * grp + 8 * u;   // 8 units
                    float z0[8], bb[8];
                    tmem_ld8(lane_addr + (uint32_t)j0, z0);
                    const float4 b0 = __ldg(reinterpret_cast<const float4 *>(bias + j0));
                    const float4 b1 = __ldg(reinterpret_cast<const float4 *>(bias + j0 + 4));
                    bb[0] = b0.x; bb[1] = b0.y; bb[2] = b0.z; bb[3] = b0.w;
                    bb[4] = b1.x; bb[5] = b1.y; bb[6] = b1.z; bb[7] = b1.w;
                    if (a.nch == 1) {
                        float h[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float d1, d2;
                            softplus_jet(z0[j] + bb[j], h[j], d1, d2);
                        }
                        store_h8(sH, 0, row, j0, h);
                    } else {
                        float zx[8], zy[8], zz[8];
                        tmem_ld8(lane_addr + 128u + (uint32_t)j0, zx);
                        tmem_ld8(lane_addr + 256u + (uint32_t)j0, zy);
                        tmem_ld8(lane_addr + 384u + (uint32_t)j0, zz);
                        float h0[8], t[8], d1v[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float d2;
                            softplus_jet(z0[j] + bb[j], h0[j], d1v[j], d2);
                            t[j] = d2 * fmaf(zx[j], zx[j], fmaf(zy[j], zy[j], zz[j] * zz[j]));
                            zx[j] *= d1v[j];
                            zy[j] *= d1v[j];
                            zz[j] *= d1v[j];
                        }
                        store_h8(sH, 0, row, j0, h0);
                        store_h8(sH, 1, row, j0, zx);
                        store_h8(sH, 2, row, j0, zy);
                        store_h8(sH, 3, row, j0, zz);
                        // park T and sp' in columns this thread has read (its own lane)
                        tmem_st8(lane_addr + 128u + (uint32_t)j0, t);
                        tmem_st8(lane_addr + 256u + (uint32_t)j0, d1v);
                    }
                }
                if (a.nch == 5) tmem_wait_st();
                fence_proxy_async_smem();
                tc_fence_before_sync();
                __syncthreads();

                if (a.nch == 5) {
                    // ---- phase 2 (Laplacian channel) into columns 0..127
                    if (leader) {
                        tc_fence_after_sync();
                        for (int kk = 0; kk < K / 16; ++kk) {
                            const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
                            umma_bf16(tmem, umma_desc_sw128(sH + 4 * kChan + kb * kBlock + ko),
                                      umma_desc_sw128(stage + kb * kBlock + ko), umma_idesc_bf16(128, kHidden), kk > 0);
                        }
                        umma_commit(mma_bar);
                    }
                    if (!wait_mma(false)) { failed = true; break; }
                    if (leader) release(g0);
                    for (int u = 0; u < 4; ++u) {
                        const int j0 = 32 * grp + 8 * u;
                        float zl[8], t[8], d1v[8];
                        tmem_ld8(lane_addr + (uint32_t)j0, zl);
                        tmem_ld8(lane_addr + 128u + (uint32_t)j0, t);
                        tmem_ld8(lane_addr + 256u + (uint32_t)j0, d1v);
#pragma unroll
                        for (int j = 0; j < 8; ++j) zl[j] = fmaf(d1v[j], zl[j], t[j]);
                        store_h8(sH, 4, row, j0, zl);
                    }
                    fence_proxy_async_smem();
                    tc_fence_before_sync();
                    __syncthreads();
                }
            } else {
                // ---- output layer: per chunk of 128 outputs, D_c[output][position]
                // = W_chunk H[c]^T, N = the tile's positions rounded up to 16
                const float *bias = a.b[l];
                const int np16 = (a.tile_pos + 15) & ~15;
                const int cpr = min(a.nch, (int)kTmemCols / np16);   // channels per round
                const int64_t p0 = tile * a.tile_pos;
                const int npos = (int)min((int64_t)a.tile_pos, a.P - p0);
                const int subs = (npos + 15) / 16;
                for (int n0 = 0, ci = 0; n0 < a.N && !failed; n0 += kChunk, ++ci) {
                    const uint64_t g = (uint64_t)it * (uint64_t)a.nloads + (uint64_t)(l + ci);
                    const uint32_t stage = sStage + (uint32_t)(g & 1) * kStage;
                    const int o = n0 + row;   // this thread's output: its tensor-memory lane
                    const float bo = o < a.N ? __ldg(bias + o) : 0.0f;
                    const int64_t step = (int64_t)a.nch * a.N;       // one position in out
                    float *const obase = a.out + p0 * step + o;      // position p0, channel 0
                    for (int c0 = 0; c0 < a.nch; c0 += cpr) {
                        const int nc = min(cpr, a.nch - c0);
                        bool bad = false;
                        if (leader) {
                            tc_fence_after_sync();
                            if (c0 == 0) bad = !weights_ready(g);
                            if (!bad) {
                                for (int c = 0; c < nc; ++c)
                                    for (int kk = 0; kk < kHidden / 16; ++kk) {
                                        const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
                                        umma_bf16(tmem + (uint32_t)(np16 * c),
                                                  umma_desc_sw128(stage + kb * kBlock + ko),
                                                  umma_desc_sw128(sH + (c0 + c) * kChan + kb * kBlock + ko),
                                                  umma_idesc_bf16(128, np16), kk > 0);
                                    }
                            }
                            umma_commit(mma_bar);
                        }
                        if (!wait_mma(bad)) { failed = true; break; }
                        if (c0 + nc >= a.nch) {
                            if (leader) release(g);
                            if (leader && n0 + kChunk >= a.N && tile + gridDim.x < ntiles) {
                                // H is no longer read: bring in the next tile's features
                                issue_features(tile + gridDim.x);
                                feat_pending = true;
                            }
                        }
                        for (int i = grp; i < nc * subs; i += 4) {
                            const int c = i / subs, s = i - c * subs;
                            float z[16];
                            tmem_ld16(lane_addr + (uint32_t)(np16 * c + 16 * s), z);
                            if (o < a.N) {
                                const float add = c0 + c == 0 ? bo : 0.0f;
                                float *dst = obase + (int64_t)(16 * s) * step + (int64_t)(c0 + c) * a.N;
                                if (16 * s + 16 <= npos) {   // a full group of 16 positions
#pragma unroll
                                    for (int j = 0; j < 16; ++j, dst += step) __stcs(dst, z[j] + add);
                                } else {
                                    const int jn = npos - 16 * s;
#pragma unroll
                                    for (int j = 0; j < 16; ++j, dst += step)
                                        if (j < jn) __stcs(dst, z[j] + add);
                                }
                            }
                        }
                        tc_fence_before_sync();
                        __syncthreads();
                    }
                }
            }
        }
    }

    if (failed) {
        if (leader) {
            atomicOr(a.status, 1u);
            // let the weight copies in flight land (bounded) before the memory goes away
            for (uint64_t g = consumed; g < issued; ++g) weights_ready(g);
            if (feat_pending) mbar_wait_bounded(feat_bar, feat_phase);
        }
        mbar_wait_bounded(mma_bar, mma_phase ^ 1u);   // the phase that was being waited for
        tc_fence_before_sync();
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Writes the weight image: load 0 = W0 ([128][K0], one K-block, columns
// K0..63 zero), loads 1 .. nl-2 = hidden matrices (two K-blocks), then the
// output matrix in chunks of kChunk rows (two K-blocks of 128 rows each,
// rows past the last output zero).
// One thread per 16-byte chunk of a block.
struct ImageArgs {
    const __nv_bfloat16 *W[spo_detail::kSurrMaxMats];
    uint32_t load_off[kSurrMaxLoads];
    int load_layer[kSurrMaxLoads], load_row0[kSurrMaxLoads], load_rows[kSurrMaxLoads], load_kblocks[kSurrMaxLoads];
    int load_valid[kSurrMaxLoads];   // rows taken from W; the rest are zero
    int in_width[kSurrMaxLoads];
    int nloads;
};

__global__ void weight_image_kernel(const __grid_constant__ ImageArgs ia, uint8_t *img) {
    for (int i = 0; i < ia.nloads; ++i) {
        const int rows = ia.load_rows[i], kbs = ia.load_kblocks[i], in = ia.in_width[i];
        const int valid = ia.load_valid[i];
        const __nv_bfloat16 *W = ia.W[ia.load_layer[i]];
        const int n = rows * kbs * 8;   // 16-byte chunks
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
            const int kb = e / (rows * 8), rem = e - kb * rows * 8;
            const int r = rem / 8, kc = rem - r * 8;
            const int k = kb * 64 + kc * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k < in && r < valid) v = *reinterpret_cast<const uint4 *>(W + (size_t)(ia.load_row0[i] + r) * in + k);
            *reinterpret_cast<uint4 *>(img + ia.load_off[i] + (uint32_t)kb * (uint32_t)rows * 128u +
                                       sw128_offset(r, kc * 8)) = v;
        }
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

SurrImagePlan surrogate_image_plan(const SurrMlpView &v) {
    SurrImagePlan plan{};
    uint32_t off = 0;
    int n = 0;
    for (int l = 0; l < v.nl - 1; ++l) {
        plan.off[n] = off;
        plan.bytes[n] = (l == 0 ? 1u : 2u) * kBlock;
        off += plan.bytes[n++];
    }
    const int N = v.widths[v.nl];
    for (int n0 = 0; n0 < N; n0 += kChunk) {
        plan.off[n] = off;
        plan.bytes[n] = 2u * kBlock;   // a full 128-row A operand
        off += plan.bytes[n++];
    }
    plan.nloads = n;
    plan.total = off;
    return plan;
}

cudaError_t surrogate_write_image(const SurrMlpView &v, const SurrImagePlan &plan, uint8_t *img,
                                  cudaStream_t stream) {
    ImageArgs ia{};
    for (int l = 0; l < v.nl; ++l) ia.W[l] = v.W[l];
    int n = 0;
    for (int l = 0; l < v.nl - 1; ++l, ++n) {
        ia.load_off[n] = plan.off[n];
        ia.load_layer[n] = l;
        ia.load_row0[n] = 0;
        ia.load_rows[n] = kHidden;
        ia.load_valid[n] = kHidden;
        ia.load_kblocks[n] = l == 0 ? 1 : 2;
        ia.in_width[n] = v.widths[l];
    }
    const int N = v.widths[v.nl];
    for (int n0 = 0; n0 < N; n0 += kChunk, ++n) {
        ia.load_off[n] = plan.off[n];
        ia.load_layer[n] = v.nl - 1;
        ia.load_row0[n] = n0;
        ia.load_rows[n] = kChunk;
        ia.load_valid[n] = std::min(kChunk, N - n0);
        ia.load_kblocks[n] = 2;
        ia.in_width[n] = kHidden;
    }
    ia.nloads = n;
    weight_image_kernel<<<64, 256, 0, stream>>>(ia, img);
    return cudaGetLastError();
}

size_t surrogate_feature_bytes(int64_t P, bool values_only, int num_sms) {
    const int sms = num_sms > 0 ? num_sms : 148;
    const int64_t waves = (P + (int64_t)kTile * sms - 1) / ((int64_t)kTile * sms);
    const int64_t tiles_wanted = waves * sms;
    const int64_t tile_pos = std::max<int64_t>(1, (P + tiles_wanted - 1) / tiles_wanted);
    const int64_t ntiles = (P + tile_pos - 1) / tile_pos;
    return (size_t)ntiles * (values_only ? 1 : 5) * kBlock;
}

cudaError_t surrogate_fused_tc(const SurrMlpView &v, const uint8_t *img, const SurrImagePlan &plan,
                               const __half *grid, const SurrLevels &lv, const float *pos, int64_t P,
                               float *out, bool values_only, int num_sms, uint8_t *feat,
                               cudaStream_t stream) {
    if (P <= 0) return cudaSuccess;
    FusedArgs a{};
    a.grid = reinterpret_cast<const __half2 *>(grid);
    a.lv = lv;
    a.pos = pos;
    a.P = P;
    a.wimg = img;
    for (int i = 0; i < plan.nloads; ++i) {
        a.load_off[i] = plan.off[i];
        a.load_bytes[i] = plan.bytes[i];
    }
    a.nloads = plan.nloads;
    for (int l = 0; l < v.nl; ++l) a.b[l] = v.b[l];
    a.nl = v.nl;
    a.K0 = v.widths[0];
    a.N = v.widths[v.nl];
    a.nch = values_only ? 1 : 5;
    a.out = out;
    cudaError_t e = device_status_address(&a.status);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(surrogate_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    // tiles of at most 128 positions, as many per CTA as the waves need, so
    // that every CTA gets the same number of tiles of nearly equal size
    const int sms = num_sms > 0 ? num_sms : 148;
    const int64_t waves = (P + (int64_t)kTile * sms - 1) / ((int64_t)kTile * sms);
    const int64_t tiles_wanted = waves * sms;
    a.tile_pos = (int)std::max<int64_t>(1, (P + tiles_wanted - 1) / tiles_wanted);
    const int64_t ntiles = (P + a.tile_pos - 1) / a.tile_pos;
    const int grid_x = (int)std::min<int64_t>(ntiles, sms);
    a.feat = feat;
    {
        const int64_t items = P * lv.levels;
        const int blocks = (int)std::min<int64_t>((items + 255) / 256, (int64_t)sms * 16);
        encode_image_kernel<<<blocks, 256, 0, stream>>>(a.grid, lv, pos, P, a.tile_pos, a.nch, feat);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // a programmatic dependent of the encoding: its set-up (tensor memory,
    // barriers, the first weight copies) overlaps the encoding's last blocks,
    // and the leader waits for the encoding before copying the first images
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid_x);
    cfg.blockDim = dim3((unsigned)kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, surrogate_fused_kernel, a);
}

}  // namespace spo_detail
