// Brick kernel over a batch of walkers and orbital sets: one CTA per
// (set, brick, orbital tile) unit of the whole batch.  The sets' tensor maps
// and shapes arrive in one __grid_constant__ parameter block; positions come
// as weight records in sorted order from the batch binning (its basis
// weights, formed once for every orbital tile), each with the address of its
// own output rows (every walker has its own output buffer).  The per-position
// arithmetic is the single-set brick kernel's (spo_device.cuh), so a
// walker's outputs are bit-identical to an spo_eval of that walker alone.
#include <cuda.h>

#include <algorithm>

#include "spo_batch.h"
#include "spo_device.cuh"
#include "spo_internal.h"
#include "spo_tma.cuh"

namespace {

using namespace spo_dev;
using spo_detail::BatchParams;
using spo_detail::BatchSetDesc;
using spo_detail::kBlockEdge;
using spo_detail::kBrick;

constexpr int kBlockRows = kBlockEdge * kBlockEdge * kBlockEdge;   // 343
constexpr int kVec = 4;

template <int TILE>
struct Shape {
    static constexpr int threads = TILE >= 64 ? 256 : 128;
    static constexpr int ctas_per_sm = TILE >= 64 ? 2 : 4;
};

// PAIR (32-orbital tiles, every set with brick-pair maps): a unit is a
// z-adjacent pair of bricks, its block one 7 x 7 x 11-node box and its
// positions the two bricks' contiguous ranges of the sorted order, as in the
// single-set kernel's pair form (3 CTAs per SM).
template <typename T, int KIND, int TILE, bool VEC_OUT, bool PAIR = false>
__global__ void __launch_bounds__(Shape<TILE>::threads, PAIR ? 3 : Shape<TILE>::ctas_per_sm)
spo_brick_batch_kernel(const __grid_constant__ BatchParams bp, const int *__restrict__ offsets,
                       const float4 *__restrict__ wrec, float *const *__restrict__ dst,
                       unsigned int *status)
{
    static_assert(!PAIR || TILE == 32, "brick pairs with 32-orbital tiles");
    constexpr int NC = Rows<KIND>::value;
    constexpr int kThreads = Shape<TILE>::threads;
    constexpr int TPP = TILE / kVec;
    constexpr int PPR = kThreads / TPP;
    constexpr int kBZ = PAIR ? 2 * kBrick + 3 : kBlockEdge;   // block nodes along z
    constexpr uint32_t kBytes = kBlockEdge * kBlockEdge * kBZ * TILE * sizeof(T);
    extern __shared__ __align__(1024) unsigned char smem[];
    T *block = reinterpret_cast<T *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kBytes);
    float4 *wslots = reinterpret_cast<float4 *>(smem + kBytes + 16);   // [PPR][kSlotF4]

    const int unit = blockIdx.x;
    int s = 0;
    while (s + 1 < bp.nsets && unit >= bp.sets[s + 1].unit_base) ++s;
    const BatchSetDesc &d = bp.sets[s];
    const int local = unit - d.unit_base;
    const int lbrick = local / d.ntiles, tile = local - lbrick * d.ntiles;   // brick (or pair) of the set
    const int nbzu = PAIR ? (d.nbz + 1) / 2 : d.nbz;
    const int bzu = lbrick % nbzu, by = (lbrick / nbzu) % d.nby, bx = lbrick / (nbzu * d.nby);
    const int bz = PAIR ? 2 * bzu : bzu;
    const int gbrick = d.brick_base + (bx * d.nby + by) * d.nbz + bz;
    const int gend = gbrick + ((PAIR && bz + 1 < d.nbz) ? 2 : 1);
    const uint32_t bar_s = smem_addr(bar);

    int begin = 0, end = 0;
    if (!bp.eager) {
        begin = __ldg(offsets + gbrick);
        end = __ldg(offsets + gend);
        if (begin == end) return;
    }
    if (threadIdx.x == 0) {
        mbar_init(bar_s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar_s, kBytes);
        tma_load_4d(smem_addr(block), &bp.maps[s], bar_s, tile * TILE, bz * kBrick, by * kBrick,
                    bx * kBrick);
    }
    if (bp.eager) {
        begin = __ldg(offsets + gbrick);
        end = __ldg(offsets + gend);
    }
    __syncthreads();
    if (begin == end) {
        if (threadIdx.x == 0 && !mbar_wait_bounded(bar_s, 0)) atomicOr(status, 1u);
        return;
    }

    const int q = threadIdx.x % TPP;
    const int64_t N = d.N;
    const int64_t o0 = (int64_t)tile * TILE + q * kVec;
    // rounds of PPR positions, the trip count uniform over each warp (the
    // weight slots are shared within it), as in the single-set kernel
    const int wg0 = (int)(threadIdx.x >> 5) * (32 / TPP);
    float4 *slot = wslots + (threadIdx.x / TPP) * kSlotF4;
    int i = begin + threadIdx.x / TPP;
    // lane q of a position's group copies parts q, q + TPP, ... of the
    // position's weight record (formed by the binning) into the slot, one
    // round ahead
    constexpr int NPART = (kSlotF4 + TPP - 1) / TPP;
    auto fetch = [&](int ii, float4 (&r)[NPART]) {
#pragma unroll
        for (int k = 0; k < NPART; ++k)
            if (q + k * TPP < kSlotF4) r[k] = __ldg(wrec + (int64_t)ii * kSlotF4 + q + k * TPP);
    };
    float4 cur[NPART];
#pragma unroll
    for (int k = 0; k < NPART; ++k) cur[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < end) fetch(i, cur);
    float *ocur = i < end ? dst[i] : nullptr;
    bool ready = false;
    for (int ib = begin + wg0; ib < end; ib += PPR, i += PPR) {
        const bool more = i + PPR < end;
        float4 nxt[NPART];
#pragma unroll
        for (int k = 0; k < NPART; ++k) nxt[k] = cur[k];
        if (more) fetch(i + PPR, nxt);
        float *onxt = more ? dst[i + PPR] : ocur;
        __syncwarp();   // the previous round's reads of the slots are done
#pragma unroll
        for (int k = 0; k < NPART; ++k)
            if (q + k * TPP < kSlotF4) slot[q + k * TPP] = cur[k];
        __syncwarp();
        if (!ready) {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_s, 0))) {
                if ((threadIdx.x & 31) == 0) atomicOr(status, 1u);
                return;
            }
            ready = true;
        }
        if (i < end) {
            Axis Y, Z;
            const int4 cells = *reinterpret_cast<const int4 *>(slot + 10);
            unpack4(slot[4], Y.w);
            unpack4(slot[5], Y.d);
            unpack4(slot[6], Y.dd);
            unpack4(slot[7], Z.w);
            unpack4(slot[8], Z.d);
            unpack4(slot[9], Z.dd);
            const int lx = min(max(cells.x - bx * kBrick, 0), kBrick - 1);
            const int ly = min(max(cells.y - by * kBrick, 0), kBrick - 1);
            const int lz = min(max(cells.z - bz * kBrick, 0), (PAIR ? 2 : 1) * kBrick - 1);
            const T *base = block + ((lx * kBlockEdge + ly) * kBZ + lz) * TILE + q * kVec;
            float acc[NC][kVec];
            window_reduce_staged<KIND, kVec, true>(slot, Y, Z,
                                [&](int a, int b, int g, float *v) {
                                    load_coefs<T, kVec, false>(
                                        base + ((a * kBlockEdge + b) * kBZ + g) * TILE, v);
                                },
                                acc);
            if (o0 < N) store_rows<NC, kVec, VEC_OUT>(ocur + o0, N, N - o0, acc);
        }
#pragma unroll
        for (int k = 0; k < NPART; ++k) cur[k] = nxt[k];
        ocur = onxt;
    }
    if (!ready && threadIdx.x == 0 && !mbar_wait_bounded(bar_s, 0)) atomicOr(status, 1u);
}

// dynamic shared memory: the 7x7x7-node block, the barrier, one weight slot
// per position of a round
template <typename T, int TILE, bool PAIR = false>
constexpr size_t batch_smem() {
    return (size_t)kBlockEdge * kBlockEdge * (PAIR ? 2 * kBrick + 3 : kBlockEdge) * TILE * sizeof(T) + 16 +
           (size_t)(Shape<TILE>::threads / (TILE / kVec)) * kSlotF4 * 16;
}

template <typename T, int KIND, int TILE>
cudaError_t launch_typed(const BatchParams &bp, const int *offsets, const float4 *wrec,
                         float *const *dst, bool vec_out, unsigned int *status, cudaStream_t stream) {
    if (bp.total_units <= 0) return cudaSuccess;
    if constexpr (TILE == 32) {
        if (bp.pair) {
            constexpr size_t kSmemP = batch_smem<T, 32, true>();
            auto kernel = vec_out ? spo_brick_batch_kernel<T, KIND, 32, true, true>
                                  : spo_brick_batch_kernel<T, KIND, 32, false, true>;
            kernel<<<(unsigned)bp.total_units, Shape<32>::threads, kSmemP, stream>>>(bp, offsets, wrec, dst,
                                                                                     status);
            return cudaGetLastError();
        }
    }
    constexpr size_t kSmem = batch_smem<T, TILE>();
    auto kernel = vec_out ? spo_brick_batch_kernel<T, KIND, TILE, true>
                          : spo_brick_batch_kernel<T, KIND, TILE, false>;
    kernel<<<(unsigned)bp.total_units, Shape<TILE>::threads, kSmem, stream>>>(bp, offsets, wrec, dst,
                                                                             status);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t launch_tile(int tile, const BatchParams &bp, const int *offsets, const float4 *wrec,
                        float *const *dst, bool vec_out, unsigned int *status, cudaStream_t stream) {
    return tile == 64 ? launch_typed<T, KIND, 64>(bp, offsets, wrec, dst, vec_out, status, stream)
                      : launch_typed<T, KIND, 32>(bp, offsets, wrec, dst, vec_out, status, stream);
}

template <typename T>
cudaError_t launch_kind(spo_kind kind, int tile, const BatchParams &bp, const int *offsets,
                        const float4 *wrec, float *const *dst, bool vec_out, unsigned int *status,
                        cudaStream_t stream) {
    switch (kind) {
        case SPO_KIND_V:
            return launch_tile<T, SPO_KIND_V>(tile, bp, offsets, wrec, dst, vec_out, status, stream);
        case SPO_KIND_VGL:
            return launch_tile<T, SPO_KIND_VGL>(tile, bp, offsets, wrec, dst, vec_out, status, stream);
        case SPO_KIND_VGH:
            return launch_tile<T, SPO_KIND_VGH>(tile, bp, offsets, wrec, dst, vec_out, status, stream);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int KIND>
cudaError_t prepare_kind() {
    cudaError_t e = cudaSuccess;
    const int s32 = (int)batch_smem<T, 32>();
    const int s64 = (int)batch_smem<T, 64>();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spo_brick_batch_kernel<T, KIND, 32, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spo_brick_batch_kernel<T, KIND, 32, false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spo_brick_batch_kernel<T, KIND, 64, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spo_brick_batch_kernel<T, KIND, 64, false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    const int sp = (int)batch_smem<T, 32, true>();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spo_brick_batch_kernel<T, KIND, 32, true, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, sp);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spo_brick_batch_kernel<T, KIND, 32, false, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, sp);
    return e;
}

template <typename T>
cudaError_t prepare_type() {
    cudaError_t e = prepare_kind<T, SPO_KIND_V>();
    if (e == cudaSuccess) e = prepare_kind<T, SPO_KIND_VGL>();
    if (e == cudaSuccess) e = prepare_kind<T, SPO_KIND_VGH>();
    return e;
}

}  // namespace

namespace spo_detail {

cudaError_t prepare_brick_batch() {
    cudaError_t e = prepare_type<float>();
    if (e == cudaSuccess) e = prepare_type<__nv_bfloat16>();
    if (e == cudaSuccess) e = prepare_type<__half>();
    return e;
}

cudaError_t launch_brick_batch(spo_dtype storage, spo_kind kind, int tile, const BatchParams &bp,
                               const int *offsets, const float4 *wrec, float *const *dst,
                               bool vec_out, unsigned int *status, cudaStream_t stream) {
    switch (storage) {
        case SPO_F32:
            return launch_kind<float>(kind, tile, bp, offsets, wrec, dst, vec_out, status, stream);
        case SPO_BF16:
            return launch_kind<__nv_bfloat16>(kind, tile, bp, offsets, wrec, dst, vec_out, status,
                                              stream);
        case SPO_F16:
            return launch_kind<__half>(kind, tile, bp, offsets, wrec, dst, vec_out, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spo_detail
