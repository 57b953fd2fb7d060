// Brick kernel: one CTA per (brick, orbital tile).
//
// Positions are binned by brick (kBrick^3 cells, spo_bin.cu).  Every window
// of a position in brick (bx, by, bz) lies in the padded table nodes
// [4bx, 4bx+7) x [4by, 4by+7) x [4bz, 4bz+7), so one TMA copy (a 4-D box of
// 64 orbitals x 7 x 7 x 7 nodes, 88 KB in FP32) stages everything the
// brick's positions need for one orbital tile.  The positions of the brick
// are then evaluated from shared memory by one warp per position (2 orbitals
// per thread, so a corner row is one 8-byte (FP32) or 4-byte (BF16/FP16)
// conflict-free shared load per thread); the z -> y -> x reduction and
// its FMA order are those of the gather kernel (spo_device.cuh), and outputs
// are scattered back to each position's own rows with streaming stores.
//
// Against the gather kernel, the table bytes moved from L2 to the SMs drop
// from 64 rows per evaluation to 343 rows per (brick, tile), and the L2 sees
// neighbouring bricks' blocks in launch order, so DRAM reads approach one
// pass over the table per batch.  Two CTAs fit per SM, so one CTA's copy
// overlaps the other's arithmetic.
//
// The wait on the copy is bounded (2 s of %globaltimer): if it ever gives up,
// the CTA sets bit 0 of the device status word and returns.
#include <cuda.h>

#include <algorithm>

#include "spo_device.cuh"
#include "spo_internal.h"

__device__ unsigned int g_spo_device_status = 0;

namespace {

using namespace spo_dev;
using spo_detail::kBlockEdge;
using spo_detail::kBrick;

constexpr int kThreads = 256;
constexpr int kBlockRows = kBlockEdge * kBlockEdge * kBlockEdge;   // 343
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier for at most kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > kWaitLimitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

template <typename T, int KIND, int TILE, int V, bool VEC_OUT>
__global__ void __launch_bounds__(kThreads, 2)
spo_brick_kernel(const __grid_constant__ CUtensorMap map, GridAxis gx, GridAxis gy, GridAxis gz,
                 int nby, int nbz, int ntiles, int64_t N, const float *__restrict__ pos,
                 const int *__restrict__ offsets, const int *__restrict__ perm,
                 float *__restrict__ out)
{
    constexpr int NC = Rows<KIND>::value;
    constexpr int kVec = V;                   // orbitals per thread
    constexpr int TPP = TILE / kVec;          // threads per position
    constexpr int PPR = kThreads / TPP;       // positions per round
    constexpr uint32_t kBytes = kBlockRows * TILE * sizeof(T);
    extern __shared__ __align__(128) unsigned char smem[];
    T *block = reinterpret_cast<T *>(smem);   // [7][7][7][TILE]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kBytes);

    const int brick = blockIdx.x / ntiles;
    const int tile = blockIdx.x - brick * ntiles;
    const int begin = __ldg(offsets + brick), end = __ldg(offsets + brick + 1);
    if (begin == end) return;
    const int bz = brick % nbz, by = (brick / nbz) % nby, bx = brick / (nbz * nby);

    const uint32_t bar_s = smem_addr(bar);
    if (threadIdx.x == 0) {
        mbar_init(bar_s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar_s, kBytes);
        tma_load_4d(smem_addr(block), &map, bar_s, tile * TILE, bz * kBrick, by * kBrick, bx * kBrick);
    }

    const int q = threadIdx.x % TPP;
    const int64_t o0 = (int64_t)tile * TILE + q * kVec;   // first orbital of this thread
    bool ready = false;
    for (int i = begin + threadIdx.x / TPP; i < end; i += PPR) {
        const int p = __ldg(perm + i);
        Axis X, Y, Z;
        make_axis(__ldg(pos + 3 * p + 0), gx, X);
        make_axis(__ldg(pos + 3 * p + 1), gy, Y);
        make_axis(__ldg(pos + 3 * p + 2), gz, Z);
        if (!ready) {   // first position's weights were computed while the copy flew
            if (!mbar_wait_bounded(bar_s, 0)) {
                atomicOr(&g_spo_device_status, 1u);
                return;
            }
            ready = true;
        }
        // the binning put the cell in this brick; the clamp keeps the shared
        // memory index in range even if it had not
        const int lx = min(max(X.cell - bx * kBrick, 0), kBrick - 1);
        const int ly = min(max(Y.cell - by * kBrick, 0), kBrick - 1);
        const int lz = min(max(Z.cell - bz * kBrick, 0), kBrick - 1);
        const T *base = block + ((lx * kBlockEdge + ly) * kBlockEdge + lz) * TILE + q * kVec;
        float acc[NC][kVec];
        window_reduce<KIND, kVec, true>(X, Y, Z,
                            [&](int a, int b, int g, float *v) {
                                load_coefs<T, kVec, false>(
                                    base + ((a * kBlockEdge + b) * kBlockEdge + g) * TILE, v);
                            },
                            acc);
        if (o0 < N) store_rows<NC, kVec, VEC_OUT>(out + (int64_t)p * NC * N + o0, N, N - o0, acc);
    }
    if (!ready && threadIdx.x == 0) {
        // a thread with no position still must not leave while the copy
        // writes shared memory that another CTA could reuse
        if (!mbar_wait_bounded(bar_s, 0)) atomicOr(&g_spo_device_status, 1u);
    }
}

// orbitals per tile: one warp (2 orbitals per thread) per position
constexpr int kTile = 64;

template <typename T, int KIND, int V>
cudaError_t brick_typed(const spo_set *s, const float *pos, const spo_detail::Workspace &w,
                        float *out, cudaStream_t stream) {
    constexpr int TILE = kTile;
    constexpr size_t kSmem = (size_t)kBlockRows * TILE * sizeof(T) + 16;
    const int nbins = s->nbx * s->nby * s->nbz;
    const int ntiles = (int)((s->N + TILE - 1) / TILE);
    const int64_t blocks = (int64_t)nbins * ntiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool vec_out = (s->N % V == 0) && ((reinterpret_cast<uintptr_t>(out) % (4 * V)) == 0);
    auto kernel = vec_out ? spo_brick_kernel<T, KIND, TILE, V, true>
                          : spo_brick_kernel<T, KIND, TILE, V, false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    kernel<<<(unsigned)blocks, kThreads, kSmem, stream>>>(s->block_map, grid_axis(s->nx),
                                                          grid_axis(s->ny), grid_axis(s->nz), s->nby,
                                                          s->nbz, ntiles, s->N, pos, w.offsets,
                                                          w.perm, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t brick_kind(spo_kind kind, const spo_set *s, const float *pos,
                       const spo_detail::Workspace &w, float *out, cudaStream_t stream) {
    const bool v4 = s->brick_vec == 4;
    switch (kind) {
        case SPO_KIND_V:
            return v4 ? brick_typed<T, SPO_KIND_V, 4>(s, pos, w, out, stream)
                      : brick_typed<T, SPO_KIND_V, 2>(s, pos, w, out, stream);
        case SPO_KIND_VGL:
            return v4 ? brick_typed<T, SPO_KIND_VGL, 4>(s, pos, w, out, stream)
                      : brick_typed<T, SPO_KIND_VGL, 2>(s, pos, w, out, stream);
        case SPO_KIND_VGH:
            return v4 ? brick_typed<T, SPO_KIND_VGH, 4>(s, pos, w, out, stream)
                      : brick_typed<T, SPO_KIND_VGH, 2>(s, pos, w, out, stream);
    }
    return cudaErrorInvalidValue;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

}  // namespace

namespace spo_detail {

cudaError_t launch_brick(spo_dtype storage, spo_kind kind, const spo_set *set, const float *pos,
                         const Workspace &w, int64_t P, float *out, cudaStream_t stream) {
    (void)P;
    switch (storage) {
        case SPO_F32: return brick_kind<float>(kind, set, pos, w, out, stream);
        case SPO_BF16: return brick_kind<__nv_bfloat16>(kind, set, pos, w, out, stream);
        case SPO_F16: return brick_kind<__half>(kind, set, pos, w, out, stream);
        default: return cudaErrorInvalidValue;
    }
}

spo_status make_block_map(spo_set *s) {
    s->has_block_map = false;
    const int tile = kTile;
    s->tile = tile;
    if (s->Np < tile) return SPO_OK;   // too few orbitals: the gather kernel serves this set
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(SPO_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const size_t es = s->storage == SPO_F32 ? 4 : 2;
    const CUtensorMapDataType dt = s->storage == SPO_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : s->storage == SPO_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[4] = {(cuuint64_t)s->Np, (cuuint64_t)s->zp, (cuuint64_t)s->yp,
                                (cuuint64_t)s->xp};
    const cuuint64_t strides[3] = {(cuuint64_t)s->Np * es, (cuuint64_t)s->zp * s->Np * es,
                                   (cuuint64_t)s->yp * s->zp * s->Np * es};
    const cuuint32_t box[4] = {(cuuint32_t)tile, kBlockEdge, kBlockEdge, kBlockEdge};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&s->block_map, dt, 4, s->table, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SPO_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    s->has_block_map = true;
    return SPO_OK;
}

cudaError_t read_device_status(unsigned int *flags, bool clear, cudaStream_t stream) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(flags, g_spo_device_status, sizeof(unsigned int), 0,
                                              cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_spo_device_status, &zero, sizeof(zero), 0,
                                    cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    }
    return e;
}

}  // namespace spo_detail
