// Brick kernel dispatch: storage type -> the per-type instantiations of
// spo_brick.cuh (spo_brick_f32.cu, spo_brick_bf16.cu, spo_brick_f16.cu); the
// TMA maps of a set's table; the device status word that bounded waits set.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "spo_batch.h"
#include "spo_internal.h"

__device__ unsigned int g_spo_device_status = 0;

namespace {

using spo_detail::kBlockEdge;
using spo_detail::kBrick;

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
    (void)pos;   // the brick kernel reads the sorted copy of the positions
    switch (storage) {
        case SPO_F32: return brick_eval_typed<float>(kind, set, w, P, out, stream);
        case SPO_BF16: return brick_eval_typed<__nv_bfloat16>(kind, set, w, P, out, stream);
        case SPO_F16: return brick_eval_typed<__half>(kind, set, w, P, out, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_brick_ratio(const spo_set *set, const Workspace &w, int64_t P, float *out,
                               const RatioArgs &r, cudaStream_t stream) {
    switch (set->storage) {
        case SPO_F32: return brick_ratio_typed<float>(set, w, P, out, r, stream);
        case SPO_BF16: return brick_ratio_typed<__nv_bfloat16>(set, w, P, out, r, stream);
        case SPO_F16: return brick_ratio_typed<__half>(set, w, P, out, r, stream);
        default: return cudaErrorInvalidValue;
    }
}

int brick_tiles_of(const spo_set *s) {
    const int tile = brick_tile_of(s);
    return (int)((s->N + tile - 1) / tile);
}

int brick_tile_of(const spo_set *s) {
    return (s->brick_tile == 64 && s->Np >= 64) ? 64 : 32;
}

spo_status make_block_map(spo_set *s) {
    s->has_block_map = false;
    if (device_status_address(&s->status) != cudaSuccess)
        return fail(SPO_ECUDA, "device status word: %s", cudaGetErrorString(cudaGetLastError()));
    if (s->Np < 32) return SPO_OK;   // too few orbitals: the gather kernels serve this set
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
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {   // box widths 32 and 64 orbitals
        const cuuint32_t tile = k == 0 ? 32 : 64;
        if (s->Np < (int64_t)tile) continue;
        const cuuint32_t box[4] = {tile, kBlockEdge, kBlockEdge, kBlockEdge};
        CUresult r = enc(&s->block_map[k], dt, 4, s->table, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(SPO_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    s->has_block_map = true;
    // brick pairs along z: box (32, 11, 7, 7), for grids of at least two bricks in z
    s->has_pair_map = false;
    if (s->nbz >= 2 && s->zp >= 2 * kBrick + 3) {
        const cuuint32_t box[4] = {32, 2 * kBrick + 3, kBlockEdge, kBlockEdge};
        const CUresult r = enc(&s->block_map[2], dt, 4, s->table, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        s->has_pair_map = r == CUDA_SUCCESS;
    }
    return SPO_OK;
}

cudaError_t device_status_address(unsigned int **addr) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_spo_device_status);
    *addr = static_cast<unsigned int *>(p);
    return e;
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
