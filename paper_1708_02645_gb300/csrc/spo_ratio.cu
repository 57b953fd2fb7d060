// Determinant ratios (Sec. 3, eq. md_lemma): rho_p = sum_j rows[r(p)][j]
// phi_j(pos_p).  The brick kernel's ratio epilogue leaves one partial dot
// product per (orbital tile, position); ratio_reduce_kernel adds the tiles
// in order.  For sets the brick kernel does not serve, the values are
// evaluated first and ratio_dot_kernel forms the dot products (one warp per
// position, fixed reduction order).  Both are deterministic.
#include <algorithm>

#include "spo_internal.h"

namespace {

__global__ void ratio_reduce_kernel(const float *__restrict__ partials, int ntiles, int64_t P,
                                    float *__restrict__ ratio) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        float s = __ldg(partials + p);
        for (int t = 1; t < ntiles; ++t) s += __ldg(partials + (int64_t)t * P + p);
        ratio[p] = s;
    }
}

__global__ void ratio_dot_kernel(const float *__restrict__ v, int64_t P, int64_t N,
                                 spo_detail::RatioArgs ra, float *__restrict__ ratio) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
        int64_t r = ra.row_of ? (int64_t)__ldg(ra.row_of + p) : p;
        r = r < 0 ? 0 : (r >= ra.nrows ? ra.nrows - 1 : r);
        const float *a = ra.rows + r * ra.ld;
        const float *vp = v + p * N;
        float s = 0.0f;
        for (int64_t j = lane; j < N; j += 32) s = fmaf(__ldg(a + j), __ldg(vp + j), s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) ratio[p] = s;
    }
}

}  // namespace

namespace spo_detail {

cudaError_t launch_ratio_reduce(const float *partials, int ntiles, int64_t P, float *ratio,
                                cudaStream_t stream) {
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((P + threads - 1) / threads, 152 * 16);
    ratio_reduce_kernel<<<blocks, threads, 0, stream>>>(partials, ntiles, P, ratio);
    return cudaGetLastError();
}

cudaError_t launch_ratio_dot(const float *v, int64_t P, int64_t N, const RatioArgs &r, float *ratio,
                             cudaStream_t stream) {
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((P + 7) / 8, 152 * 16);
    ratio_dot_kernel<<<blocks, threads, 0, stream>>>(v, P, N, r, ratio);
    return cudaGetLastError();
}

}  // namespace spo_detail
