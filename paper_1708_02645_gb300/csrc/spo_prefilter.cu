// spo_prefilter: interpolating B-spline coefficients from periodic grid
// samples, in place on the device.
//
// Along each axis the samples f and coefficients c satisfy
// (c[m-1] + 4 c[m] + c[m+1]) / 6 = f[m] (periodic): the spline passes
// through the samples at the nodes.  The inverse operator 6 / (z + 4 + 1/z)
// factors as -6 z1 / ((1 - z1 / z)(1 - z1 z)) with the pole z1 = sqrt(3) - 2,
// i.e. a causal and an anticausal first-order recursion (Unser, Aldroubi and
// Eden's recursive B-spline filtering), each started from its periodic
// initial value (the geometric sum over one period, truncated where
// |z1|^j < 1e-23).  One thread runs one line; lines along an axis are
// indexed (outer, inner) with inner the faster index, so neighbouring
// threads touch neighbouring orbitals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "spo.h"
#include "spo_internal.h"

namespace {

using spo_detail::fail;

constexpr int kInitTerms = 40;   // |z1|^40 < 1e-22

template <typename T>
__global__ void prefilter_axis_kernel(T *__restrict__ data, int L, int64_t S, int64_t nlines) {
    const double z1 = 1.7320508075688772 - 2.0;
    // 1 / (1 - z1^L)
    double zl = 1.0;
    for (int j = 0; j < L && j < 64; ++j) zl *= z1;
    const double norm = 1.0 / (1.0 - zl);
    const double gain = -6.0 * z1;
    const int K = min(L, kInitTerms);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nlines;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = t / S, i = t - o * S;
        T *line = data + o * (int64_t)L * S + i;
        // causal: y[k] = f[k] + z1 y[k-1], y[0] = sum_j z1^j f[-j mod L] / (1 - z1^L)
        double s = 0.0, zj = 1.0;
        for (int j = 0; j < K; ++j) {
            s += zj * (double)line[(int64_t)((L - j) % L) * S];
            zj *= z1;
        }
        double y = s * norm;
        line[0] = (T)y;
        // keep y in FP64 along the line; the stored value is only re-read by
        // the anticausal pass below
        double ylast = y;
        for (int k = 1; k < L; ++k) {
            ylast = (double)line[(int64_t)k * S] + z1 * ylast;
            line[(int64_t)k * S] = (T)ylast;
        }
        // anticausal: c[k] = y[k] + z1 c[k+1],
        // c[L-1] = sum_j z1^j y[(L-1+j) mod L] / (1 - z1^L)
        s = 0.0;
        zj = 1.0;
        for (int j = 0; j < K; ++j) {
            s += zj * (double)line[(int64_t)((L - 1 + j) % L) * S];
            zj *= z1;
        }
        double c = s * norm;
        line[(int64_t)(L - 1) * S] = (T)(gain * c);
        for (int k = L - 2; k >= 0; --k) {
            c = (double)line[(int64_t)k * S] + z1 * c;
            line[(int64_t)k * S] = (T)(gain * c);
        }
    }
}

template <typename T>
cudaError_t prefilter_all(T *data, const spo_grid &g, int64_t N, cudaStream_t st) {
    const int ext[3] = {g.nx, g.ny, g.nz};
    int64_t stride[3];
    stride[2] = N;
    stride[1] = (int64_t)g.nz * N;
    stride[0] = (int64_t)g.ny * g.nz * N;
    const int64_t total = (int64_t)g.nx * g.ny * g.nz * N;
    for (int ax = 0; ax < 3; ++ax) {
        const int64_t nlines = total / ext[ax];
        const int blocks = (int)std::min<int64_t>((nlines + 255) / 256, 152 * 32);
        prefilter_axis_kernel<T><<<blocks, 256, 0, st>>>(data, ext[ax], stride[ax], nlines);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" spo_status spo_prefilter(const spo_grid *grid, int64_t N, void *data, spo_dtype dtype,
                                    void *stream) {
    fail(SPO_OK, "");
    if (!grid || !data) return fail(SPO_EINVAL, "grid or data is NULL");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || N < 1)
        return fail(SPO_EINVAL, "grid and N must be positive");
    if ((int64_t)grid->nx * grid->ny * grid->nz > (INT64_C(1) << 40) / N)
        return fail(SPO_EINVAL, "table too large");
    if (dtype != SPO_F64 && dtype != SPO_F32) return fail(SPO_EINVAL, "dtype must be SPO_F64 or SPO_F32");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, data) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(SPO_EINVAL, "data must be device memory");
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = dtype == SPO_F64 ? prefilter_all(static_cast<double *>(data), *grid, N, st)
                                           : prefilter_all(static_cast<float *>(data), *grid, N, st);
    return e == cudaSuccess ? SPO_OK : fail(SPO_ECUDA, "prefilter launch: %s", cudaGetErrorString(e));
}
