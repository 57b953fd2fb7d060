// Gather kernel and table conversion.
//
// Gather kernel: one thread evaluates 4 consecutive orbitals of one position
// (V, VGL or VGH: Sec. 6.1's Bspline-v / SPO-vgl / Bspline-vgh).  Threads of
// one position are adjacent, so each of the 64 corner rows of the 4x4x4
// window is one contiguous, coalesced run across the threads (16-byte loads
// for FP32, 8-byte loads for BF16/FP16).  The table carries 3 ghost nodes per
// axis, so a window is always the padded nodes i..i+3 and needs no wrap.
// Outputs use streaming stores, so a large batch's results do not evict the
// table from L2.  With a permutation (positions binned by brick) neighbouring
// threads read neighbouring windows and L2 serves most of the corner rows.
#include <algorithm>

#include "spo_batch.h"
#include "spo_device.cuh"
#include "spo_index.cuh"
#include "spo_internal.h"

namespace {

using namespace spo_dev;

constexpr int kThreads = 256;
constexpr int kVec = 4;   // orbitals per thread

// Two blocks per SM at most (128 registers): the VGH form would take 130 and
// run one block (8 warps) per SM; the loads of this latency-bound kernel
// need the warps (VGH 25-36 % faster at 2,048-16,384 positions).
template <typename T, int KIND, bool VEC_OUT>
__global__ void __launch_bounds__(kThreads, 2)
spo_gather_kernel(const T *__restrict__ table, GridAxis gx, GridAxis gy, GridAxis gz, int yp, int zp,
                  int64_t Np, int64_t N, const float *__restrict__ pos, const int *__restrict__ perm,
                  int64_t P, int G, float *__restrict__ out, unsigned int *__restrict__ status)
{
    constexpr int NC = Rows<KIND>::value;
    const int64_t item = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (item >= P * G) return;
    int q;
    const int64_t i = div_index(item, G, q);
    const int64_t p = perm ? (int64_t)__ldg(perm + i) : i;
    if (!bounds_ok(p >= 0 && p < P, status)) return;   // debug builds: a permutation entry in range

    XAxis X;
    Axis Y, Z;
    make_xaxis(__ldg(pos + 3 * p + 0), gx, X);
    make_axis(__ldg(pos + 3 * p + 1), gy, Y);
    make_axis(__ldg(pos + 3 * p + 2), gz, Z);
    // debug builds: the window's 4 x 4 x 4 padded nodes lie in the table
    if (!bounds_ok((unsigned)X.cell < (unsigned)gx.n && (unsigned)Y.cell < (unsigned)gy.n &&
                       (unsigned)Z.cell < (unsigned)gz.n,
                   status))
        return;

    // padded node of corner (a, b, g) = (cell_x + a, cell_y + b, cell_z + g)
    const T *tq = table + (((int64_t)X.cell * yp + Y.cell) * zp + Z.cell) * Np + (int64_t)q * kVec;
    const int64_t sx = (int64_t)yp * zp * Np, sy = (int64_t)zp * Np;
    float acc[NC][kVec];
    window_reduce<KIND, kVec, false>(X, gx, Y, Z,
                        [&](int a, int b, int g, float *v) {
                            load_coefs<T, kVec, true>(tq + a * sx + b * sy + g * Np, v);
                        },
                        acc);
    const int64_t o0 = (int64_t)q * kVec;
    store_rows<NC, kVec, VEC_OUT>(out + p * NC * N + o0, N, N - o0, acc);
}

template <typename T, int KIND>
cudaError_t gather_typed(const spo_detail::TableView &t, const float *pos, const int *perm,
                         int64_t P, float *out, cudaStream_t stream) {
    const int G = (int)((t.N + kVec - 1) / kVec);
    const int64_t blocks = (P * G + kThreads - 1) / kThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool vec_out = (t.N % kVec == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    const T *table = static_cast<const T *>(t.table);
    unsigned int *status = nullptr;   // the index checks' flag word (SPO_CHECK_BOUNDS builds)
#ifdef SPO_CHECK_BOUNDS
    if (cudaError_t e = spo_detail::device_status_address(&status); e != cudaSuccess) return e;
#endif
    if (vec_out)
        spo_gather_kernel<T, KIND, true><<<(unsigned)blocks, kThreads, 0, stream>>>(
            table, grid_axis(t.nx), grid_axis(t.ny), grid_axis(t.nz), t.yp, t.zp, t.Np, t.N, pos,
            perm, P, G, out, status);
    else
        spo_gather_kernel<T, KIND, false><<<(unsigned)blocks, kThreads, 0, stream>>>(
            table, grid_axis(t.nx), grid_axis(t.ny), grid_axis(t.nz), t.yp, t.zp, t.Np, t.N, pos,
            perm, P, G, out, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_kind(spo_kind kind, const spo_detail::TableView &t, const float *pos,
                        const int *perm, int64_t P, float *out, cudaStream_t stream) {
    switch (kind) {
        case SPO_KIND_V: return gather_typed<T, SPO_KIND_V>(t, pos, perm, P, out, stream);
        case SPO_KIND_VGL: return gather_typed<T, SPO_KIND_VGL>(t, pos, perm, P, out, stream);
        case SPO_KIND_VGH: return gather_typed<T, SPO_KIND_VGH>(t, pos, perm, P, out, stream);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// coefficient conversion into the padded table
// ---------------------------------------------------------------------------
template <typename D>
__device__ __forceinline__ D from_double(double x);
template <>
__device__ __forceinline__ float from_double<float>(double x) { return __double2float_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <>
__device__ __forceinline__ __half from_double<__half>(double x) { return __double2half(x); }

template <typename D>
__device__ __forceinline__ D from_float(float x);
template <>
__device__ __forceinline__ float from_float<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half from_float<__half>(float x) { return __float2half_rn(x); }

// Each source value is widened exactly (to FP64 for an FP64 source, to FP32
// otherwise) and rounded once to the storage type.
template <typename D>
__device__ __forceinline__ D convert_one(const void *src, spo_dtype sd, int64_t i) {
    switch (sd) {
        case SPO_F64: return from_double<D>(static_cast<const double *>(src)[i]);
        case SPO_F32: return from_float<D>(static_cast<const float *>(src)[i]);
        case SPO_BF16: return from_float<D>(__bfloat162float(static_cast<const __nv_bfloat16 *>(src)[i]));
        case SPO_F16: return from_float<D>(__half2float(static_cast<const __half *>(src)[i]));
    }
    return from_float<D>(0.0f);
}

// Padded planes x' = x0+1 .. x1 (grid nodes x0 .. x1-1), every padded y', z'
// and every padded orbital.  Padded node i' holds grid node (i' - 1) mod n;
// orbitals N .. Np-1 are zero.
template <typename D>
__global__ void convert_kernel(const void *__restrict__ src, spo_dtype sd, D *__restrict__ dst,
                               int x0, int x1, int ny, int nz, int yp, int zp, int64_t N, int64_t Np) {
    const int64_t plane = (int64_t)yp * zp * Np;
    const int64_t total = (int64_t)(x1 - x0) * plane;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xs = e / plane;               // 0 .. x1-x0-1
        int64_t r = e - xs * plane;
        const int64_t yq = r / ((int64_t)zp * Np);
        r -= yq * (int64_t)zp * Np;
        const int64_t zq = r / Np;
        const int64_t j = r - zq * Np;
        const int64_t y = (yq - 1 + ny) % ny, z = (zq - 1 + nz) % nz;
        const int64_t didx = (((x0 + 1 + xs) * yp + yq) * zp + zq) * Np + j;
        dst[didx] = j < N ? convert_one<D>(src, sd, ((xs * ny + y) * nz + z) * N + j) : from_float<D>(0.0f);
    }
}

}  // namespace

namespace spo_detail {

cudaError_t launch_gather(spo_dtype storage, spo_kind kind, const TableView &t, const float *pos,
                          const int *perm, int64_t P, float *out, cudaStream_t stream) {
    switch (storage) {
        case SPO_F32: return gather_kind<float>(kind, t, pos, perm, P, out, stream);
        case SPO_BF16: return gather_kind<__nv_bfloat16>(kind, t, pos, perm, P, out, stream);
        case SPO_F16: return gather_kind<__half>(kind, t, pos, perm, P, out, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_convert(const void *src, spo_dtype src_dtype, int x0, int x1, const spo_set *s,
                           cudaStream_t stream) {
    const int threads = 256;
    const int64_t total = (int64_t)(x1 - x0) * s->yp * s->zp * s->Np;
    if (total == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 64);
    switch (s->storage) {
        case SPO_F32:
            convert_kernel<float><<<blocks, threads, 0, stream>>>(src, src_dtype,
                static_cast<float *>(s->table), x0, x1, s->ny, s->nz, s->yp, s->zp, s->N, s->Np);
            break;
        case SPO_BF16:
            convert_kernel<__nv_bfloat16><<<blocks, threads, 0, stream>>>(src, src_dtype,
                static_cast<__nv_bfloat16 *>(s->table), x0, x1, s->ny, s->nz, s->yp, s->zp, s->N, s->Np);
            break;
        case SPO_F16:
            convert_kernel<__half><<<blocks, threads, 0, stream>>>(src, src_dtype,
                static_cast<__half *>(s->table), x0, x1, s->ny, s->nz, s->yp, s->zp, s->N, s->Np);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace spo_detail
