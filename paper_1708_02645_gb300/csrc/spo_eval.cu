// Tricubic B-spline orbital evaluation kernels for sm_103a.
//
// One thread evaluates 4 consecutive orbitals of one position (V, VGL or VGH
// of Sec. 6.1's Bspline-v / SPO-vgl / Bspline-vgh).  Threads of one position
// are adjacent, so each of the 64 corner rows of the 4x4x4 window is read as
// one contiguous, coalesced run across a warp (16-byte loads for FP32, 8-byte
// loads for BF16/FP16), straight from the orbital-contiguous table.  The
// basis weights of the position live in registers; the 64-term sums are
// factored z -> y -> x, with FP32 accumulation.  Outputs are written with
// streaming stores, so that the 1.5 GB of VGH results of a large batch do not
// evict the table from L2.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "spo_internal.h"

namespace {

constexpr int kThreads = 256;   // threads per block
constexpr int kVec = 4;         // orbitals per thread

// ---------------------------------------------------------------------------
// loads of 4 consecutive coefficients, widened to FP32
// ---------------------------------------------------------------------------
template <typename T>
struct Load4;

template <>
struct Load4<float> {
    static __device__ __forceinline__ void get(const float *p, float v[4]) {
        const float4 r = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = r.x; v[1] = r.y; v[2] = r.z; v[3] = r.w;
    }
};

template <>
struct Load4<__nv_bfloat16> {
    static __device__ __forceinline__ void get(const __nv_bfloat16 *p, float v[4]) {
        const uint2 r = __ldg(reinterpret_cast<const uint2 *>(p));
        // a bf16 is the upper half of the FP32 with the same value
        v[0] = __uint_as_float(r.x << 16);
        v[1] = __uint_as_float(r.x & 0xffff0000u);
        v[2] = __uint_as_float(r.y << 16);
        v[3] = __uint_as_float(r.y & 0xffff0000u);
    }
};

template <>
struct Load4<__half> {
    static __device__ __forceinline__ void get(const __half *p, float v[4]) {
        const uint2 r = __ldg(reinterpret_cast<const uint2 *>(p));
        __half2 h0, h1;
        memcpy(&h0, &r.x, 4);
        memcpy(&h1, &r.y, 4);
        const float2 f0 = __half22float2(h0);
        const float2 f1 = __half22float2(h1);
        v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
    }
};

// ---------------------------------------------------------------------------
// per-position geometry
// ---------------------------------------------------------------------------

// Cell index i in [0, n) and fraction t in [0, 1] of coordinate r on a
// periodic axis of n intervals.  t = r*n - floor(r*n) is formed with one
// fused multiply-add, so it is the FP32 rounding of the exact fraction.
// NaN or Inf coordinates end in cell 0 with t = 0.
__device__ __forceinline__ void reduce_axis(float r, int n, int &cell, float &t) {
    const float fn = (float)n;
    float fl = floorf(r * fn);
    float tt = fmaf(r, fn, -fl);
    if (tt < 0.0f) {
        fl -= 1.0f;
        tt += 1.0f;
    } else if (tt >= 1.0f) {
        fl += 1.0f;
        tt -= 1.0f;
    }
    if (!(tt >= 0.0f && tt <= 1.0f)) tt = 0.0f;
    fl = fminf(fmaxf(fl, -1.0e9f), 1.0e9f);   // fmaxf maps NaN to the bound
    int c = (int)fl % n;
    if (c < 0) c += n;
    cell = c;
    t = tt;
}

__device__ __forceinline__ int wrap(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Cubic B-spline weights of the four window nodes (i-1, i, i+1, i+2) at
// fraction t, with first and second derivatives scaled to d/dr (factors n
// and n^2).
struct Axis {
    float w[4], d[4], dd[4];
    int idx[4];
};

__device__ __forceinline__ void make_axis(float r, int n, Axis &ax) {
    int c;
    float t;
    reduce_axis(r, n, c, t);
    const float fn = (float)n, fn2 = fn * fn;
    const float s = 1.0f - t, t2 = t * t, s2 = s * s;
    ax.w[0] = (1.0f / 6.0f) * s2 * s;
    ax.w[1] = fmaf(t2, fmaf(0.5f, t, -1.0f), 2.0f / 3.0f);
    ax.w[2] = fmaf(fmaf(fmaf(-0.5f, t, 0.5f), t, 0.5f), t, 1.0f / 6.0f);
    ax.w[3] = (1.0f / 6.0f) * t2 * t;
    ax.d[0] = -0.5f * s2 * fn;
    ax.d[1] = fmaf(1.5f, t, -2.0f) * t * fn;
    ax.d[2] = fmaf(fmaf(-1.5f, t, 1.0f), t, 0.5f) * fn;
    ax.d[3] = 0.5f * t2 * fn;
    ax.dd[0] = s * fn2;
    ax.dd[1] = fmaf(3.0f, t, -2.0f) * fn2;
    ax.dd[2] = fmaf(-3.0f, t, 1.0f) * fn2;
    ax.dd[3] = t * fn2;
#pragma unroll
    for (int k = 0; k < 4; ++k) ax.idx[k] = wrap(c + k - 1, n);
}

template <int KIND>
struct Rows {
    static constexpr int value = KIND == SPO_KIND_V ? 1 : (KIND == SPO_KIND_VGL ? 5 : 10);
};

// ---------------------------------------------------------------------------
// the evaluation kernel
// ---------------------------------------------------------------------------
template <typename T, int KIND, bool VEC_OUT>
__global__ void __launch_bounds__(kThreads)
spo_eval_kernel(const T *__restrict__ table, int nx, int ny, int nz, int64_t Np, int64_t N,
                const float *__restrict__ pos, int64_t P, int G, float *__restrict__ out)
{
    constexpr int NC = Rows<KIND>::value;
    const int64_t item = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (item >= P * G) return;
    const int64_t p = item / G;
    const int q = (int)(item - p * G);

    Axis X, Y, Z;
    make_axis(__ldg(pos + 3 * p + 0), nx, X);
    make_axis(__ldg(pos + 3 * p + 1), ny, Y);
    make_axis(__ldg(pos + 3 * p + 2), nz, Z);

    const T *tq = table + (int64_t)q * kVec;
    float acc[NC][kVec];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < kVec; ++k) acc[c][k] = 0.0f;

#pragma unroll
    for (int a = 0; a < 4; ++a) {
        // y-stage partial sums for this x node
        //   VGH: wy*v, dy*v, ddy*v, wy*dz, dy*dz, wy*ddz
        //   VGL: wy*v, dy*v, ddy*v, wy*dz, wy*ddz
        //   V:   wy*v
        constexpr int NY = KIND == SPO_KIND_V ? 1 : (KIND == SPO_KIND_VGL ? 5 : 6);
        float ys[NY][kVec];
#pragma unroll
        for (int j = 0; j < NY; ++j)
#pragma unroll
            for (int k = 0; k < kVec; ++k) ys[j][k] = 0.0f;

#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t row = ((int64_t)X.idx[a] * ny + Y.idx[b]) * nz;
            float cv[4][kVec];
#pragma unroll
            for (int g = 0; g < 4; ++g) Load4<T>::get(tq + (row + Z.idx[g]) * Np, cv[g]);
#pragma unroll
            for (int k = 0; k < kVec; ++k) {
                float zv = Z.w[0] * cv[0][k];
                zv = fmaf(Z.w[1], cv[1][k], zv);
                zv = fmaf(Z.w[2], cv[2][k], zv);
                zv = fmaf(Z.w[3], cv[3][k], zv);
                ys[0][k] = fmaf(Y.w[b], zv, ys[0][k]);
                if constexpr (KIND != SPO_KIND_V) {
                    float zd = Z.d[0] * cv[0][k];
                    zd = fmaf(Z.d[1], cv[1][k], zd);
                    zd = fmaf(Z.d[2], cv[2][k], zd);
                    zd = fmaf(Z.d[3], cv[3][k], zd);
                    float zdd = Z.dd[0] * cv[0][k];
                    zdd = fmaf(Z.dd[1], cv[1][k], zdd);
                    zdd = fmaf(Z.dd[2], cv[2][k], zdd);
                    zdd = fmaf(Z.dd[3], cv[3][k], zdd);
                    ys[1][k] = fmaf(Y.d[b], zv, ys[1][k]);
                    ys[2][k] = fmaf(Y.dd[b], zv, ys[2][k]);
                    ys[3][k] = fmaf(Y.w[b], zd, ys[3][k]);
                    if constexpr (KIND == SPO_KIND_VGH) {
                        ys[4][k] = fmaf(Y.d[b], zd, ys[4][k]);
                        ys[5][k] = fmaf(Y.w[b], zdd, ys[5][k]);
                    } else {
                        ys[4][k] = fmaf(Y.w[b], zdd, ys[4][k]);
                    }
                }
            }
        }
        // x stage
#pragma unroll
        for (int k = 0; k < kVec; ++k) {
            acc[0][k] = fmaf(X.w[a], ys[0][k], acc[0][k]);                 // v
            if constexpr (KIND == SPO_KIND_VGH) {
                acc[1][k] = fmaf(X.d[a], ys[0][k], acc[1][k]);             // gx
                acc[2][k] = fmaf(X.w[a], ys[1][k], acc[2][k]);             // gy
                acc[3][k] = fmaf(X.w[a], ys[3][k], acc[3][k]);             // gz
                acc[4][k] = fmaf(X.dd[a], ys[0][k], acc[4][k]);            // hxx
                acc[5][k] = fmaf(X.d[a], ys[1][k], acc[5][k]);             // hxy
                acc[6][k] = fmaf(X.d[a], ys[3][k], acc[6][k]);             // hxz
                acc[7][k] = fmaf(X.w[a], ys[2][k], acc[7][k]);             // hyy
                acc[8][k] = fmaf(X.w[a], ys[4][k], acc[8][k]);             // hyz
                acc[9][k] = fmaf(X.w[a], ys[5][k], acc[9][k]);             // hzz
            } else if constexpr (KIND == SPO_KIND_VGL) {
                acc[1][k] = fmaf(X.d[a], ys[0][k], acc[1][k]);             // gx
                acc[2][k] = fmaf(X.w[a], ys[1][k], acc[2][k]);             // gy
                acc[3][k] = fmaf(X.w[a], ys[3][k], acc[3][k]);             // gz
                // lap = hxx + hyy + hzz
                float l = fmaf(X.dd[a], ys[0][k], acc[4][k]);
                l = fmaf(X.w[a], ys[2][k], l);
                acc[4][k] = fmaf(X.w[a], ys[4][k], l);
            }
        }
    }

    float *o = out + p * NC * N + (int64_t)q * kVec;
    if constexpr (VEC_OUT) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            __stcs(reinterpret_cast<float4 *>(o + c * N),
                   make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]));
    } else {
        const int64_t left = N - (int64_t)q * kVec;
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int k = 0; k < kVec; ++k)
                if (k < left) __stcs(o + c * N + k, acc[c][k]);
    }
}

template <typename T, int KIND>
cudaError_t launch_typed(const spo_detail::EvalArgs &a, cudaStream_t stream) {
    const int G = (int)((a.N + kVec - 1) / kVec);
    const int64_t items = a.P * G;
    const int64_t blocks = (items + kThreads - 1) / kThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool vec_out = (a.N % kVec == 0) && ((reinterpret_cast<uintptr_t>(a.out) & 15) == 0);
    const T *table = static_cast<const T *>(a.table);
    if (vec_out)
        spo_eval_kernel<T, KIND, true><<<(unsigned)blocks, kThreads, 0, stream>>>(
            table, a.nx, a.ny, a.nz, a.Np, a.N, a.pos, a.P, G, a.out);
    else
        spo_eval_kernel<T, KIND, false><<<(unsigned)blocks, kThreads, 0, stream>>>(
            table, a.nx, a.ny, a.nz, a.Np, a.N, a.pos, a.P, G, a.out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kind(spo_kind kind, const spo_detail::EvalArgs &a, cudaStream_t stream) {
    switch (kind) {
        case SPO_KIND_V: return launch_typed<T, SPO_KIND_V>(a, stream);
        case SPO_KIND_VGL: return launch_typed<T, SPO_KIND_VGL>(a, stream);
        case SPO_KIND_VGH: return launch_typed<T, SPO_KIND_VGH>(a, stream);
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

template <typename D>
__global__ void convert_kernel(const void *__restrict__ src, spo_dtype sd, D *__restrict__ dst,
                               int64_t rows, int64_t N, int64_t Np) {
    const int64_t total = rows * Np;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Np, j = e - r * Np;
        dst[e] = j < N ? convert_one<D>(src, sd, r * N + j) : from_float<D>(0.0f);
    }
}

}  // namespace

namespace spo_detail {

cudaError_t launch_eval(spo_dtype storage, spo_kind kind, const EvalArgs &args,
                        cudaStream_t stream) {
    switch (storage) {
        case SPO_F32: return launch_kind<float>(kind, args, stream);
        case SPO_BF16: return launch_kind<__nv_bfloat16>(kind, args, stream);
        case SPO_F16: return launch_kind<__half>(kind, args, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_convert(const void *src, spo_dtype src_dtype, void *dst, spo_dtype storage,
                           int64_t rows, int64_t N, int64_t Np, cudaStream_t stream) {
    const int threads = 256;
    const int64_t total = rows * Np;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
    if (total == 0) return cudaSuccess;
    switch (storage) {
        case SPO_F32:
            convert_kernel<float><<<blocks, threads, 0, stream>>>(src, src_dtype,
                static_cast<float *>(dst), rows, N, Np);
            break;
        case SPO_BF16:
            convert_kernel<__nv_bfloat16><<<blocks, threads, 0, stream>>>(src, src_dtype,
                static_cast<__nv_bfloat16 *>(dst), rows, N, Np);
            break;
        case SPO_F16:
            convert_kernel<__half><<<blocks, threads, 0, stream>>>(src, src_dtype,
                static_cast<__half *>(dst), rows, N, Np);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace spo_detail
