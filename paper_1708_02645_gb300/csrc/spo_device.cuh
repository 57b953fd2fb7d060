// Device helpers shared by the evaluation kernels: coordinate reduction,
// cubic B-spline weights, widening loads and the z -> y -> x reduction of one
// 4x4x4 window for V consecutive orbitals.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "spo.h"

namespace spo_dev {

template <int KIND>
struct Rows {
    static constexpr int value = KIND == SPO_KIND_V ? 1 : (KIND == SPO_KIND_VGL ? 5 : 10);
};

// ---------------------------------------------------------------------------
// debug builds (-DSPO_CHECK_BOUNDS): index checks inside the kernels
// ---------------------------------------------------------------------------
// An index the kernel is about to use satisfies `cond`; when it does not,
// bit 1 of the device status word is set and the caller skips the access.
// Without SPO_CHECK_BOUNDS this is `true` and costs nothing.
__device__ __forceinline__ bool bounds_ok(bool cond, unsigned int *status) {
#ifdef SPO_CHECK_BOUNDS
    if (!cond && status) atomicOr(status, 2u);
    return cond;
#else
    (void)cond;
    (void)status;
    return true;
#endif
}

// ---------------------------------------------------------------------------
// widening loads of V = 2 or 4 consecutive coefficients (global memory via
// the read-only path, or shared memory)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bf16x2(uint32_t r, float *v) {
    // a bf16 is the upper half of the FP32 with the same value
    v[0] = __uint_as_float(r << 16);
    v[1] = __uint_as_float(r & 0xffff0000u);
}

__device__ __forceinline__ void f16x2(uint32_t r, float *v) {
    __half2 h;
    memcpy(&h, &r, 4);
    const float2 f = __half22float2(h);
    v[0] = f.x;
    v[1] = f.y;
}

template <bool GLOBAL, typename W>
__device__ __forceinline__ W fetch(const void *p) {
    if constexpr (GLOBAL) return __ldg(reinterpret_cast<const W *>(p));
    else return *reinterpret_cast<const W *>(p);
}

template <typename T, int V, bool GLOBAL>
__device__ __forceinline__ void load_coefs(const T *p, float *v) {
    static_assert(V == 2 || V == 4, "2 or 4 orbitals per thread");
    if constexpr (sizeof(T) == 4) {
        if constexpr (V == 4) {
            const float4 r = fetch<GLOBAL, float4>(p);
            v[0] = r.x; v[1] = r.y; v[2] = r.z; v[3] = r.w;
        } else {
            const float2 r = fetch<GLOBAL, float2>(p);
            v[0] = r.x; v[1] = r.y;
        }
    } else {
        constexpr bool BF = std::is_same<T, __nv_bfloat16>::value;
        if constexpr (V == 4) {
            const uint2 r = fetch<GLOBAL, uint2>(p);
            if constexpr (BF) { bf16x2(r.x, v); bf16x2(r.y, v + 2); }
            else { f16x2(r.x, v); f16x2(r.y, v + 2); }
        } else {
            const uint32_t r = fetch<GLOBAL, uint32_t>(p);
            if constexpr (BF) bf16x2(r, v);
            else f16x2(r, v);
        }
    }
}

// ---------------------------------------------------------------------------
// per-position geometry
// ---------------------------------------------------------------------------

// Per-axis constants of a grid: n intervals, n and n^2 as floats, 1/n.
struct GridAxis {
    int n;
    float fn, fn2, inv;
};

inline GridAxis grid_axis(int n) {
    return GridAxis{n, (float)n, (float)n * (float)n, 1.0f / (float)n};
}

// Cell index i in [0, n) and fraction t in [0, 1] of coordinate r on a
// periodic axis of n intervals.  t = r*n - floor(r*n) is formed with one
// fused multiply-add, so it is the FP32 rounding of the exact fraction.
// The cell is reduced modulo n in floating point: with |floor(r n)| <= 2^22
// the quotient q = floor(fl / n) is off by at most one, which one range
// check corrects, and fl - q n is an exact small integer.  Coordinates
// beyond 2^22 cells (which carry no fractional bits in FP32 anyway), NaN and
// Inf land in an unspecified cell; the final clamp keeps every index in
// range whatever the input.
__device__ __forceinline__ void reduce_axis(float r, const GridAxis &g, int &cell, float &t) {
    float fl = floorf(r * g.fn);
    float tt = fmaf(r, g.fn, -fl);
    if (tt < 0.0f) {
        fl -= 1.0f;
        tt += 1.0f;
    } else if (tt >= 1.0f) {
        fl += 1.0f;
        tt -= 1.0f;
    }
    if (!(tt >= 0.0f && tt <= 1.0f)) tt = 0.0f;
    fl = fminf(fmaxf(fl, -4194304.0f), 4194304.0f);   // |fl| <= 2^22; fmaxf maps NaN to the bound
    const float q = floorf(fl * g.inv);
    float c = fmaf(-q, g.fn, fl);
    if (c < 0.0f) c += g.fn;
    else if (c >= g.fn) c -= g.fn;
    cell = min(max((int)c, 0), g.n - 1);
    t = tt;
}

// Cubic B-spline weight of window node A (A = 0..3 for nodes i-1 .. i+2) at
// fraction t, with its first and second derivatives scaled to d/dr
// (factors n and n^2).  Every kernel computes a weight with this one
// function, so weights (and the sums built from them) agree bit for bit.
template <int A>
__device__ __forceinline__ void node_weights(float t, const GridAxis &g, float &w, float &d,
                                             float &dd) {
    if constexpr (A == 0) {
        const float s = 1.0f - t, s2 = s * s;
        w = (1.0f / 6.0f) * s2 * s;
        d = -0.5f * s2 * g.fn;
        dd = s * g.fn2;
    } else if constexpr (A == 1) {
        const float t2 = t * t;
        w = fmaf(t2, fmaf(0.5f, t, -1.0f), 2.0f / 3.0f);
        d = fmaf(1.5f, t, -2.0f) * t * g.fn;
        dd = fmaf(3.0f, t, -2.0f) * g.fn2;
    } else if constexpr (A == 2) {
        w = fmaf(fmaf(fmaf(-0.5f, t, 0.5f), t, 0.5f), t, 1.0f / 6.0f);
        d = fmaf(fmaf(-1.5f, t, 1.0f), t, 0.5f) * g.fn;
        dd = fmaf(-3.0f, t, 1.0f) * g.fn2;
    } else {
        const float t2 = t * t;
        w = (1.0f / 6.0f) * t2 * t;
        d = 0.5f * t2 * g.fn;
        dd = t * g.fn2;
    }
}

// Fraction, cell and all twelve weights of one axis (y and z, which every
// x node of the window reuses).
struct Axis {
    float w[4], d[4], dd[4];
    int cell;
};

__device__ __forceinline__ void make_axis(float r, const GridAxis &g, Axis &ax) {
    float t;
    reduce_axis(r, g, ax.cell, t);
    node_weights<0>(t, g, ax.w[0], ax.d[0], ax.dd[0]);
    node_weights<1>(t, g, ax.w[1], ax.d[1], ax.dd[1]);
    node_weights<2>(t, g, ax.w[2], ax.d[2], ax.dd[2]);
    node_weights<3>(t, g, ax.w[3], ax.d[3], ax.dd[3]);
}

// Fraction and cell of the x axis: its weights are formed node by node
// inside the window reduction (fewer live registers).
struct XAxis {
    float t;
    int cell;
};

__device__ __forceinline__ void make_xaxis(float r, const GridAxis &g, XAxis &ax) {
    reduce_axis(r, g, ax.cell, ax.t);
}

// ---------------------------------------------------------------------------
// the window reduction
// ---------------------------------------------------------------------------
// Accumulate the terms of x node A (weights xw, xd, xdd) of one window into
// acc[NC][V], for V consecutive orbitals; node A = 0 initialises acc.
// load(a, b, g, v) fetches the V coefficients of corner (a, b, g).  The
// first term of every sum is a product and each later term one FMA, in a
// fixed order, so all kernels produce the same bits for the same position
// and orbitals.
// Packed form for an even number of orbitals: every operation acts on two
// orbitals at once (fma.rn.f32x2 / mul.rn.f32x2 on sm_100 and later), each
// lane rounding exactly as the scalar form, so the results are the same bits.
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

template <int KIND, int V, int A, typename Load>
__device__ __forceinline__ void window_x_node_packed(float xw, float xd, float xdd, const Axis &Y,
                                                     const Axis &Z, Load &load,
                                                     float (&acc)[Rows<KIND>::value][V]) {
    constexpr int NY = KIND == SPO_KIND_V ? 1 : (KIND == SPO_KIND_VGL ? 5 : 6);
    constexpr int NP = V / 2;
    float2 ys[NY][NP];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float cv[4][V];
#pragma unroll
        for (int g = 0; g < 4; ++g) load(A, b, g, cv[g]);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 c0 = make_float2(cv[0][2 * k], cv[0][2 * k + 1]);
            const float2 c1 = make_float2(cv[1][2 * k], cv[1][2 * k + 1]);
            const float2 c2 = make_float2(cv[2][2 * k], cv[2][2 * k + 1]);
            const float2 c3 = make_float2(cv[3][2 * k], cv[3][2 * k + 1]);
            float2 zv = __fmul2_rn(bc2(Z.w[0]), c0);
            zv = __ffma2_rn(bc2(Z.w[1]), c1, zv);
            zv = __ffma2_rn(bc2(Z.w[2]), c2, zv);
            zv = __ffma2_rn(bc2(Z.w[3]), c3, zv);
            float2 zd = make_float2(0.0f, 0.0f), zdd = make_float2(0.0f, 0.0f);
            if constexpr (KIND != SPO_KIND_V) {
                zd = __fmul2_rn(bc2(Z.d[0]), c0);
                zd = __ffma2_rn(bc2(Z.d[1]), c1, zd);
                zd = __ffma2_rn(bc2(Z.d[2]), c2, zd);
                zd = __ffma2_rn(bc2(Z.d[3]), c3, zd);
                zdd = __fmul2_rn(bc2(Z.dd[0]), c0);
                zdd = __ffma2_rn(bc2(Z.dd[1]), c1, zdd);
                zdd = __ffma2_rn(bc2(Z.dd[2]), c2, zdd);
                zdd = __ffma2_rn(bc2(Z.dd[3]), c3, zdd);
            }
            if (b == 0) {
                ys[0][k] = __fmul2_rn(bc2(Y.w[0]), zv);
                if constexpr (KIND != SPO_KIND_V) {
                    ys[1][k] = __fmul2_rn(bc2(Y.d[0]), zv);
                    ys[2][k] = __fmul2_rn(bc2(Y.dd[0]), zv);
                    ys[3][k] = __fmul2_rn(bc2(Y.w[0]), zd);
                    if constexpr (KIND == SPO_KIND_VGH) {
                        ys[4][k] = __fmul2_rn(bc2(Y.d[0]), zd);
                        ys[5][k] = __fmul2_rn(bc2(Y.w[0]), zdd);
                    } else {
                        ys[4][k] = __fmul2_rn(bc2(Y.w[0]), zdd);
                    }
                }
            } else {
                ys[0][k] = __ffma2_rn(bc2(Y.w[b]), zv, ys[0][k]);
                if constexpr (KIND != SPO_KIND_V) {
                    ys[1][k] = __ffma2_rn(bc2(Y.d[b]), zv, ys[1][k]);
                    ys[2][k] = __ffma2_rn(bc2(Y.dd[b]), zv, ys[2][k]);
                    ys[3][k] = __ffma2_rn(bc2(Y.w[b]), zd, ys[3][k]);
                    if constexpr (KIND == SPO_KIND_VGH) {
                        ys[4][k] = __ffma2_rn(bc2(Y.d[b]), zd, ys[4][k]);
                        ys[5][k] = __ffma2_rn(bc2(Y.w[b]), zdd, ys[5][k]);
                    } else {
                        ys[4][k] = __ffma2_rn(bc2(Y.w[b]), zdd, ys[4][k]);
                    }
                }
            }
        }
    }
    // x stage
    const float2 w2 = bc2(xw), d2 = bc2(xd), dd2 = bc2(xdd);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        constexpr int NC = Rows<KIND>::value;
        float2 a[NC];
        if constexpr (A == 0) {
            a[0] = __fmul2_rn(w2, ys[0][k]);                        // v
            if constexpr (KIND == SPO_KIND_VGH) {
                a[1] = __fmul2_rn(d2, ys[0][k]);                    // gx
                a[2] = __fmul2_rn(w2, ys[1][k]);                    // gy
                a[3] = __fmul2_rn(w2, ys[3][k]);                    // gz
                a[4] = __fmul2_rn(dd2, ys[0][k]);                   // hxx
                a[5] = __fmul2_rn(d2, ys[1][k]);                    // hxy
                a[6] = __fmul2_rn(d2, ys[3][k]);                    // hxz
                a[7] = __fmul2_rn(w2, ys[2][k]);                    // hyy
                a[8] = __fmul2_rn(w2, ys[4][k]);                    // hyz
                a[9] = __fmul2_rn(w2, ys[5][k]);                    // hzz
            } else if constexpr (KIND == SPO_KIND_VGL) {
                a[1] = __fmul2_rn(d2, ys[0][k]);
                a[2] = __fmul2_rn(w2, ys[1][k]);
                a[3] = __fmul2_rn(w2, ys[3][k]);
                float2 l = __fmul2_rn(dd2, ys[0][k]);
                l = __ffma2_rn(w2, ys[2][k], l);
                a[4] = __ffma2_rn(w2, ys[4][k], l);
            }
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) a[c] = make_float2(acc[c][2 * k], acc[c][2 * k + 1]);
            a[0] = __ffma2_rn(w2, ys[0][k], a[0]);
            if constexpr (KIND == SPO_KIND_VGH) {
                a[1] = __ffma2_rn(d2, ys[0][k], a[1]);
                a[2] = __ffma2_rn(w2, ys[1][k], a[2]);
                a[3] = __ffma2_rn(w2, ys[3][k], a[3]);
                a[4] = __ffma2_rn(dd2, ys[0][k], a[4]);
                a[5] = __ffma2_rn(d2, ys[1][k], a[5]);
                a[6] = __ffma2_rn(d2, ys[3][k], a[6]);
                a[7] = __ffma2_rn(w2, ys[2][k], a[7]);
                a[8] = __ffma2_rn(w2, ys[4][k], a[8]);
                a[9] = __ffma2_rn(w2, ys[5][k], a[9]);
            } else if constexpr (KIND == SPO_KIND_VGL) {
                a[1] = __ffma2_rn(d2, ys[0][k], a[1]);
                a[2] = __ffma2_rn(w2, ys[1][k], a[2]);
                a[3] = __ffma2_rn(w2, ys[3][k], a[3]);
                float2 l = __ffma2_rn(dd2, ys[0][k], a[4]);
                l = __ffma2_rn(w2, ys[2][k], l);
                a[4] = __ffma2_rn(w2, ys[4][k], l);
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            acc[c][2 * k] = a[c].x;
            acc[c][2 * k + 1] = a[c].y;
        }
    }
}

template <int KIND, int V, int A, typename Load>
__device__ __forceinline__ void window_x_node(float xw, float xd, float xdd, const Axis &Y,
                                              const Axis &Z, Load &load,
                                              float (&acc)[Rows<KIND>::value][V]) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (V % 2 == 0) {
        window_x_node_packed<KIND, V, A>(xw, xd, xdd, Y, Z, load, acc);
        return;
    }
#endif
    constexpr int NY = KIND == SPO_KIND_V ? 1 : (KIND == SPO_KIND_VGL ? 5 : 6);
    // y-stage partial sums for this x node
    //   VGH: wy*v, dy*v, ddy*v, wy*dz, dy*dz, wy*ddz
    //   VGL: wy*v, dy*v, ddy*v, wy*dz, wy*ddz
    //   V:   wy*v
    float ys[NY][V];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float cv[4][V];
#pragma unroll
        for (int g = 0; g < 4; ++g) load(A, b, g, cv[g]);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            float zv = Z.w[0] * cv[0][k];
            zv = fmaf(Z.w[1], cv[1][k], zv);
            zv = fmaf(Z.w[2], cv[2][k], zv);
            zv = fmaf(Z.w[3], cv[3][k], zv);
            float zd = 0.0f, zdd = 0.0f;
            if constexpr (KIND != SPO_KIND_V) {
                zd = Z.d[0] * cv[0][k];
                zd = fmaf(Z.d[1], cv[1][k], zd);
                zd = fmaf(Z.d[2], cv[2][k], zd);
                zd = fmaf(Z.d[3], cv[3][k], zd);
                zdd = Z.dd[0] * cv[0][k];
                zdd = fmaf(Z.dd[1], cv[1][k], zdd);
                zdd = fmaf(Z.dd[2], cv[2][k], zdd);
                zdd = fmaf(Z.dd[3], cv[3][k], zdd);
            }
            if (b == 0) {
                ys[0][k] = Y.w[0] * zv;
                if constexpr (KIND != SPO_KIND_V) {
                    ys[1][k] = Y.d[0] * zv;
                    ys[2][k] = Y.dd[0] * zv;
                    ys[3][k] = Y.w[0] * zd;
                    if constexpr (KIND == SPO_KIND_VGH) {
                        ys[4][k] = Y.d[0] * zd;
                        ys[5][k] = Y.w[0] * zdd;
                    } else {
                        ys[4][k] = Y.w[0] * zdd;
                    }
                }
            } else {
                ys[0][k] = fmaf(Y.w[b], zv, ys[0][k]);
                if constexpr (KIND != SPO_KIND_V) {
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
    }
    // x stage
#pragma unroll
    for (int k = 0; k < V; ++k) {
        if constexpr (A == 0) {
            acc[0][k] = xw * ys[0][k];                              // v
            if constexpr (KIND == SPO_KIND_VGH) {
                acc[1][k] = xd * ys[0][k];                          // gx
                acc[2][k] = xw * ys[1][k];                          // gy
                acc[3][k] = xw * ys[3][k];                          // gz
                acc[4][k] = xdd * ys[0][k];                         // hxx
                acc[5][k] = xd * ys[1][k];                          // hxy
                acc[6][k] = xd * ys[3][k];                          // hxz
                acc[7][k] = xw * ys[2][k];                          // hyy
                acc[8][k] = xw * ys[4][k];                          // hyz
                acc[9][k] = xw * ys[5][k];                          // hzz
            } else if constexpr (KIND == SPO_KIND_VGL) {
                acc[1][k] = xd * ys[0][k];                          // gx
                acc[2][k] = xw * ys[1][k];                          // gy
                acc[3][k] = xw * ys[3][k];                          // gz
                // lap = hxx + hyy + hzz
                float l = xdd * ys[0][k];
                l = fmaf(xw, ys[2][k], l);
                acc[4][k] = fmaf(xw, ys[4][k], l);
            }
        } else {
            acc[0][k] = fmaf(xw, ys[0][k], acc[0][k]);
            if constexpr (KIND == SPO_KIND_VGH) {
                acc[1][k] = fmaf(xd, ys[0][k], acc[1][k]);
                acc[2][k] = fmaf(xw, ys[1][k], acc[2][k]);
                acc[3][k] = fmaf(xw, ys[3][k], acc[3][k]);
                acc[4][k] = fmaf(xdd, ys[0][k], acc[4][k]);
                acc[5][k] = fmaf(xd, ys[1][k], acc[5][k]);
                acc[6][k] = fmaf(xd, ys[3][k], acc[6][k]);
                acc[7][k] = fmaf(xw, ys[2][k], acc[7][k]);
                acc[8][k] = fmaf(xw, ys[4][k], acc[8][k]);
                acc[9][k] = fmaf(xw, ys[5][k], acc[9][k]);
            } else if constexpr (KIND == SPO_KIND_VGL) {
                acc[1][k] = fmaf(xd, ys[0][k], acc[1][k]);
                acc[2][k] = fmaf(xw, ys[1][k], acc[2][k]);
                acc[3][k] = fmaf(xw, ys[3][k], acc[3][k]);
                float l = fmaf(xdd, ys[0][k], acc[4][k]);
                l = fmaf(xw, ys[2][k], l);
                acc[4][k] = fmaf(xw, ys[4][k], l);
            }
        }
    }
}

// acc[NC][V] = the 64-term sums of one window (x nodes 0..3 in order).
// FENCE puts a compiler barrier between x nodes, so that the loads of one
// node are not hoisted above the arithmetic of the previous one: with
// short-latency shared-memory loads this keeps register use under the
// launch bound; global-memory kernels leave the scheduler free.
template <int KIND, int V, bool FENCE, typename Load>
__device__ __forceinline__ void window_reduce(const XAxis &X, const GridAxis &gx, const Axis &Y,
                                              const Axis &Z, Load load,
                                              float (&acc)[Rows<KIND>::value][V]) {
    float xw, xd, xdd;
    node_weights<0>(X.t, gx, xw, xd, xdd);
    window_x_node<KIND, V, 0>(xw, xd, xdd, Y, Z, load, acc);
    if constexpr (FENCE) asm volatile("" ::: "memory");
    node_weights<1>(X.t, gx, xw, xd, xdd);
    window_x_node<KIND, V, 1>(xw, xd, xdd, Y, Z, load, acc);
    if constexpr (FENCE) asm volatile("" ::: "memory");
    node_weights<2>(X.t, gx, xw, xd, xdd);
    window_x_node<KIND, V, 2>(xw, xd, xdd, Y, Z, load, acc);
    if constexpr (FENCE) asm volatile("" ::: "memory");
    node_weights<3>(X.t, gx, xw, xd, xdd);
    window_x_node<KIND, V, 3>(xw, xd, xdd, Y, Z, load, acc);
}

// Weight slot of one position (kSlotF4 float4), used by the brick kernels:
// x-node weights (w, w', w'', 0) for nodes 0..3, then y's w[4], w'[4],
// w''[4], then z's, then the cells (x, y, z) and the position's index as
// ints.  The binning can form the slots of all positions once
// (make_weight_record, one thread per position) so that every orbital tile
// only copies them; otherwise lanes 0, 1 and 2 of a position's group each
// reduce one axis and form its four nodes' weights (stage_axis_weights) and
// the group reads them back.  Either way the weights come from reduce_axis
// and node_weights, the functions every kernel uses, so the bits are those
// of the gather kernel.  A slot is 176 bytes (44 words), so the four
// 16-byte reads of a warp's four groups fall in disjoint banks.
constexpr int kSlotF4 = 11;

__device__ __forceinline__ void unpack4(const float4 &r, float (&v)[4]) {
    v[0] = r.x; v[1] = r.y; v[2] = r.z; v[3] = r.w;
}

// Cell, and the weights of the four window nodes, of coordinate u on axis g.
__device__ __forceinline__ void axis_weights(float u, const GridAxis &g, int &cell, float (&w)[4],
                                             float (&d)[4], float (&dd)[4]) {
    float t;
    reduce_axis(u, g, cell, t);
    node_weights<0>(t, g, w[0], d[0], dd[0]);
    node_weights<1>(t, g, w[1], d[1], dd[1]);
    node_weights<2>(t, g, w[2], d[2], dd[2]);
    node_weights<3>(t, g, w[3], d[3], dd[3]);
}

// The whole slot of position p at r = (x, y, z), formed by one thread.
__device__ __forceinline__ void make_weight_record(const float4 &r, int p, const GridAxis &gx,
                                                   const GridAxis &gy, const GridAxis &gz,
                                                   float4 *__restrict__ rec) {
    int cx, cy, cz;
    float w[4], d[4], dd[4];
    axis_weights(r.x, gx, cx, w, d, dd);
#pragma unroll
    for (int n = 0; n < 4; ++n) rec[n] = make_float4(w[n], d[n], dd[n], 0.0f);
    axis_weights(r.y, gy, cy, w, d, dd);
    rec[4] = make_float4(w[0], w[1], w[2], w[3]);
    rec[5] = make_float4(d[0], d[1], d[2], d[3]);
    rec[6] = make_float4(dd[0], dd[1], dd[2], dd[3]);
    axis_weights(r.z, gz, cz, w, d, dd);
    rec[7] = make_float4(w[0], w[1], w[2], w[3]);
    rec[8] = make_float4(d[0], d[1], d[2], d[3]);
    rec[9] = make_float4(dd[0], dd[1], dd[2], dd[3]);
    rec[10] = make_float4(__int_as_float(cx), __int_as_float(cy), __int_as_float(cz), __int_as_float(p));
}

// Lane q of a position's group forms its part of the slot from the
// position record r = (x, y, z, index bits): lanes 0, 1, 2 the x, y, z axes
// (and lane 0 the index); lanes 3.. repeat the x axis and store nothing.
__device__ __forceinline__ void stage_axis_weights(int q, const float4 &r, const GridAxis &gx,
                                                   const GridAxis &gy, const GridAxis &gz,
                                                   float4 *slot) {
    const int a = q < 3 ? q : 0;
    const GridAxis g = a == 0 ? gx : (a == 1 ? gy : gz);
    const float u = a == 0 ? r.x : (a == 1 ? r.y : r.z);
    int cell;
    float w[4], d[4], dd[4];
    axis_weights(u, g, cell, w, d, dd);
    if (q == 0) {
#pragma unroll
        for (int n = 0; n < 4; ++n) slot[n] = make_float4(w[n], d[n], dd[n], 0.0f);
    } else if (q < 3) {
        float4 *s = slot + 4 + 3 * (q - 1);
        s[0] = make_float4(w[0], w[1], w[2], w[3]);
        s[1] = make_float4(d[0], d[1], d[2], d[3]);
        s[2] = make_float4(dd[0], dd[1], dd[2], dd[3]);
    }
    if (q < 3) reinterpret_cast<int *>(slot + 10)[q] = cell;
    if (q == 0) reinterpret_cast<int *>(slot + 10)[3] = __float_as_int(r.w);
}

// window_reduce with the x-node weights taken from xs[A] = (w, w', w'', -)
// (formed elsewhere by node_weights<A>, so the sums carry the same bits).
// With FENCE each node's weights are read after the previous node's
// arithmetic.
template <int KIND, int V, bool FENCE, typename Load>
__device__ __forceinline__ void window_reduce_staged(const float4 *xs, const Axis &Y, const Axis &Z,
                                                     Load load, float (&acc)[Rows<KIND>::value][V]) {
    float4 x = xs[0];
    window_x_node<KIND, V, 0>(x.x, x.y, x.z, Y, Z, load, acc);
    if constexpr (FENCE) asm volatile("" ::: "memory");
    x = xs[1];
    window_x_node<KIND, V, 1>(x.x, x.y, x.z, Y, Z, load, acc);
    if constexpr (FENCE) asm volatile("" ::: "memory");
    x = xs[2];
    window_x_node<KIND, V, 2>(x.x, x.y, x.z, Y, Z, load, acc);
    if constexpr (FENCE) asm volatile("" ::: "memory");
    x = xs[3];
    window_x_node<KIND, V, 3>(x.x, x.y, x.z, Y, Z, load, acc);
}

// Streaming store of the NC x V results of one thread; o points at this
// thread's first orbital in component 0 of one position, N is the row
// stride, `left` orbitals remain in the row from that first orbital.  With
// VEC_OUT, V values go out as one 8- or 16-byte store per component (the
// caller guarantees alignment and N % V == 0).
template <int NC, int V, bool VEC_OUT>
__device__ __forceinline__ void store_rows(float *o, int64_t N, int64_t left,
                                           const float (&acc)[NC][V]) {
    if constexpr (VEC_OUT) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if constexpr (V == 4)
                __stcs(reinterpret_cast<float4 *>(o + c * N),
                       make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]));
            else
                __stcs(reinterpret_cast<float2 *>(o + c * N), make_float2(acc[c][0], acc[c][1]));
        }
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (k < left) __stcs(o + c * N + k, acc[c][k]);
    }
}

}  // namespace spo_dev
