// Hashed-grid encoding of the surrogate: per level, the cell and fraction of
// a position, the C2 quintic interpolation weights with their first and
// second derivatives, and the 8 corner slots with their 5-channel weights
// (value, d/dx, d/dy, d/dz, Laplacian).  Shared by the CUDA-core and the
// tensor-core kernels.
#pragma once

#include <stdint.h>

#include "spo_index.cuh"

namespace spo_dev {

__device__ __forceinline__ void smooth_w(float t, float &s, float &ds, float &d2s) {
    s = t * t * t * fmaf(t, fmaf(6.0f, t, -15.0f), 10.0f);
    const float tm = t - 1.0f;
    ds = 30.0f * t * t * tm * tm;
    d2s = 60.0f * t * tm * fmaf(2.0f, t, -1.0f);
}

// cell (mod R) and fraction of one coordinate at resolution R
__device__ __forceinline__ void level_axis(float r, int R, int &cell, float &t) {
    const float fR = (float)R;
    float fl = floorf(r * fR);
    float tt = fmaf(r, fR, -fl);
    if (tt < 0.0f) { fl -= 1.0f; tt += 1.0f; }
    else if (tt >= 1.0f) { fl += 1.0f; tt -= 1.0f; }
    if (!(tt >= 0.0f && tt <= 1.0f)) tt = 0.0f;
    fl = fminf(fmaxf(fl, -4194304.0f), 4194304.0f);
    int c = (int)fl;
    if ((unsigned)c >= (unsigned)R) {   // outside the unit cell: reduce modulo R
        c %= R;
        if (c < 0) c += R;
    }
    cell = c;
    t = tt;
}

__device__ __forceinline__ uint32_t corner_slot(int R, bool dense, uint32_t mask, int i, int j, int k) {
    if (dense) return (uint32_t)((i * R + j) * R + k);
    return ((uint32_t)i ^ ((uint32_t)j * 2654435761u) ^ ((uint32_t)k * 805459861u)) & mask;
}

// The 8 corner slots of a level (cells already reduced modulo R).
__device__ __forceinline__ void corner_slots(const int (&c)[3], int R, bool dense, uint32_t mask,
                                             uint32_t (&slot)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int bx = (q >> 2) & 1, by = (q >> 1) & 1, bz = q & 1;
        const int i = c[0] + bx == R ? 0 : c[0] + bx;
        const int j = c[1] + by == R ? 0 : c[1] + by;
        const int k = c[2] + bz == R ? 0 : c[2] + bz;
        slot[q] = corner_slot(R, dense, mask, i, j, k);
    }
}

// The 5-channel weights of the 8 corners from the fractions t.
__device__ __forceinline__ void corner_weights(const float (&t)[3], int R, float (&cw)[5][8]) {
    float w[3][2], dw[3][2], d2w[3][2];
    const float fR = (float)R;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float s, ds, d2s;
        smooth_w(t[d], s, ds, d2s);
        w[d][0] = 1.0f - s;
        w[d][1] = s;
        dw[d][0] = -ds * fR;
        dw[d][1] = ds * fR;
        d2w[d][0] = -d2s * fR * fR;
        d2w[d][1] = d2s * fR * fR;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int bx = (q >> 2) & 1, by = (q >> 1) & 1, bz = q & 1;
        const float wx = w[0][bx], wy = w[1][by], wz = w[2][bz];
        cw[0][q] = wx * wy * wz;
        cw[1][q] = dw[0][bx] * wy * wz;
        cw[2][q] = wx * dw[1][by] * wz;
        cw[3][q] = wx * wy * dw[2][bz];
        cw[4][q] = d2w[0][bx] * wy * wz + wx * d2w[1][by] * wz + wx * wy * d2w[2][bz];
    }
}

// The 8 corner slots of a level and their 5-channel weights.
__device__ __forceinline__ void level_corners(const float *pos3, int R, bool dense, uint32_t mask,
                                              uint32_t (&slot)[8], float (&cw)[5][8]) {
    int c[3];
    float t[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) level_axis(pos3[d], R, c[d], t[d]);
    corner_slots(c, R, dense, mask, slot);
    corner_weights(t, R, cw);
}

}  // namespace spo_dev
