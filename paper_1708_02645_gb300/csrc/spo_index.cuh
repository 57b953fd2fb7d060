// Splitting a flat grid-stride index into (outer, inner) parts.  A 64-bit
// integer division is a long software sequence on the GPU; a 32-bit one is a
// few instructions, so the common case (index below 2^31) takes it.
#pragma once

#include <stdint.h>

namespace spo_dev {

// q = a / b and r = a - q b, for a >= 0 and b > 0.
__device__ __forceinline__ int64_t div_index(int64_t a, int b, int &r) {
    if (a <= 0x7fffffff) {
        const uint32_t q = (uint32_t)a / (uint32_t)b;
        r = (int)((uint32_t)a - q * (uint32_t)b);
        return (int64_t)q;
    }
    const int64_t q = a / b;
    r = (int)(a - q * b);
    return q;
}

}  // namespace spo_dev
