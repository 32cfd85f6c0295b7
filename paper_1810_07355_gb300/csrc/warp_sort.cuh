// Register-resident bitonic sort of 32*N 64-bit keys held by one warp.
// Element e = i * 32 + lane lives in register v[i] of lane `lane`; after the
// call the keys are ascending in e.
#pragma once

#include <stdint.h>

namespace onng {

template <int N> __device__ __forceinline__ void warp_bitonic_sort(unsigned long long (&v)[N], int lane)
{
    static_assert((N & (N - 1)) == 0, "N must be a power of two");
#pragma unroll
    for (int size = 2; size <= 32 * N; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int ii = i ^ jr;
                    if (ii > i) {
                        const bool asc = (((i << 5) | lane) & size) == 0;
                        unsigned long long a = v[i], b = v[ii];
                        const bool sw = asc ? (a > b) : (a < b);
                        v[i] = sw ? b : a;
                        v[ii] = sw ? a : b;
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const bool asc = (((i << 5) | lane) & size) == 0;
                    unsigned long long o = __shfl_xor_sync(0xffffffffu, v[i], j);
                    const bool take_min = (lower == asc);
                    v[i] = take_min ? (o < v[i] ? o : v[i]) : (o > v[i] ? o : v[i]);
                }
            }
        }
    }
}

}  // namespace onng
