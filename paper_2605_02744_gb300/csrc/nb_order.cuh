// Space-filling-curve order of particles: the cell of a coordinate, its
// Hilbert index, and a CTA-wide bitonic sort of 64-bit keys in shared
// memory.  A Hilbert curve has no jumps between neighbouring indices, so a
// run of consecutive particles is spatially more compact than along a Morton
// (Z-order) curve: fewer overlapping boxes, fewer near (hi/lo) j-sets.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {
namespace dev {

// Spreads the low 10 bits of v so that bit k lands at bit 3k.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 10; ++k) r |= ((v >> k) & 1u) << (3 * k);
    return r;
}

// Index of the cell (x, y, z) (10 bits each) along a 3D Hilbert curve,
// 30 bits: J. Skilling's transposition method (Programming the Hilbert
// curve, AIP Conf. Proc. 707, 2004) -- undo the excess work level by level
// (invert or exchange the low bits), Gray-encode across the axes, then
// interleave the transposed bits with the first axis most significant.
__device__ __forceinline__ uint32_t hilbert30(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t X[3] = {x, y, z};
    for (uint32_t Q = 1u << 9; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = 1u << 9; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

// The cell of one coordinate: (x - lo) * scale clamped to [0, 1023].
__device__ __forceinline__ uint32_t cell10(double x, double lo, double scale) {
    double q = (x - lo) * scale;
    q = q < 0.0 ? 0.0 : (q > 1023.0 ? 1023.0 : q);
    return (uint32_t)q;
}

// Ascending bitonic sort of P (a power of two) 64-bit keys in shared memory
// by the whole CTA (every thread calls it; it ends with a barrier).
__device__ __forceinline__ void block_bitonic_sort(unsigned long long *keys, int P) {
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = threadIdx.x; e < P; e += blockDim.x) {
                const int x = e ^ j;
                if (x > e) {
                    const bool asc = (e & k) == 0;
                    const unsigned long long a = keys[e], b = keys[x];
                    if ((a > b) == asc) {
                        keys[e] = b;
                        keys[x] = a;
                    }
                }
            }
            __syncthreads();
        }
}

}  // namespace dev
}  // namespace nb
