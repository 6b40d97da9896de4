// FP32 <-> FP64 conversions and the FP64 finiteness test in integer
// arithmetic on the IEEE 754 bit patterns, for kernels bound by the FP64
// pipe: on this part FP64 runs at a small fraction of the FP32 rate and the
// conversion and comparison instructions share that pipe, while the integer
// pipes are idle in those kernels.
//
// f2d gives exactly the IEEE result of (double)f (the conversion is exact)
// and d2f that of (float)d in round-to-nearest-even, for every input:
// zeros, subnormals, normal numbers, overflow to infinity, infinities; NaNs
// stay NaNs with their sign, quiet bit set.  The same source runs on the
// host, where nb_check_fp_conversions compares it with the C conversions.
#pragma once

#include <stdint.h>
#include <string.h>

#include <cuda_runtime.h>

namespace nb {
namespace fpconv {

__host__ __device__ inline uint32_t bits_f(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
#endif
}
__host__ __device__ inline float from_bits_f(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}
__host__ __device__ inline uint64_t bits_d(double d) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    memcpy(&b, &d, 8);
    return b;
#endif
}
__host__ __device__ inline double from_bits_d(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, 8);
    return d;
#endif
}
__host__ __device__ inline int clz32(uint32_t x) {  // x != 0
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return __builtin_clz(x);
#endif
}

// (double)f: the exponent re-biased from 127 to 1023 and the significand
// moved up by 52 - 23 = 29 bits; a subnormal f is normalised first.
__host__ __device__ inline double f2d(float f) {
    const uint32_t b = bits_f(f);
    const uint64_t sign = (uint64_t)(b >> 31) << 63;
    uint32_t e = (b >> 23) & 0xffu;
    uint32_t m = b & 0x7fffffu;
    uint64_t ed;
    if (e == 0xffu) {
        ed = 0x7ffu;                     // inf, NaN
        if (m) m |= 0x400000u;           // NaN: quiet
    } else if (e != 0u) {
        ed = e + 896u;                   // normal
    } else if (m == 0u) {
        ed = 0u;                         // +-0
    } else {
        const int sh = clz32(m) - 8;     // subnormal: shift the leading one to bit 23
        m = (m << sh) & 0x7fffffu;
        ed = (uint64_t)(897 - sh);
    }
    return from_bits_d(sign | (ed << 52) | ((uint64_t)m << 29));
}

// (float)d, round to nearest even.  With S the 53-bit significand, d =
// S 2^(ed - 1075); the float keeps K = S >> sh, sh = 29 for a normal result
// and more for a subnormal one, plus one where the dropped bits are above
// half, or exactly half with K odd.  A carry out of K moves into the
// exponent field (to infinity past the largest float); a subnormal K that
// rounds up to 2^23 becomes the smallest normal number the same way.
__host__ __device__ inline float d2f(double d) {
    const uint64_t b = bits_d(d);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const uint32_t ed = (uint32_t)(b >> 52) & 0x7ffu;
    const uint64_t m = b & 0xfffffffffffffull;
    if (ed == 0x7ffu)  // inf, NaN (quiet)
        return from_bits_f(sign | 0x7f800000u | (m ? 0x400000u | (uint32_t)(m >> 29) : 0u));
    if (ed == 0u) return from_bits_f(sign);  // zero or below 2^-1022: rounds to zero
    const int fe = (int)ed - 896;            // float exponent field of a normal result
    if (fe >= 0xff) return from_bits_f(sign | 0x7f800000u);
    const int sh = fe >= 1 ? 29 : 30 - fe;
    if (sh > 54) return from_bits_f(sign);   // below half the smallest subnormal
    const uint64_t S = m | (1ull << 52);
    uint32_t K = (uint32_t)(S >> sh);
    const uint64_t rest = S & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rest > half || (rest == half && (K & 1u))) ++K;
    return from_bits_f(sign | ((fe >= 1 ? (uint32_t)(fe - 1) << 23 : 0u) + K));
}

// isfinite(d) from the exponent field alone.
__host__ __device__ inline bool finite_d(double d) {
    return (bits_d(d) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

}  // namespace fpconv
}  // namespace nb
