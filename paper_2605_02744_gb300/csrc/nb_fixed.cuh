// Exact, order-independent accumulation of floating-point partial sums in
// two-word fixed point, for sums that many CTAs add to at once.
//
// A call fixes one exponent F for every accumulator.  A partial sum v (FP32
// or FP64) becomes the integer X = v 2^F rounded half away from zero (in
// integer arithmetic on the bits of v), split as X = hi 2^40 + lo
// with 0 <= lo < 2^40; hi goes into one 64-bit word and lo into another with
// integer atomic adds.  Integer addition is associative, so the words end the
// same whatever order the adds arrive in: results are bitwise reproducible,
// and the only rounding is the one of each partial to the grid 2^-F.  F is
// chosen from an a-priori bound Bd on every partial and on every total
// (|X| < 2^100), so the words cannot overflow: |hi| < 2^60 per add, and lo
// has 24 bits of headroom (2^24 adds per accumulator).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "nb_internal.h"

namespace nb {
namespace fx {

constexpr int kLoBits = 40;
constexpr int kMagBits = 100;  // |X| < 2^100

// Exponent for totals bounded by `bound` (>= 0): bound 2^F < 2^100.
__host__ __device__ inline int exponent_for(double bound) {
    if (!(bound > 0.0)) return 0;          // all partials are zero
    if (!isfinite(bound)) return -900;     // the FP32 / FP64 sums overflow first
    int e = 0;
    frexp(bound, &e);                      // bound < 2^e
    int F = kMagBits - e;
    return F < -900 ? -900 : (F > 900 ? 900 : F);
}

// The two words' increments (hi, lo) of an FP64 partial v, in integer
// arithmetic on its bits (no FP64 operations, which are slow on this part):
// with v = m 2^(k - 52), m the 53-bit significand, X = m 2^(k - 52 + F) is m
// shifted left (exact) or right (rounded half away from zero), split as
// |X| = H 2^40 + L and negated in two's complement for v < 0.  false (no
// increments) if v is not finite or |X| >= 2^100.  The same source runs on
// the host, where nb_check_fp_conversions checks it.
__host__ __device__ inline bool split_f64(double v, int F, unsigned long long &hi,
                                          unsigned long long &lo) {
    unsigned long long b;
    memcpy(&b, &v, 8);
    const int be = (int)((b >> 52) & 0x7ffu);
    hi = lo = 0;
    if (be == 0x7ff) return false;  // inf or NaN
    unsigned long long m = b & 0xfffffffffffffull;
    if (be) m |= 1ull << 52;
    if (!m) return true;  // +-0
    const int s = (be ? be : 1) - 1075 + F;  // X = m 2^s
    unsigned __int128 X;
    if (s >= 0) {
        if (s > kMagBits - 53) return false;  // beyond the bound
        X = (unsigned __int128)m << s;
    } else {
        if (s < -54) return true;  // below half a grid step
        X = ((unsigned __int128)m + ((unsigned __int128)1 << (-s - 1))) >> (-s);
    }
    if (X >> kMagBits) return false;
    const unsigned long long H = (unsigned long long)(X >> kLoBits);
    const unsigned long long L = (unsigned long long)X & ((1ull << kLoBits) - 1);
    if (b >> 63) {  // two's complement of H 2^40 + L
        hi = L ? ~H : (0ull - H);
        lo = L ? (1ull << kLoBits) - L : 0ull;
    } else {
        hi = H;
        lo = L;
    }
    return true;
}

// Adds v to accumulator (word_hi, word_lo); false (nothing added) if v is
// not finite or outside the bound.
__device__ __forceinline__ bool add(unsigned long long *word_hi, unsigned long long *word_lo,
                                    double v, int F) {
    unsigned long long hi, lo;
    if (!split_f64(v, F, hi, lo)) return false;
    if (hi) atomicAdd(word_hi, hi);
    if (lo) atomicAdd(word_lo, lo);
    return true;
}

// add() for an FP32 partial, in integer arithmetic on its bits (no FP64
// operations, which are slow on this part): with v = m 2^(k - 23), m the
// 24-bit significand, X = m 2^(k - 23 + F) is m shifted left (exact) or
// right (rounded half away from zero; the result is the same for any
// arrival order either way).
__device__ __forceinline__ bool add_f32(unsigned long long *word_hi,
                                        unsigned long long *word_lo, float v, int F) {
    const uint32_t b = __float_as_uint(v);
    const int be = (int)((b >> 23) & 0xffu);
    if (be == 0xff) return false;  // inf or NaN
    uint32_t m = b & 0x7fffffu;
    if (be) m |= 0x800000u;
    if (!m) return true;  // +-0
    const int s = (be ? be : 1) - 150 + F;  // X = m 2^s
    unsigned long long H, L;                // |X| = H 2^40 + L
    if (s >= 0) {
        if (s > kMagBits - 24) return false;  // beyond the bound
        if (s >= kLoBits) {
            H = (unsigned long long)m << (s - kLoBits);
            L = 0;
        } else {
            const unsigned long long X = (unsigned long long)m << s;  // < 2^64
            H = X >> kLoBits;
            L = X & ((1ull << kLoBits) - 1);
        }
    } else {
        if (s < -25) return true;  // below half a grid step
        H = 0;
        L = ((unsigned long long)m + (1ull << (-s - 1))) >> (-s);
    }
    unsigned long long hi, lo;
    if (b >> 31) {  // two's complement of H 2^40 + L
        hi = L ? ~H : (0ull - H);
        lo = L ? (1ull << kLoBits) - L : 0ull;
    } else {
        hi = H;
        lo = L;
    }
    if (hi) atomicAdd(word_hi, hi);
    if (lo) atomicAdd(word_lo, lo);
    return true;
}

// The accumulated value: (signed) hi 2^40 + lo, exactly as a 128-bit
// integer, then rounded once to double and scaled by 2^-F.
__device__ __forceinline__ double value(unsigned long long word_hi, unsigned long long word_lo,
                                        int F) {
    const __int128 t = ((__int128)(long long)word_hi) * ((__int128)1 << kLoBits) +
                       (__int128)word_lo;
    const bool neg = t < 0;
    const unsigned __int128 m = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
    const unsigned long long mh = (unsigned long long)(m >> 64);
    const unsigned long long ml = (unsigned long long)m;
    // mh < 2^40 converts exactly; one more rounding in the sum
    const double d = mh ? ldexp((double)mh, 64) + (double)ml : (double)ml;
    return ldexp(neg ? -d : d, -F);
}

}  // namespace fx
}  // namespace nb
