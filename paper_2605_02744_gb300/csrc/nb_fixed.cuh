// Exact, order-independent accumulation of floating-point partial sums in
// two-word fixed point, for sums that many CTAs add to at once.
//
// A call fixes one exponent F for every accumulator.  A partial sum v (FP32
// or FP64) becomes the integer X = rint(v 2^F), split as X = hi 2^40 + lo
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

// Adds v to accumulator (word_hi, word_lo); false (nothing added) if v is
// not finite or outside the bound.
__device__ __forceinline__ bool add(unsigned long long *word_hi, unsigned long long *word_lo,
                                    double v, int F) {
    const double X = rint(ldexp(v, F));
    if (!(fabs(X) < 0x1p100)) return false;  // NaN, inf, or beyond the bound
    const double h = floor(X * 0x1p-40);
    const long long hi = (long long)h;
    const unsigned long long lo = (unsigned long long)(X - h * 0x1p40);
    if (hi != 0) atomicAdd(word_hi, (unsigned long long)hi);
    if (lo != 0) atomicAdd(word_lo, lo);
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
