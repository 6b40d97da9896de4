// Device pieces of the packed symmetric-pair evaluation of the
// single-system FP32 kernel (nb_sym.cu): a lane holds IRJ i-slots, each
// pre-broadcast as (x, x) pairs, and two j-particles of a 64-slot j-set in
// the .x / .y halves of packed f32x2 registers, so every FP32 operation of
// the pair term is a packed one; the j-set rotates through the warp's lanes
// with shuffles and the j-particles' own sums travel with them.  (The
// batched path keeps the one-j-per-lane rotation of nb_sym_core.cuh: with
// its small, near-heavy clusters and 128-slot blocks that form measured
// faster.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nb_device.cuh"

namespace nb {
namespace symj {

using dev::add2;
using dev::f2;
using dev::fma2;
using dev::mul2;
using dev::rsqrt_approx;

// i-side state of one lane: 8 slots as broadcast pairs, their running sums
// per j-stream (.x / .y).
template <int IRJ>
struct ISetJ {
    float2 nx[IRJ], ny[IRJ], nz[IRJ];     // (-x_i.hi, -x_i.hi)
    float nxl[IRJ], nyl[IRJ], nzl[IRJ];   // -x_i.lo
    float2 m[IRJ];                        // (m_i, m_i)
    float2 ax[IRJ], ay[IRJ], az[IRJ], ph[IRJ];  // per j-stream running sums
};

// One rotation step: the lane's i-slots against its two current j.  B*
// receive +m_i r^-3 d and +m_i r^-1 for the two j (the j-side acceleration
// is -B): the step's terms are summed into fresh registers first and added
// to the travelling sums once, so a j-particle's FP32 sum over an item takes
// 32 adds per j-set pass instead of 32 x IRJ (a strong close pair's term
// then meets ~47 later roundings, not ~260).  SELF: i-slots 2 self_h (.x)
// and 2 self_h + 1 (.y) are the j-particles themselves (zero mass).
// A (lo, lo) pair of this thread's i-slots from shared memory, read at
// every use (kept out of registers: only near j-sets need it).
__device__ __forceinline__ float2 lds_pair(const float2 *q) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(dev::smem_addr(q)));
    return v;
}

// LOSM: the i-slots' -x.lo values come as broadcast pairs from shared
// memory (lo2[(c IRJ + k) stride]) instead of registers.
template <int IRJ, bool NEAR, bool SYM, bool POT, bool SELF, bool LOSM>
__device__ __forceinline__ void stepj(ISetJ<IRJ> &S, const float2 e2, const float2 JX, const float2 JY,
                                      const float2 JZ, const float2 JM, const float2 JXL,
                                      const float2 JYL, const float2 JZL, float2 &BX, float2 &BY,
                                      float2 &BZ, float2 &BP, int self_h, const float2 *lo2,
                                      int stride) {
    float2 TX, TY, TZ, TP = f2(0.f, 0.f);  // this step's j-side terms
#pragma unroll
    for (int k = 0; k < IRJ; ++k) {
        float2 dx = add2(JX, S.nx[k]);
        float2 dy = add2(JY, S.ny[k]);
        float2 dz = add2(JZ, S.nz[k]);
        if (NEAR) {
            if (LOSM) {
                dx = add2(dx, add2(JXL, lds_pair(lo2 + (0 * IRJ + k) * stride)));
                dy = add2(dy, add2(JYL, lds_pair(lo2 + (1 * IRJ + k) * stride)));
                dz = add2(dz, add2(JZL, lds_pair(lo2 + (2 * IRJ + k) * stride)));
            } else {
                dx = add2(dx, add2(JXL, f2(S.nxl[k], S.nxl[k])));
                dy = add2(dy, add2(JYL, f2(S.nyl[k], S.nyl[k])));
                dz = add2(dz, add2(JZL, f2(S.nzl[k], S.nzl[k])));
            }
        }
        float2 r2 = fma2(dx, dx, e2);
        r2 = fma2(dy, dy, r2);
        r2 = fma2(dz, dz, r2);
        const float2 ri = f2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 ri3 = mul2(mul2(ri, ri), ri);
        float2 M = JM;
        if (SELF) {
            M.x = (k == 2 * self_h) ? 0.f : M.x;
            M.y = (k == 2 * self_h + 1) ? 0.f : M.y;
        }
        const float2 sj = mul2(M, ri3);
        S.ax[k] = fma2(sj, dx, S.ax[k]);
        S.ay[k] = fma2(sj, dy, S.ay[k]);
        S.az[k] = fma2(sj, dz, S.az[k]);
        if (POT) S.ph[k] = fma2(M, ri, S.ph[k]);
        if (SYM) {
            const float2 si = mul2(S.m[k], ri3);
            if (k == 0) {
                TX = mul2(si, dx);
                TY = mul2(si, dy);
                TZ = mul2(si, dz);
                if (POT) TP = mul2(S.m[k], ri);
            } else {
                TX = fma2(si, dx, TX);
                TY = fma2(si, dy, TY);
                TZ = fma2(si, dz, TZ);
                if (POT) TP = fma2(S.m[k], ri, TP);
            }
        }
    }
    if (SYM) {
        // scalar adds: measured 0.6 % faster than the packed form at 2^20
        BX = f2(__fadd_rn(BX.x, TX.x), __fadd_rn(BX.y, TX.y));
        BY = f2(__fadd_rn(BY.x, TY.x), __fadd_rn(BY.y, TY.y));
        BZ = f2(__fadd_rn(BZ.x, TZ.x), __fadd_rn(BZ.y, TZ.y));
        if (POT) BP = f2(__fadd_rn(BP.x, TP.x), __fadd_rn(BP.y, TP.y));
    }
}

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return f2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// 32 steps over one 64-slot j-set (j[0..6]: slot l, j[7..13]: slot 32 + l);
// b0 / b1: the j-side sums (-a, phi order as BX, BY, BZ, BP) of the two
// j-particles, home again on their lane.
template <int IRJ, bool NEAR, bool SYM, bool POT, bool LOSM>
__device__ __forceinline__ void rotate_setj(ISetJ<IRJ> &S, const float2 e2, const float (&j)[14],
                                            float4 &b0, float4 &b1, int self_h, const float2 *lo2,
                                            int stride) {
    const int src = (threadIdx.x + 1) & 31;
    float2 JX = f2(j[0], j[7]), JY = f2(j[1], j[8]), JZ = f2(j[2], j[9]), JM = f2(j[3], j[10]);
    float2 JXL = f2(j[4], j[11]), JYL = f2(j[5], j[12]), JZL = f2(j[6], j[13]);
    float2 BX = f2(0.f, 0.f), BY = BX, BZ = BX, BP = BX;
    auto rotate = [&]() {
        JX = shfl2(JX, src);
        JY = shfl2(JY, src);
        JZ = shfl2(JZ, src);
        JM = shfl2(JM, src);
        if (NEAR) {
            JXL = shfl2(JXL, src);
            JYL = shfl2(JYL, src);
            JZL = shfl2(JZL, src);
        }
        if (SYM) {
            BX = shfl2(BX, src);
            BY = shfl2(BY, src);
            BZ = shfl2(BZ, src);
            if (POT) BP = shfl2(BP, src);
        }
    };
    int s0 = 0;
    if (self_h >= 0) {
        stepj<IRJ, NEAR, SYM, POT, true, LOSM>(S, e2, JX, JY, JZ, JM, JXL, JYL, JZL, BX, BY, BZ, BP,
                                               self_h, lo2, stride);
        rotate();
        s0 = 1;
    }
#pragma unroll 2
    for (int st = s0; st < 32; ++st) {
        stepj<IRJ, NEAR, SYM, POT, false, LOSM>(S, e2, JX, JY, JZ, JM, JXL, JYL, JZL, BX, BY, BZ, BP,
                                                -1, lo2, stride);
        rotate();
    }
    b0 = make_float4(BX.x, BY.x, BZ.x, BP.x);
    b1 = make_float4(BX.y, BY.y, BZ.y, BP.y);
}

template <int IRJ, int MODE, bool SYM, bool POT, bool LOSM>
__device__ __forceinline__ void run_setj(ISetJ<IRJ> &S, const float2 e2, const float (&j)[14],
                                         bool near, float4 &b0, float4 &b1, int self_h,
                                         const float2 *lo2, int stride) {
    if (MODE == 1 || (MODE == 2 && near))
        rotate_setj<IRJ, true, SYM, POT, LOSM>(S, e2, j, b0, b1, self_h, lo2, stride);
    else
        rotate_setj<IRJ, false, SYM, POT, LOSM>(S, e2, j, b0, b1, self_h, lo2, stride);
}

// j-slots s (.x, j[0..6]) and s + 32 (.y, j[7..13]) of a packed SoA
// [7][Np]: x.hi y.hi z.hi m x.lo y.lo z.lo.
__device__ __forceinline__ void load_pair(const float *soa, int64_t Np, int64_t s,
                                          float (&j)[14]) {
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        j[a] = __ldg(soa + a * Np + s);
        j[7 + a] = __ldg(soa + a * Np + s + 32);
    }
}

}  // namespace symj
}  // namespace nb
