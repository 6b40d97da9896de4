// Device pieces shared by the symmetric-pair kernels (single system:
// nb_sym.cu; batches of systems: nb_bsym.cu): the lane-rotation evaluation
// of one 32-particle j-set against a warp's 128 i-slots, the box test of
// the adaptive displacement.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace symcore {

using dev::Acc;
using dev::add2;
using dev::f2;
using dev::fma2;
using dev::mul2;
using dev::rsqrt_approx;

constexpr int NW = 16;              // warps per CTA
constexpr int NT = NW * 32;         // threads per CTA
constexpr int IR = 4;               // i-slots per lane (two packed pairs)
constexpr int JS = 32;              // slots per j-set (one per lane)

__device__ __forceinline__ bool boxes_near(const float *a, const float *b, float gamma) {
    float g2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gap = fmaxf(0.f, fmaxf(b[c] - a[3 + c], a[c] - b[3 + c]));
        g2 = fmaf(gap, gap, g2);
    }
    const float X = gamma * fmaxf(a[6], b[6]);
    return g2 < X * X;
}

// i-side state of one lane: four slots as two packed pairs (g = 0, 1).
struct ISet {
    float2 nx[2], ny[2], nz[2];     // -x.hi
    float2 nxl[2], nyl[2], nzl[2];  // -x.lo
    float2 m[2], nm[2];             // m_i, -m_i
    float2 ax[2], ay[2], az[2], ph[2];
};

// One rotation step: the lane's four i-slots against its current j.  NEAR:
// bit g set = packed group g (i-slots 2g, 2g + 1) takes the hi/lo
// displacement.  With SELF, i-slot self_k is the j-particle itself: its half
// of the pair gets a zero mass (Eq. 1 leaves out j = i).  POT: also the
// potential sums (2 of the 18 FP32 operations per unordered pair).
template <int NEAR, bool SYM, bool SELF, bool POT>
__device__ __forceinline__ void step(ISet &S, const float2 e2, float jx, float jy, float jz,
                                     float jm, float jxl, float jyl, float jzl, float &bx,
                                     float &by, float &bz, float &bp, int self_k = -1) {
    const float2 X = f2(jx, jx), Y = f2(jy, jy), Z = f2(jz, jz);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const float2 M = SELF ? f2(self_k == 2 * g ? 0.f : jm, self_k == 2 * g + 1 ? 0.f : jm)
                              : f2(jm, jm);
        float2 dx = add2(X, S.nx[g]);
        float2 dy = add2(Y, S.ny[g]);
        float2 dz = add2(Z, S.nz[g]);
        if ((NEAR >> g) & 1) {
            dx = add2(dx, add2(f2(jxl, jxl), S.nxl[g]));
            dy = add2(dy, add2(f2(jyl, jyl), S.nyl[g]));
            dz = add2(dz, add2(f2(jzl, jzl), S.nzl[g]));
        }
        float2 r2 = fma2(dx, dx, e2);
        r2 = fma2(dy, dy, r2);
        r2 = fma2(dz, dz, r2);
        const float2 ri = f2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 ri3 = mul2(mul2(ri, ri), ri);
        const float2 sj = mul2(M, ri3);
        S.ax[g] = fma2(sj, dx, S.ax[g]);
        S.ay[g] = fma2(sj, dy, S.ay[g]);
        S.az[g] = fma2(sj, dz, S.az[g]);
        if (POT) S.ph[g] = fma2(M, ri, S.ph[g]);
        if (SYM) {
            const float2 si = mul2(S.nm[g], ri3);  // -m_i r^-3
            bx = fmaf(si.x, dx.x, bx);
            bx = fmaf(si.y, dx.y, bx);
            by = fmaf(si.x, dy.x, by);
            by = fmaf(si.y, dy.y, by);
            bz = fmaf(si.x, dz.x, bz);
            bz = fmaf(si.y, dz.y, bz);
            if (POT) {
                bp = fmaf(S.m[g].x, ri.x, bp);
                bp = fmaf(S.m[g].y, ri.y, bp);
            }
        }
    }
}

// 32 steps over one j-set; the j values (and sums) end on their home lane.
// self_k >= 0 (diagonal items only): the j-set is the warp's own i-slots
// 32 self_k + [0, 32), so step 0 pairs every lane with itself.
template <int NEAR, bool SYM, bool POT>
__device__ __forceinline__ void rotate_set(ISet &S, const float2 e2, const float (&j)[7],
                                           float4 &b, int self_k) {
    const int src = (threadIdx.x + 1) & 31;
    float jx = j[0], jy = j[1], jz = j[2], jm = j[3], jxl = j[4], jyl = j[5], jzl = j[6];
    float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
    auto rotate = [&]() {
        jx = __shfl_sync(0xffffffffu, jx, src);
        jy = __shfl_sync(0xffffffffu, jy, src);
        jz = __shfl_sync(0xffffffffu, jz, src);
        jm = __shfl_sync(0xffffffffu, jm, src);
        if (NEAR != 0) {
            jxl = __shfl_sync(0xffffffffu, jxl, src);
            jyl = __shfl_sync(0xffffffffu, jyl, src);
            jzl = __shfl_sync(0xffffffffu, jzl, src);
        }
        if (SYM) {
            bx = __shfl_sync(0xffffffffu, bx, src);
            by = __shfl_sync(0xffffffffu, by, src);
            bz = __shfl_sync(0xffffffffu, bz, src);
            if (POT) bp = __shfl_sync(0xffffffffu, bp, src);
        }
    };
    int s0 = 0;
    if (self_k >= 0) {
        step<NEAR, SYM, true, POT>(S, e2, jx, jy, jz, jm, jxl, jyl, jzl, bx, by, bz, bp, self_k);
        rotate();
        s0 = 1;
    }
#pragma unroll 4
    for (int s = s0; s < JS; ++s) {
        step<NEAR, SYM, false, POT>(S, e2, jx, jy, jz, jm, jxl, jyl, jzl, bx, by, bz, bp);
        rotate();
    }
    b = make_float4(bx, by, bz, bp);
}

template <int MODE, bool SYM, bool POT>
__device__ __forceinline__ void run_set(ISet &S, const float2 e2, const float (&j)[7], bool near,
                                        float4 &b, int self_k) {
    if (MODE == 1 || (MODE == 2 && near))
        rotate_set<3, SYM, POT>(S, e2, j, b, self_k);
    else
        rotate_set<0, SYM, POT>(S, e2, j, b, self_k);
}

// The same with a separate near/far choice for the two packed groups (the
// warp's 64-slot halves): near2 bit g = group g near.
template <int MODE, bool SYM, bool POT>
__device__ __forceinline__ void run_set2(ISet &S, const float2 e2, const float (&j)[7], int near2,
                                         float4 &b, int self_k) {
    const int m = MODE == 1 ? 3 : (MODE == 2 ? near2 : 0);
    switch (m) {
        case 0: rotate_set<0, SYM, POT>(S, e2, j, b, self_k); break;
        case 1: rotate_set<1, SYM, POT>(S, e2, j, b, self_k); break;
        case 2: rotate_set<2, SYM, POT>(S, e2, j, b, self_k); break;
        default: rotate_set<3, SYM, POT>(S, e2, j, b, self_k); break;
    }
}

}  // namespace symcore
}  // namespace nb
