// Device-side building blocks: mbarrier + bulk-copy (TMA) staging with
// bounded waits, the FP32 reciprocal square root, packed f32x2 arithmetic
// and the per-particle accumulation policies.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nb_internal.h"

namespace nb {
namespace dev {

// ------------------------------------------------------------ mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One potentially blocking test of phase `parity`: the thread may be
// suspended until the phase completes, for at most about `hint_ns`
// nanoseconds (the suspend-time hint of mbarrier.try_wait).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

// Waits for phase `parity` of `bar` to complete, for at most `timeout`
// SM clock cycles.  Returns false if the limit ran out.  Each try_wait may
// suspend the thread; its hint is a quarter of the limit (in ns at ~2 GHz,
// at most 1 ms), so a short limit is not outlived by one suspended test.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long timeout) {
    const long long q = timeout / 8;
    const uint32_t hint = (uint32_t)(q < 1 ? 1 : (q > 1000000 ? 1000000 : q));
    if (mbar_try_wait(bar, parity, hint)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity, hint)) {
        if (clock64() - t0 > timeout) return false;
    }
    return true;
}

// Bulk (non-tensor) global -> shared copy completing on `bar`.  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bits) {
    atomicOr(status, bits);
}

// ------------------------------------------------------------- arithmetic
// Hardware approximate reciprocal square root (PTX rsqrt.approx.ftz.f32):
// one MUFU operation.  Inputs here are >= eps^2 > 0 or, in the guarded
// kernels, exactly 0 (handled by the caller).
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ------------------------------------------------------------ pair loop
// Two j-particles (packed in the .x/.y halves) against IR i-particles.
// The displacement is (x_j.hi - x_i.hi) + (x_j.lo - x_i.lo) when SPLIT.
// SELF (tiles that hold some of the i-particles): kr[k] is i-particle k's
// offset from the tile base and jj the offset of the .x j-particle; the
// pair j == i gets a zero mass, so Eq. 1's j != i holds exactly.
template <int IR, bool GUARD, bool SPLIT, bool SELF = false>
__device__ __forceinline__ void pair2(const float2 xj, const float2 yj, const float2 zj,
                                      const float2 xl, const float2 yl, const float2 zl,
                                      const float2 mj, const float2 eps2, const float2 (&nx)[IR],
                                      const float2 (&ny)[IR], const float2 (&nz)[IR],
                                      const float2 (&nxl)[IR], const float2 (&nyl)[IR],
                                      const float2 (&nzl)[IR], float2 (&ax)[IR],
                                      float2 (&ay)[IR], float2 (&az)[IR], float2 (&ph)[IR],
                                      const int *kr = nullptr, int jj = 0) {
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        float2 dx = add2(xj, nx[k]);
        float2 dy = add2(yj, ny[k]);
        float2 dz = add2(zj, nz[k]);
        if (SPLIT) {
            dx = add2(dx, add2(xl, nxl[k]));
            dy = add2(dy, add2(yl, nyl[k]));
            dz = add2(dz, add2(zl, nzl[k]));
        }
        float2 r2 = fma2(dx, dx, eps2);
        r2 = fma2(dy, dy, r2);
        r2 = fma2(dz, dz, r2);
        float2 ri = f2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        if (GUARD) {
            ri.x = r2.x > 0.f ? ri.x : 0.f;
            ri.y = r2.y > 0.f ? ri.y : 0.f;
        }
        float2 m = mj;
        if (SELF) {
            m.x = kr[k] == jj ? 0.f : m.x;
            m.y = kr[k] == jj + 1 ? 0.f : m.y;
        }
        const float2 s = mul2(m, ri);
        const float2 ri2 = mul2(ri, ri);
        const float2 s3 = mul2(s, ri2);
        ax[k] = fma2(s3, dx, ax[k]);
        ay[k] = fma2(s3, dy, ay[k]);
        az[k] = fma2(s3, dz, az[k]);
        ph[k] = add2(ph[k], s);
    }
}

// --------------------------------------------------- accumulation policies
// Per-particle running sums across j-tiles.  Each tile's FP32 partial is
// folded in once per tile.
template <int POL>
struct Acc;

template <>
struct Acc<NB_PREC_FP32> {
    float s;
    __device__ __forceinline__ void zero() { s = 0.f; }
    __device__ __forceinline__ void add(float x) { s += x; }
    __device__ __forceinline__ double value() const { return (double)s; }
};

template <>
struct Acc<NB_PREC_KAHAN> {
    float s, c;  // true sum ~= s - c
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <>
struct Acc<NB_PREC_F64ACC> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(float x) { s += (double)x; }
    __device__ __forceinline__ double value() const { return s; }
};

// 32-byte partial record of the four sums (ax, ay, az, phi) of one particle.
struct alignas(16) Record {
    union {
        double d[4];
        float f[8];
    };
};

template <int POL>
__device__ __forceinline__ void store_record(Record *r, const Acc<POL> (&a)[4]);

template <>
__device__ __forceinline__ void store_record<NB_PREC_FP32>(Record *r,
                                                           const Acc<NB_PREC_FP32> (&a)[4]) {
    float4 v = make_float4(a[0].s, a[1].s, a[2].s, a[3].s);
    reinterpret_cast<float4 *>(r)[0] = v;
}
template <>
__device__ __forceinline__ void store_record<NB_PREC_KAHAN>(Record *r,
                                                            const Acc<NB_PREC_KAHAN> (&a)[4]) {
    reinterpret_cast<float4 *>(r)[0] = make_float4(a[0].s, a[1].s, a[2].s, a[3].s);
    reinterpret_cast<float4 *>(r)[1] = make_float4(a[0].c, a[1].c, a[2].c, a[3].c);
}
template <>
__device__ __forceinline__ void store_record<NB_PREC_F64ACC>(Record *r,
                                                             const Acc<NB_PREC_F64ACC> (&a)[4]) {
    reinterpret_cast<double2 *>(r)[0] = make_double2(a[0].s, a[1].s);
    reinterpret_cast<double2 *>(r)[1] = make_double2(a[2].s, a[3].s);
}

// Folds a record written by another CTA (read through L2) into `a`, in the
// policy's own arithmetic: the Kahan sums take the record's s and then -c.
template <int POL>
__device__ __forceinline__ void merge_record(Acc<POL> (&a)[4], const Record *r);

template <>
__device__ __forceinline__ void merge_record<NB_PREC_FP32>(Acc<NB_PREC_FP32> (&a)[4],
                                                           const Record *r) {
    const float4 s = __ldcg(reinterpret_cast<const float4 *>(r));
    a[0].add(s.x); a[1].add(s.y); a[2].add(s.z); a[3].add(s.w);
}
template <>
__device__ __forceinline__ void merge_record<NB_PREC_KAHAN>(Acc<NB_PREC_KAHAN> (&a)[4],
                                                            const Record *r) {
    const float4 s = __ldcg(reinterpret_cast<const float4 *>(r));
    const float4 c = __ldcg(reinterpret_cast<const float4 *>(r) + 1);
    a[0].add(s.x); a[1].add(s.y); a[2].add(s.z); a[3].add(s.w);
    a[0].add(-c.x); a[1].add(-c.y); a[2].add(-c.z); a[3].add(-c.w);
}
template <>
__device__ __forceinline__ void merge_record<NB_PREC_F64ACC>(Acc<NB_PREC_F64ACC> (&a)[4],
                                                             const Record *r) {
    const double2 p = __ldcg(reinterpret_cast<const double2 *>(r));
    const double2 q = __ldcg(reinterpret_cast<const double2 *>(r) + 1);
    a[0].s += p.x; a[1].s += p.y; a[2].s += q.x; a[3].s += q.y;
}

}  // namespace dev
}  // namespace nb
