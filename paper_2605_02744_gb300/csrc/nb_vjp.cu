// Vector-Jacobian product of the softened acceleration and potential
// (derived from Eq. 1, Sec. 2.1) with respect to positions and masses, in
// gather form (one output particle k per register slot, j streamed, no
// atomics).  With d = x_j - x_k, s^2 = |d|^2 + eps^2, r = 1/s and the
// cotangent c_j of a_j (and pbar_j of phi_j):
//
//   xbar_k = G sum_j [ r^3 (m_k c_j - m_j c_k) - 3 r^5 (d.(m_k c_j - m_j c_k)) d
//                      - r^3 (m_k pbar_j + m_j pbar_k) d ]
//   mbar_k = -G sum_j [ r^3 (c_j . d) + r pbar_j ]
//
// The pair loop keeps eight FP32 running sums per k (nine with pbar),
//   A = sum r^3 c_j,  B = sum r^3 m_j,  C = sum q d,  M = sum r^3 (c_j . d),
//   q = -r^5 (m_k (d.c_j) - m_j (d.c_k)) - r^3 (m_k pbar_j + m_j pbar_k)/3,
//   P = sum r pbar_j / 3,
// so xbar_k = G (m_k A - B c_k + 3 C) and mbar_k = -G (M + 3 P).  The pair
// j == k is skipped by index (its r^3 = 1/eps^3 terms would otherwise swamp
// A and B before cancelling).  With FUSED
// it also accumulates the force at the same positions (a = G sum m_j r^3 d,
// phi = -G sum m_j r) for the time-reversed reconstruction of the trajectory.
// The per-tile sums are folded into FP64 totals once per j-tile.  Work split,
// bulk-copy staging and fixup follow the force kernel (stream-K).
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {

using dev::Acc;

constexpr int kVjpSums = 13;  // A(3) B C(3) M P  a(3) phi

struct VjpParams {
    const float *soa;   // [7][Np] positions (split) and masses
    const float *csoa;  // [4][Np] cx cy cz pbar/3 (FP32)
    int64_t Np;
    int64_t N;
    int64_t i0, ni;       // output rows [i0, i0 + ni) of the N particles
    int64_t total;
    int32_t nblocks;
    int32_t ntiles;
    float eps2;
    double G;
    const double *mass;   // FP64 masses (epilogue)
    const double *cdbl;   // [4][Np] FP64 cotangents c, pbar (epilogue)
    double *pos_bar;      // [ni][3], row r is particle i0 + r
    double *mass_bar;     // [ni]
    int accumulate;
    double *acc_out;      // FUSED
    double *vhalf;
    double *pos_rw;
    double rewind_kick;
    double rewind_drift;
    double *records;      // [2*grid][BI][16] doubles
    uint32_t *counters;
    uint32_t *status;
    long long timeout;
    int64_t unissued;  // test hook: the ring stage whose copies are never issued (-1: none)
};

// -------------------------------------------------------- cotangent pack
// Step form: vbar += drift * xbar; c = coef * vbar.  Direct form:
// c = coef * abar, pbar scaled the same way.
// Writes FP32 SoA (cx, cy, cz, pbar/3) and the FP64 copy used by the
// epilogue and by the FP64-pair kernel.
__global__ void pack_cotangent_kernel(const double *__restrict__ abar,
                                      const double *__restrict__ pbar, double *vbar,
                                      const double *__restrict__ xbar, double drift, double coef,
                                      int step_form, int64_t N, int64_t Np, float *csoa,
                                      double *cdbl) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np;
         i += (int64_t)gridDim.x * blockDim.x) {
        double c[3] = {0.0, 0.0, 0.0}, pb = 0.0;
        if (i < N) {
            if (step_form) {
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const double v = vbar[3 * i + e] + drift * xbar[3 * i + e];
                    vbar[3 * i + e] = v;
                    c[e] = coef * v;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 3; ++e) c[e] = coef * abar[3 * i + e];
                if (pbar) pb = coef * pbar[i];
            }
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            csoa[e * Np + i] = __double2float_rn(c[e]);
            if (cdbl) cdbl[e * Np + i] = c[e];
        }
        csoa[3 * Np + i] = __double2float_rn(pb / 3.0);
        if (cdbl) cdbl[3 * Np + i] = pb;
    }
}

// ------------------------------------------------------------ pair math
// Two j-particles (halves .x/.y, tile offsets jj and jj+1) against IR
// output particles.  kr[k] is k's offset from the tile base: the pair j == k
// is skipped by index, so the large self terms never enter a sum.  The
// per-k constants arrive negated (nmk = -m_k, npbk = -pbar_k/3), which makes
// the running sums C and q carry the opposite sign (x_bar uses +3C).
template <int IR, bool GUARD, bool PB, bool FUSED, bool SPLIT>
__device__ __forceinline__ void vjp_pair2(
    const int jj, const int (&kr)[IR], const float2 xj, const float2 yj, const float2 zj,
    const float2 xl, const float2 yl, const float2 zl, const float2 mj, const float2 cxj,
    const float2 cyj, const float2 czj, const float2 pbj, const float2 eps2,
    const float2 (&nx)[IR], const float2 (&ny)[IR], const float2 (&nz)[IR],
    const float2 (&nxl)[IR], const float2 (&nyl)[IR], const float2 (&nzl)[IR],
    const float2 (&nmk)[IR], const float2 (&cxk)[IR], const float2 (&cyk)[IR],
    const float2 (&czk)[IR], const float2 (&npbk)[IR], float2 (&S)[IR][kVjpSums]) {
    using namespace dev;
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
        float2 r = f2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        if (GUARD) {
            r.x = r2.x > 0.f ? r.x : 0.f;
            r.y = r2.y > 0.f ? r.y : 0.f;
        }
        r.x = (kr[k] == jj) ? 0.f : r.x;
        r.y = (kr[k] == jj + 1) ? 0.f : r.y;
        const float2 rr = mul2(r, r);
        const float2 r3 = mul2(rr, r);
        const float2 r5 = mul2(r3, rr);
        float2 dcj = mul2(dx, cxj);
        dcj = fma2(dy, cyj, dcj);
        dcj = fma2(dz, czj, dcj);
        float2 dck = mul2(dx, cxk[k]);
        dck = fma2(dy, cyk[k], dck);
        dck = fma2(dz, czk[k], dck);
        // -dw = m_j (d.c_k) - m_k (d.c_j)
        const float2 ndw = fma2(nmk[k], dcj, mul2(mj, dck));
        float2 nq = mul2(r5, ndw);
        if (PB) {
            // -(m_k pbar_j + m_j pbar_k)/3
            const float2 ne3 = fma2(nmk[k], pbj, mul2(mj, npbk[k]));
            nq = fma2(r3, ne3, nq);
            S[k][8] = fma2(pbj, r, S[k][8]);
        }
        S[k][0] = fma2(r3, cxj, S[k][0]);
        S[k][1] = fma2(r3, cyj, S[k][1]);
        S[k][2] = fma2(r3, czj, S[k][2]);
        if (FUSED) {
            const float2 mr3 = mul2(mj, r3);
            S[k][3] = add2(S[k][3], mr3);
            S[k][9] = fma2(mr3, dx, S[k][9]);
            S[k][10] = fma2(mr3, dy, S[k][10]);
            S[k][11] = fma2(mr3, dz, S[k][11]);
            S[k][12] = fma2(mj, r, S[k][12]);
        } else {
            S[k][3] = fma2(r3, mj, S[k][3]);
        }
        S[k][4] = fma2(nq, dx, S[k][4]);
        S[k][5] = fma2(nq, dy, S[k][5]);
        S[k][6] = fma2(nq, dz, S[k][6]);
        S[k][7] = fma2(r3, dcj, S[k][7]);
    }
}

template <bool PB, bool FUSED>
__device__ __forceinline__ constexpr bool vjp_sum_live(int e) {
    return e < 8 || (e == 8 && PB) || (e >= 9 && FUSED);
}

// The FP64 totals of a thread's output rows live in shared memory,
// [kVjpSums][IR][NT] (added to once per j-tile; in registers they took 52
// of the thread's registers and held the kernel at 2 CTAs per SM).
template <int NT, int IR>
__device__ __forceinline__ double &tot_at(double *T, int k, int e) {
    return T[(e * IR + k) * NT + threadIdx.x];
}

template <int NT, int IR, bool PB, bool FUSED>
__device__ __forceinline__ void vjp_epilogue(const VjpParams &p, int64_t b, double *T) {
    constexpr int BI = NT * IR;
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        const int64_t r = b * BI + k * NT + threadIdx.x;  // output row
        if (r >= p.ni) continue;
        const int64_t i = p.i0 + r;
        double v[kVjpSums];
#pragma unroll
        for (int e = 0; e < kVjpSums; ++e) v[e] = vjp_sum_live<PB, FUSED>(e) ? tot_at<NT, IR>(T, k, e) : 0.0;
        const double mk = p.mass[i];
        const double cx = p.cdbl[i], cy = p.cdbl[p.Np + i], cz = p.cdbl[2 * p.Np + i];
        const double gx = p.G * (mk * v[0] - v[3] * cx + 3.0 * v[4]);
        const double gy = p.G * (mk * v[1] - v[3] * cy + 3.0 * v[5]);
        const double gz = p.G * (mk * v[2] - v[3] * cz + 3.0 * v[6]);
        const double gm = -p.G * (v[7] + (PB ? 3.0 * v[8] : 0.0));
        if (p.accumulate) {
            p.pos_bar[3 * r] += gx;
            p.pos_bar[3 * r + 1] += gy;
            p.pos_bar[3 * r + 2] += gz;
            p.mass_bar[r] += gm;
        } else {
            p.pos_bar[3 * r] = gx;
            p.pos_bar[3 * r + 1] = gy;
            p.pos_bar[3 * r + 2] = gz;
            p.mass_bar[r] = gm;
        }
        if (!(isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(gm))) bad = 1;
        if (FUSED) {
            const double a[3] = {p.G * v[9], p.G * v[10], p.G * v[11]};
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                p.acc_out[3 * i + e] = a[e];
                const double vh = p.vhalf[3 * i + e] - p.rewind_kick * a[e];
                p.vhalf[3 * i + e] = vh;
                p.pos_rw[3 * i + e] -= p.rewind_drift * vh;
            }
            if (!(isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]))) bad = 1;
        }
    }
    if (bad) dev::set_status(p.status, kStatusNonFinite);
}

template <int NT, int IR, int TJ, int ST, bool GUARD, bool PB, bool FUSED, bool SPLIT>
__global__ void __launch_bounds__(NT) vjp_sk_kernel(const VjpParams p) {
    using namespace dev;
    constexpr int BI = NT * IR;
    constexpr int NC = 11;  // 7 position/mass arrays + 4 cotangent arrays
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + ST * NC * 4 * TJ);
    double *T = reinterpret_cast<double *>(smem_raw + ST * NC * 4 * TJ + ST * 8);
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int64_t C = gridDim.x, c = blockIdx.x;
    const int64_t L0 = sk_lo(p.total, C, c);
    const int64_t nq = sk_lo(p.total, C, c + 1) - L0;
    if (nq <= 0) return;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int64_t q) {
        if (q == p.unissued) return;  // the wait on this stage runs out
        const int s = (int)(q % ST);
        const int64_t jt = (L0 + q) % p.ntiles;
        float *dst = stages + s * NC * TJ;
        mbar_arrive_expect_tx(&full[s], NC * 4 * TJ);
#pragma unroll
        for (int comp = 0; comp < 7; ++comp)
            bulk_g2s(dst + comp * TJ, p.soa + comp * p.Np + jt * TJ, 4 * TJ, &full[s]);
#pragma unroll
        for (int comp = 0; comp < 4; ++comp)
            bulk_g2s(dst + (7 + comp) * TJ, p.csoa + comp * p.Np + jt * TJ, 4 * TJ, &full[s]);
    };
    if (tid == 0) {
        for (int64_t q = 0; q < nq && q < ST; ++q) issue(q);
    }

    float2 nx[IR], ny[IR], nz[IR], nxl[IR], nyl[IR], nzl[IR], nmk[IR], cxk[IR], cyk[IR],
        czk[IR], npbk[IR];
    int kidx[IR];
    const float2 eps2 = f2(p.eps2, p.eps2);
    int64_t b = 0, seg_begin = 0;
    const int64_t first_block = L0 / p.ntiles;

    for (int64_t q = 0; q < nq; ++q) {
        const int64_t t = L0 + q;
        const int64_t jt = t % p.ntiles;
        if (q == 0 || jt == 0) {
            b = t / p.ntiles;
            seg_begin = jt;
#pragma unroll
            for (int k = 0; k < IR; ++k) {
                // rows past the range load particle i0 (their sums are never stored)
                const int64_t r = b * BI + k * NT + tid;
                const int64_t i = p.i0 + (r < p.ni ? r : 0);
                const float x = p.soa[i], y = p.soa[p.Np + i], z = p.soa[2 * p.Np + i];
                const float xl = p.soa[4 * p.Np + i], yl = p.soa[5 * p.Np + i],
                            zl = p.soa[6 * p.Np + i];
                const float m = p.soa[3 * p.Np + i];
                const float cx = p.csoa[i], cy = p.csoa[p.Np + i], cz = p.csoa[2 * p.Np + i];
                const float pb = p.csoa[3 * p.Np + i];
                kidx[k] = (int)i;
                nx[k] = f2(-x, -x);
                ny[k] = f2(-y, -y);
                nz[k] = f2(-z, -z);
                nxl[k] = f2(-xl, -xl);
                nyl[k] = f2(-yl, -yl);
                nzl[k] = f2(-zl, -zl);
                nmk[k] = f2(-m, -m);
                cxk[k] = f2(cx, cx);
                cyk[k] = f2(cy, cy);
                czk[k] = f2(cz, cz);
                npbk[k] = f2(-pb, -pb);
#pragma unroll
                for (int e = 0; e < kVjpSums; ++e) tot_at<NT, IR>(T, k, e) = 0.0;
            }
        }
        const int s = (int)(q % ST);
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((q / ST) & 1), p.timeout);
        const float *st = stages + s * NC * TJ;
        int kr[IR];
#pragma unroll
        for (int k = 0; k < IR; ++k) kr[k] = kidx[k] - (int)(jt * TJ);

        float2 S[IR][kVjpSums];
#pragma unroll
        for (int k = 0; k < IR; ++k)
#pragma unroll
            for (int e = 0; e < kVjpSums; ++e) S[k][e] = f2(0.f, 0.f);
#pragma unroll 1
        for (int jj = 0; jj < TJ; jj += 4) {
            float4 V[NC];
#pragma unroll
            for (int comp = 0; comp < NC; ++comp)
                V[comp] = *reinterpret_cast<const float4 *>(st + comp * TJ + jj);
            vjp_pair2<IR, GUARD, PB, FUSED, SPLIT>(
                jj, kr, f2(V[0].x, V[0].y), f2(V[1].x, V[1].y), f2(V[2].x, V[2].y), f2(V[4].x, V[4].y),
                f2(V[5].x, V[5].y), f2(V[6].x, V[6].y), f2(V[3].x, V[3].y), f2(V[7].x, V[7].y),
                f2(V[8].x, V[8].y), f2(V[9].x, V[9].y), f2(V[10].x, V[10].y), eps2, nx, ny, nz,
                nxl, nyl, nzl, nmk, cxk, cyk, czk, npbk, S);
            vjp_pair2<IR, GUARD, PB, FUSED, SPLIT>(
                jj + 2, kr, f2(V[0].z, V[0].w), f2(V[1].z, V[1].w), f2(V[2].z, V[2].w), f2(V[4].z, V[4].w),
                f2(V[5].z, V[5].w), f2(V[6].z, V[6].w), f2(V[3].z, V[3].w), f2(V[7].z, V[7].w),
                f2(V[8].z, V[8].w), f2(V[9].z, V[9].w), f2(V[10].z, V[10].w), eps2, nx, ny, nz,
                nxl, nyl, nzl, nmk, cxk, cyk, czk, npbk, S);
        }
#pragma unroll
        for (int k = 0; k < IR; ++k)
#pragma unroll
            for (int e = 0; e < kVjpSums; ++e)
                if (vjp_sum_live<PB, FUSED>(e))
                    tot_at<NT, IR>(T, k, e) += (double)(S[k][e].x + S[k][e].y);

        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                set_status(p.status, kStatusTimeout);
                // copies still in flight must land before the CTA exits: at least
                // the default bound, however short the caller's limit
                const long long drain = p.timeout > kDefaultTimeoutCycles ? p.timeout
                                                                       : kDefaultTimeoutCycles;
                for (int64_t r = q; r < nq && r < q + ST; ++r)
                    if (r != p.unissued)
                        mbar_wait_bounded(&full[r % ST], (uint32_t)((r / ST) & 1), drain);
            }
            __syncthreads();
            return;
        }
        if (tid == 0 && q + ST < nq) {
            fence_proxy_async();
            issue(q + ST);
        }

        if (jt == p.ntiles - 1 || q == nq - 1) {
            if (seg_begin == 0 && jt == p.ntiles - 1) {
                vjp_epilogue<NT, IR, PB, FUSED>(p, b, T);
            } else {
                const int slot = (b == first_block) ? 0 : 1;
                double *rec = p.records + ((2 * c + slot) * BI) * 16;
#pragma unroll
                for (int k = 0; k < IR; ++k)
#pragma unroll
                    for (int e = 0; e < kVjpSums; ++e)
                        if (vjp_sum_live<PB, FUSED>(e))
                            rec[(k * NT + tid) * 16 + e] = tot_at<NT, IR>(T, k, e);
                __threadfence();
                __syncthreads();
                const int64_t cf = sk_owner(p.total, C, b * p.ntiles);
                const int64_t cl = sk_owner(p.total, C, b * p.ntiles + p.ntiles - 1);
                if (tid == 0) {
                    const uint32_t prev = atomicAdd(&p.counters[b], 1u);
                    s_last = (prev == (uint32_t)(cl - cf));
                }
                __syncthreads();
                if (s_last) {
                    __threadfence();
#pragma unroll
                    for (int k = 0; k < IR; ++k)
#pragma unroll
                        for (int e = 0; e < kVjpSums; ++e) tot_at<NT, IR>(T, k, e) = 0.0;
                    for (int64_t cc = cf; cc <= cl; ++cc) {
                        const int sl = (b == sk_lo(p.total, C, cc) / p.ntiles) ? 0 : 1;
                        const double *r = p.records + ((2 * cc + sl) * BI) * 16;
#pragma unroll
                        for (int k = 0; k < IR; ++k)
#pragma unroll
                            for (int e = 0; e < kVjpSums; ++e)
                                if (vjp_sum_live<PB, FUSED>(e))
                                    tot_at<NT, IR>(T, k, e) += __ldcg(r + (k * NT + tid) * 16 + e);
                    }
                    vjp_epilogue<NT, IR, PB, FUSED>(p, b, T);
                    if (tid == 0) p.counters[b] = 0u;
                }
            }
        }
    }
}

// ------------------------------------------------------------ FP64 pairs
// One k per thread; cotangents from the FP64 copy; the self pair is skipped
// by index and, with eps == 0, so are coincident pairs.
template <int NT, bool GUARD>
__global__ void __launch_bounds__(NT)
    vjp_fp64_kernel(const double *__restrict__ pos, const double *__restrict__ mass,
                    const double *__restrict__ cdbl, int has_pb, int64_t N, int64_t Np,
                    int64_t i0, int64_t ni, double eps2, double G, double *pos_bar,
                    double *mass_bar, int accumulate,
                    double *acc_out, double *vhalf, double *pos_rw, double rk, double rd,
                    uint32_t *status) {
    __shared__ double sx[NT], sy[NT], sz[NT], sm[NT], scx[NT], scy[NT], scz[NT], spb[NT];
    const int64_t row = blockIdx.x * (int64_t)NT + threadIdx.x;  // output row
    const bool live = row < ni;
    const int64_t k = i0 + (live ? row : 0);
    double xk = 0, yk = 0, zk = 0, mk = 0, cxk = 0, cyk = 0, czk = 0, pbk = 0;
    if (live) {
        xk = pos[3 * k]; yk = pos[3 * k + 1]; zk = pos[3 * k + 2]; mk = mass[k];
        cxk = cdbl[k]; cyk = cdbl[Np + k]; czk = cdbl[2 * Np + k]; pbk = cdbl[3 * Np + k];
    }
    double gx = 0, gy = 0, gz = 0, gm = 0, ax = 0, ay = 0, az = 0;
    for (int64_t j0 = 0; j0 < N; j0 += NT) {
        const int64_t j = j0 + threadIdx.x;
        if (j < N) {
            sx[threadIdx.x] = pos[3 * j];
            sy[threadIdx.x] = pos[3 * j + 1];
            sz[threadIdx.x] = pos[3 * j + 2];
            sm[threadIdx.x] = mass[j];
            scx[threadIdx.x] = cdbl[j];
            scy[threadIdx.x] = cdbl[Np + j];
            scz[threadIdx.x] = cdbl[2 * Np + j];
            spb[threadIdx.x] = cdbl[3 * Np + j];
        }
        __syncthreads();
        const int nj = (int)((N - j0) < NT ? (N - j0) : NT);
        for (int jj = 0; jj < nj; ++jj) {
            if (j0 + jj == k) continue;
            const double dx = sx[jj] - xk, dy = sy[jj] - yk, dz = sz[jj] - zk;
            const double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
            if (GUARD && s2 == 0.0) continue;
            const double r = rsqrt(s2);
            const double r3 = r * r * r;
            const double r5 = r3 * r * r;
            const double mj = sm[jj];
            const double wx = mk * scx[jj] - mj * cxk;
            const double wy = mk * scy[jj] - mj * cyk;
            const double wz = mk * scz[jj] - mj * czk;
            const double dw = dx * wx + dy * wy + dz * wz;
            double coef = -3.0 * r5 * dw;
            if (has_pb) coef -= r3 * (mk * spb[jj] + mj * pbk);
            gx += r3 * wx + coef * dx;
            gy += r3 * wy + coef * dy;
            gz += r3 * wz + coef * dz;
            gm -= r3 * (scx[jj] * dx + scy[jj] * dy + scz[jj] * dz);
            if (has_pb) gm -= r * spb[jj];
            ax += mj * r3 * dx;
            ay += mj * r3 * dy;
            az += mj * r3 * dz;
        }
        __syncthreads();
    }
    if (!live) return;
    gx *= G; gy *= G; gz *= G; gm *= G;
    if (accumulate) {
        pos_bar[3 * row] += gx; pos_bar[3 * row + 1] += gy; pos_bar[3 * row + 2] += gz;
        mass_bar[row] += gm;
    } else {
        pos_bar[3 * row] = gx; pos_bar[3 * row + 1] = gy; pos_bar[3 * row + 2] = gz;
        mass_bar[row] = gm;
    }
    bool bad = !(isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(gm));
    if (acc_out) {
        const double a[3] = {G * ax, G * ay, G * az};
        for (int e = 0; e < 3; ++e) {
            acc_out[3 * k + e] = a[e];
            const double vh = vhalf[3 * k + e] - rk * a[e];
            vhalf[3 * k + e] = vh;
            pos_rw[3 * k + e] -= rd * vh;
        }
        bad = bad || !(isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]));
    }
    if (bad) dev::set_status(status, kStatusNonFinite);
}

// ---------------------------------------------------------- dispatch
#define NB_VJP_SHAPES(X) \
    X(128, 2, 128, 3)    \
    X(256, 2, 128, 3)    \
    X(256, 1, 128, 3)    \
    X(128, 1, 64, 2)

bool vjp_shape_compiled(const Shape &s) {
#define NB_MATCH(NT, IR, TJ, ST) \
    if (s.threads == NT && s.ipt == IR && s.tile_j == TJ && s.stages == ST) return true;
    NB_VJP_SHAPES(NB_MATCH)
#undef NB_MATCH
    return false;
}

template <int NT, int IR, int TJ, int ST, bool GUARD, bool PB, bool FUSED, bool SPLIT>
static int launch_vjp_sk(const VjpParams &p, int cps, cudaStream_t st) {
    auto kern = vjp_sk_kernel<NT, IR, TJ, ST, GUARD, PB, FUSED, SPLIT>;
    const size_t smem = (size_t)ST * 11 * 4 * TJ + (size_t)ST * 8 +
                        (size_t)kVjpSums * IR * NT * sizeof(double);
    static const int occ = occupancy(reinterpret_cast<const void *>(kern), NT, smem);
    const int grid = persistent_grid(cps, occ, p.total);
    kern<<<grid, NT, smem, st>>>(p);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int NT, int IR, int TJ, int ST, bool SPLIT>
static int launch_vjp_variant2(const VjpParams &p, bool guard, bool pb, bool fused, int cps,
                               cudaStream_t st) {
    if (fused && pb) return fail(NB_ERR_UNSUPPORTED, "fused force with pot_bar is not built");
    if (guard) {
        if (fused) return launch_vjp_sk<NT, IR, TJ, ST, true, false, true, SPLIT>(p, cps, st);
        return pb ? launch_vjp_sk<NT, IR, TJ, ST, true, true, false, SPLIT>(p, cps, st)
                  : launch_vjp_sk<NT, IR, TJ, ST, true, false, false, SPLIT>(p, cps, st);
    }
    if (fused) return launch_vjp_sk<NT, IR, TJ, ST, false, false, true, SPLIT>(p, cps, st);
    return pb ? launch_vjp_sk<NT, IR, TJ, ST, false, true, false, SPLIT>(p, cps, st)
              : launch_vjp_sk<NT, IR, TJ, ST, false, false, false, SPLIT>(p, cps, st);
}

template <int NT, int IR, int TJ, int ST>
static int launch_vjp_variant(const VjpParams &p, bool guard, bool pb, bool fused, bool split,
                              int cps, cudaStream_t st) {
    return split ? launch_vjp_variant2<NT, IR, TJ, ST, true>(p, guard, pb, fused, cps, st)
                 : launch_vjp_variant2<NT, IR, TJ, ST, false>(p, guard, pb, fused, cps, st);
}

int launch_vjp(const VjpJob &j) {
    const bool guard = (j.eps == 0.0);
    const bool fused = j.acc_out != nullptr;
    const bool pb = !j.step_form && j.pot_bar != nullptr;
    uint32_t *status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    float *csoa = reinterpret_cast<float *>(j.ws + j.L.packB);
    double *cdbl = reinterpret_cast<double *>(j.ws + j.L.cot64);
    {
        const int threads = 256;
        const int64_t blocks = std::min<int64_t>(cdiv(j.L.Np, threads), 8192);
        pack_cotangent_kernel<<<(unsigned)blocks, threads, 0, j.stream>>>(
            j.acc_bar, j.pot_bar, j.vel_bar, j.pos_bar, j.drift_dt, j.kick_coef,
            j.step_form ? 1 : 0, j.N, j.L.Np, csoa, cdbl);
        count_launch();
        NB_CUDA(cudaGetLastError());
    }
    if (j.precision == NB_PREC_FP64) {
        constexpr int NT = 128;
        const int64_t grid = cdiv(j.ni, NT);
        const double eps2 = j.eps * j.eps;
        auto k = guard ? vjp_fp64_kernel<NT, true> : vjp_fp64_kernel<NT, false>;
        k<<<(unsigned)grid, NT, 0, j.stream>>>(j.pos, j.mass, cdbl, pb ? 1 : 0, j.N, j.L.Np,
                                               j.i0, j.ni, eps2,
                                               j.G, j.pos_bar, j.mass_bar, j.accumulate ? 1 : 0,
                                               j.acc_out, j.vhalf, j.pos_rw, j.rewind_kick,
                                               j.rewind_drift, status);
        count_launch();
        NB_CUDA(cudaGetLastError());
        return NB_OK;
    }
    float *soa = reinterpret_cast<float *>(j.ws + j.L.packA);
    int rc = launch_pack(j.pos, j.mass, j.N, j.L.Np, soa, j.stream);
    if (rc) return rc;
    const Shape &sh = j.shape;
    VjpParams p;
    p.soa = soa;
    p.csoa = csoa;
    p.Np = j.L.Np;
    p.N = j.N;
    p.i0 = j.i0;
    p.ni = j.ni;
    p.nblocks = (int32_t)cdiv(j.ni, sh.block_i());
    p.ntiles = (int32_t)cdiv(j.N, sh.tile_j);
    p.total = (int64_t)p.nblocks * p.ntiles;
    const float eps_f = (float)j.eps;
    p.eps2 = eps_f * eps_f;
    p.G = j.G;
    p.mass = j.mass;
    p.cdbl = cdbl;
    p.pos_bar = j.pos_bar;
    p.mass_bar = j.mass_bar;
    p.accumulate = j.accumulate ? 1 : 0;
    p.acc_out = j.acc_out;
    p.vhalf = j.vhalf;
    p.pos_rw = j.pos_rw;
    p.rewind_kick = j.rewind_kick;
    p.rewind_drift = j.rewind_drift;
    p.records = reinterpret_cast<double *>(j.ws + j.L.records);
    p.counters = reinterpret_cast<uint32_t *>(j.ws + j.L.counters);
    p.status = status;
    p.timeout = j.timeout;
    p.unissued = j.unissued;
#define NB_DISPATCH(NT, IR, TJ, ST)                                              \
    if (sh.threads == NT && sh.ipt == IR && sh.tile_j == TJ && sh.stages == ST) \
        return launch_vjp_variant<NT, IR, TJ, ST>(p, guard, pb, fused, j.split, sh.ctas_per_sm, \
                                                  j.stream);
    NB_VJP_SHAPES(NB_DISPATCH)
#undef NB_DISPATCH
    return fail(NB_ERR_UNSUPPORTED, "VJP kernel shape (%d,%d,%d,%d) not compiled", sh.threads,
                sh.ipt, sh.tile_j, sh.stages);
}

}  // namespace nb
