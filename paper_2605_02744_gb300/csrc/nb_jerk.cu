// Acceleration + jerk + potential: the paper's own pair kernel (App. A,
// Algorithm 3), and the fourth-order Hermite predict / evaluate / correct
// cycle around it (Sec. 2.1's scheme, at fourth order).
//
// For d = x_j - x_i, w = v_j - v_i, r = (|d|^2 + eps^2)^(-1/2):
//   a_i    += m_j r^3 d
//   jerk_i += m_j r^3 w - 3 m_j r^5 (d . w) d
//   phi_i  -= m_j r
// i.e. t = m_j r^3 (Algorithm 3's t_j with weight G m_j applied at the end),
// q = -3 r^2 (d . w) and jerk += t (w + q d).
//
// One i-block (threads x IR particles) per CTA, grid-strided over blocks;
// j-tiles of 10 SoA arrays (split positions, mass, velocity) staged by bulk
// copies into an mbarrier ring as in the force kernel; two j per packed
// f32x2 instruction (34 packed FP32 operations + 2 MUFU per two pairs).  The
// epilogue either stores (a, jerk, phi) or applies the Hermite corrector.
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {

using dev::Acc;
using dev::f2;

constexpr int kJerkArrays = 10;  // x.hi y.hi z.hi m x.lo y.lo z.lo vx vy vz

struct JerkParams {
    const float *soa;  // [10][Np]
    int64_t Np;
    int64_t N;
    int32_t nblocks;
    int32_t ntiles;
    float eps2;
    double G;
    // outputs / Hermite state
    double *pos;
    double *vel;
    double *acc;
    double *jerk;
    double *pot;
    double h;       // corrector step; 0 = store a, jerk, phi only
    uint32_t *status;
    long long timeout;
    int64_t unissued;  // test hook: the ring stage whose copies are never issued (-1: none)
};

// Prediction (h > 0) or the current state (h == 0), packed for the kernel:
//   xp = x + v h + a h^2/2 + j h^3/6,  vp = v + a h + j h^2/2
__global__ void hermite_predict_pack_kernel(const double *__restrict__ pos,
                                            const double *__restrict__ vel,
                                            const double *__restrict__ acc,
                                            const double *__restrict__ jerk,
                                            const double *__restrict__ mass, int64_t N, int64_t Np,
                                            double h, float *__restrict__ soa) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np;
         i += (int64_t)gridDim.x * blockDim.x) {
        float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f}, vf[3] = {0.f, 0.f, 0.f}, m = 0.f;
        if (i < N) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double x = pos[3 * i + c], v = vel[3 * i + c];
                if (h != 0.0) {
                    const double a = acc[3 * i + c], j = jerk[3 * i + c];
                    x = x + v * h + a * h * h / 2.0 + j * h * h * h / 6.0;
                    v = v + a * h + j * h * h / 2.0;
                }
                hi[c] = __double2float_rn(x);
                lo[c] = __double2float_rn(x - (double)hi[c]);
                vf[c] = __double2float_rn(v);
            }
            m = __double2float_rn(mass[i]);
        }
        store_packed(soa, Np, i, hi, lo, m);
        soa[7 * Np + i] = vf[0];
        soa[8 * Np + i] = vf[1];
        soa[9 * Np + i] = vf[2];
    }
}

// SELF (a tile that holds some of the i-particles): kr[k] is i-particle k's
// offset from the tile base; the pair j == i gets a zero mass (exact j != i).
template <int IR, bool GUARD, bool SELF = false>
__device__ __forceinline__ void jerk_pair2(const float *st, int jj, int TJ, const float2 eps2,
                                           const float2 (&nx)[IR], const float2 (&ny)[IR],
                                           const float2 (&nz)[IR], const float2 (&nxl)[IR],
                                           const float2 (&nyl)[IR], const float2 (&nzl)[IR],
                                           const float2 (&nvx)[IR], const float2 (&nvy)[IR],
                                           const float2 (&nvz)[IR], float2 (&S)[IR][7],
                                           const int *kr = nullptr) {
    using namespace dev;
    const float2 xj = *reinterpret_cast<const float2 *>(st + jj);
    const float2 yj = *reinterpret_cast<const float2 *>(st + TJ + jj);
    const float2 zj = *reinterpret_cast<const float2 *>(st + 2 * TJ + jj);
    const float2 mj = *reinterpret_cast<const float2 *>(st + 3 * TJ + jj);
    const float2 xl = *reinterpret_cast<const float2 *>(st + 4 * TJ + jj);
    const float2 yl = *reinterpret_cast<const float2 *>(st + 5 * TJ + jj);
    const float2 zl = *reinterpret_cast<const float2 *>(st + 6 * TJ + jj);
    const float2 vx = *reinterpret_cast<const float2 *>(st + 7 * TJ + jj);
    const float2 vy = *reinterpret_cast<const float2 *>(st + 8 * TJ + jj);
    const float2 vz = *reinterpret_cast<const float2 *>(st + 9 * TJ + jj);
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        const float2 dx = add2(add2(xj, nx[k]), add2(xl, nxl[k]));
        const float2 dy = add2(add2(yj, ny[k]), add2(yl, nyl[k]));
        const float2 dz = add2(add2(zj, nz[k]), add2(zl, nzl[k]));
        const float2 wx = add2(vx, nvx[k]);
        const float2 wy = add2(vy, nvy[k]);
        const float2 wz = add2(vz, nvz[k]);
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
        const float2 t = mul2(s, ri2);  // m r^3
        float2 dw = mul2(dx, wx);
        dw = fma2(dy, wy, dw);
        dw = fma2(dz, wz, dw);
        // t q = -3 m r^5 (d.w)
        const float2 tq = mul2(mul2(t, f2(-3.f, -3.f)), mul2(dw, ri2));
        S[k][0] = fma2(t, dx, S[k][0]);
        S[k][1] = fma2(t, dy, S[k][1]);
        S[k][2] = fma2(t, dz, S[k][2]);
        S[k][3] = fma2(tq, dx, fma2(t, wx, S[k][3]));
        S[k][4] = fma2(tq, dy, fma2(t, wy, S[k][4]));
        S[k][5] = fma2(tq, dz, fma2(t, wz, S[k][5]));
        S[k][6] = add2(S[k][6], s);
    }
}

template <int NT, int IR, int TJ, int ST, int POL, bool GUARD>
__global__ void __launch_bounds__(NT) jerk_kernel(const JerkParams p) {
    using namespace dev;
    constexpr int BI = NT * IR;
    constexpr int NC = kJerkArrays;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + ST * NC * 4 * TJ);
    const int tid = threadIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // all tiles of all this CTA's blocks form one stream q = 0 .. nq-1
    const int64_t nmine = (p.nblocks - (int64_t)blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int64_t nq = nmine * p.ntiles;
    if (nq <= 0) return;
    auto issue = [&](int64_t q) {
        if (q == p.unissued) return;  // the wait on this stage runs out
        const int s = (int)(q % ST);
        const int64_t jt = q % p.ntiles;
        float *dst = stages + s * NC * TJ;
        mbar_arrive_expect_tx(&full[s], NC * 4 * TJ);
#pragma unroll
        for (int comp = 0; comp < NC; ++comp)
            bulk_g2s(dst + comp * TJ, p.soa + comp * p.Np + jt * TJ, 4 * TJ, &full[s]);
    };
    if (tid == 0)
        for (int64_t q = 0; q < nq && q < ST; ++q) issue(q);

    float2 nx[IR], ny[IR], nz[IR], nxl[IR], nyl[IR], nzl[IR], nvx[IR], nvy[IR], nvz[IR];
    Acc<POL> T[IR][7];
    const float2 eps2 = f2(p.eps2, p.eps2);
    for (int64_t q = 0; q < nq; ++q) {
        const int64_t jt = q % p.ntiles;
        const int64_t b = blockIdx.x + (q / p.ntiles) * gridDim.x;
        if (jt == 0) {
#pragma unroll
            for (int k = 0; k < IR; ++k) {
                const int64_t i = b * BI + k * NT + tid;
                float v[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) v[c] = p.soa[c * p.Np + i];
                nx[k] = f2(-v[0], -v[0]);
                ny[k] = f2(-v[1], -v[1]);
                nz[k] = f2(-v[2], -v[2]);
                nxl[k] = f2(-v[4], -v[4]);
                nyl[k] = f2(-v[5], -v[5]);
                nzl[k] = f2(-v[6], -v[6]);
                nvx[k] = f2(-v[7], -v[7]);
                nvy[k] = f2(-v[8], -v[8]);
                nvz[k] = f2(-v[9], -v[9]);
#pragma unroll
                for (int e = 0; e < 7; ++e) T[k][e].zero();
            }
        }
        const int s = (int)(q % ST);
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((q / ST) & 1), p.timeout);
        const float *st = stages + s * NC * TJ;
        float2 S[IR][7];
#pragma unroll
        for (int k = 0; k < IR; ++k)
#pragma unroll
            for (int e = 0; e < 7; ++e) S[k][e] = f2(0.f, 0.f);
        if (jt * TJ < (b + 1) * BI && (jt + 1) * TJ > b * BI) {
            // the tile holds some of block b's particles: mask the self pairs
            int kr[IR];
#pragma unroll
            for (int k = 0; k < IR; ++k) kr[k] = (int)(b * BI + k * NT + tid - jt * TJ);
#pragma unroll 2
            for (int jj = 0; jj < TJ; jj += 2)
                jerk_pair2<IR, GUARD, true>(st, jj, TJ, eps2, nx, ny, nz, nxl, nyl, nzl, nvx, nvy,
                                            nvz, S, kr);
        } else {
#pragma unroll 2
            for (int jj = 0; jj < TJ; jj += 2)
                jerk_pair2<IR, GUARD>(st, jj, TJ, eps2, nx, ny, nz, nxl, nyl, nzl, nvx, nvy, nvz,
                                      S);
        }
#pragma unroll
        for (int k = 0; k < IR; ++k)
#pragma unroll
            for (int e = 0; e < 7; ++e) T[k][e].add(S[k][e].x + S[k][e].y);
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
        if (jt == p.ntiles - 1) {
            uint32_t bad = 0;
#pragma unroll
            for (int k = 0; k < IR; ++k) {
                const int64_t i = b * BI + k * NT + tid;
                if (i >= p.N) continue;
                const double phs = T[k][6].value();
                double a1[3], j1[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a1[c] = p.G * T[k][c].value();
                    j1[c] = p.G * T[k][3 + c].value();
                }
                if (p.pot) p.pot[i] = -p.G * phs;
                const double h = p.h;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (h != 0.0) {
                        const double x0 = p.pos[3 * i + c], v0 = p.vel[3 * i + c];
                        const double a0 = p.acc[3 * i + c], j0 = p.jerk[3 * i + c];
                        const double v1 = v0 + (a0 + a1[c]) * h / 2.0 + (j0 - j1[c]) * h * h / 12.0;
                        p.pos[3 * i + c] = x0 + (v0 + v1) * h / 2.0 + (a0 - a1[c]) * h * h / 12.0;
                        p.vel[3 * i + c] = v1;
                    }
                    p.acc[3 * i + c] = a1[c];
                    p.jerk[3 * i + c] = j1[c];
                    if (!isfinite(a1[c]) || !isfinite(j1[c])) bad = 1;
                }
            }
            if (bad) set_status(p.status, kStatusNonFinite);
        }
    }
}

template <int POL, bool GUARD>
static int launch_jerk_kernel(const JerkParams &p, cudaStream_t st) {
    constexpr int NT = 128, IR = 2, TJ = 128, ST = 3;
    auto kern = jerk_kernel<NT, IR, TJ, ST, POL, GUARD>;
    const size_t smem = (size_t)ST * kJerkArrays * 4 * TJ + (size_t)ST * 8;
    static const int occ = occupancy(reinterpret_cast<const void *>(kern), NT, smem);
    int64_t grid = (int64_t)occ * device_sm_count();
    if (grid > p.nblocks) grid = p.nblocks;
    kern<<<(unsigned)grid, NT, smem, st>>>(p);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

int launch_jerk(const JerkJob &j) {
    if (j.precision == NB_PREC_FP64)
        return fail(NB_ERR_UNSUPPORTED, "the jerk kernel computes FP32 pairs (FP32, KAHAN, F64ACC)");
    constexpr int NT = 128, IR = 2, TJ = 128;
    float *soa = reinterpret_cast<float *>(j.ws + j.L.packA);
    JerkParams p;
    p.soa = soa;
    p.Np = j.L.Np;
    p.N = j.N;
    p.nblocks = (int32_t)cdiv(j.N, NT * IR);
    p.ntiles = (int32_t)cdiv(j.N, TJ);
    const float ef = (float)j.eps;
    p.eps2 = ef * ef;
    p.G = j.G;
    p.pos = j.pos;
    p.vel = j.vel;
    p.acc = j.acc;
    p.jerk = j.jerk;
    p.pot = j.pot;
    p.status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    p.timeout = j.timeout;
    p.unissued = j.unissued;
    const bool guard = j.eps == 0.0;
    const int threads = 256;
    const int64_t pblocks = std::min<int64_t>(cdiv(j.L.Np, threads), 8192);
    // nsteps == 0: one evaluation at the current state (h = 0 stores a,
    // jerk, phi); otherwise nsteps predict / evaluate+correct cycles
    for (int64_t n = 0; n < (j.nsteps > 0 ? j.nsteps : 1); ++n) {
        const double h = j.nsteps > 0 ? j.h : 0.0;
        hermite_predict_pack_kernel<<<(unsigned)pblocks, threads, 0, j.stream>>>(
            j.pos, j.vel, j.acc, j.jerk, j.mass, j.N, j.L.Np, h, soa);
        count_launch();
        NB_CUDA(cudaGetLastError());
        p.h = h;
        int rc;
        switch (j.precision * 2 + (guard ? 1 : 0)) {
            case NB_PREC_FP32 * 2: rc = launch_jerk_kernel<NB_PREC_FP32, false>(p, j.stream); break;
            case NB_PREC_FP32 * 2 + 1: rc = launch_jerk_kernel<NB_PREC_FP32, true>(p, j.stream); break;
            case NB_PREC_KAHAN * 2: rc = launch_jerk_kernel<NB_PREC_KAHAN, false>(p, j.stream); break;
            case NB_PREC_KAHAN * 2 + 1: rc = launch_jerk_kernel<NB_PREC_KAHAN, true>(p, j.stream); break;
            case NB_PREC_F64ACC * 2: rc = launch_jerk_kernel<NB_PREC_F64ACC, false>(p, j.stream); break;
            default: rc = launch_jerk_kernel<NB_PREC_F64ACC, true>(p, j.stream); break;
        }
        if (rc) return rc;
    }
    return NB_OK;
}

}  // namespace nb
