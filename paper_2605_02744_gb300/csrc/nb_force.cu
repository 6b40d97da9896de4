// All-pairs softened acceleration + potential (Eq. 1, Sec. 2.1; pair kernel of
// App. A, Algorithm 3, without the jerk terms).
//
// FP32-pair kernel ("stream-K"): the iteration space is (i-block, j-tile)
// pairs, i-block = NT*IR particles held in registers, j-tile = TJ particles
// staged in shared memory.  The pairs are laid out i-block-major and cut into
// equal contiguous ranges, one per persistent CTA, so every SM gets the same
// number of pair interactions whatever N is.  A CTA whose range covers an
// i-block only in part writes that block's partial sums to a record in the
// workspace; the last CTA to arrive at a block (arrival counter) folds the
// records in CTA order, so the result does not depend on timing.
//
// j-tiles are streamed through a ST-deep ring of shared-memory stages filled
// by bulk asynchronous copies (cp.async.bulk, one per SoA component) that
// complete on mbarriers -- the GB300 analogue of the read kernel feeding
// circular buffers in Algorithm 1.  The pair loop processes two j-particles
// per packed f32x2 instruction (13 packed FP32 operations and 2 MUFU rsqrt
// per two pairs).
#include <cuda_runtime.h>
#include <stdio.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {

using dev::Acc;
using dev::Record;
using dev::pair2;

// ------------------------------------------------------------------ pack
// FP64 [N][3] positions + [N] masses -> float SoA of 7 arrays of Np:
//   x.hi y.hi z.hi m x.lo y.lo z.lo
// hi = the coordinate rounded to nearest FP32, lo = (x - hi) rounded to
// FP32 (the split "double-single" representation); entries N..Np-1 are
// zero-mass particles at the origin.
__global__ void pack_soa_kernel(const double *__restrict__ pos, const double *__restrict__ mass,
                                int64_t N, int64_t Np, float *__restrict__ soa) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np;
         i += (int64_t)gridDim.x * blockDim.x) {
        float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f}, m = 0.f;
        if (i < N) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double x = pos[3 * i + c];
                hi[c] = __double2float_rn(x);
                lo[c] = __double2float_rn(x - (double)hi[c]);
            }
            m = __double2float_rn(mass[i]);
        }
        store_packed(soa, Np, i, hi, lo, m);
    }
}

int launch_pack(const double *pos, const double *mass, int64_t N, int64_t Np, float *soa,
                cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>(cdiv(Np, threads), 8192);
    pack_soa_kernel<<<(unsigned)blocks, threads, 0, st>>>(pos, mass, N, Np, soa);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// ----------------------------------------------------------- FP32 pairs
struct ForceParams {
    const float *soa;  // [7][Np]: x.hi y.hi z.hi m x.lo y.lo z.lo
    int64_t Np;
    int64_t i0;   // packed index of the first i-particle (row) of this call
    int64_t ni;   // rows: i-slot s is packed particle i0 + s, output row s
    int64_t total;  // nblocks * ntiles
    int32_t nblocks;
    int32_t ntiles;
    float eps2;
    double G;
    double *acc;
    double *pot;
    double *vel;
    double kick;
    Record *records;
    uint32_t *counters;
    uint32_t *status;
    long long timeout;
    int64_t unissued;  // test hook: the ring stage whose copies are never issued (-1: none)
    // adaptive displacement (NF): particles packed in Hilbert order
    const float *tile_box;   // [N/64][8]: lo[3] hi[3] max|x| pad, per 64 j-slots
    const float *block_box;  // [N/(32 IR)][8], per warp's 32 IR i-slots
    const int *perm;         // packed slot -> particle index
    float gamma;             // far iff box gap >= gamma * max|x|
};

// Packed slot of register row k of thread tid in i-block b.  The adaptive
// path (NF) gives each warp 32*IR contiguous slots, so a warp's particles
// share one small box in the Hilbert-sorted pack; otherwise rows are strided
// by the CTA width (coalesced loads and stores).
template <int NT, int IR, bool NF>
__device__ __forceinline__ int64_t slot_of(int64_t b, int k, int tid) {
    if (NF) return b * NT * IR + (int64_t)(tid >> 5) * 32 * IR + k * 32 + (tid & 31);
    return b * NT * IR + k * NT + tid;
}

template <int NT, int IR, int POL, bool GUARD, bool NF>
__device__ __forceinline__ void force_epilogue(const ForceParams &p, int64_t b,
                                               const Acc<POL> (&acc)[IR][4]) {
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        const int64_t slot = slot_of<NT, IR, NF>(b, k, threadIdx.x);
        if (slot < p.ni) {
            const int64_t i = NF ? (int64_t)p.perm[slot] : slot;
            const double phs = acc[k][3].value();
            const double gx = p.G * acc[k][0].value();
            const double gy = p.G * acc[k][1].value();
            const double gz = p.G * acc[k][2].value();
            const double gp = -p.G * phs;
            p.acc[3 * i] = gx;
            p.acc[3 * i + 1] = gy;
            p.acc[3 * i + 2] = gz;
            if (p.pot) p.pot[i] = gp;
            if (p.vel) {
                p.vel[3 * i] += p.kick * gx;
                p.vel[3 * i + 1] += p.kick * gy;
                p.vel[3 * i + 2] += p.kick * gz;
            }
            if (!(isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(gp))) bad = 1;
        }
    }
    if (bad) dev::set_status(p.status, kStatusNonFinite);
}

// Staged j-particles [j0, j1) of one tile against the thread's IR
// i-particles (two j per packed instruction); SPLIT picks the hi/lo
// displacement; SELF masks the pair j == i (kr: the i-particles' offsets
// from the tile base).
template <int IR, int TJ, bool GUARD, bool SPLIT, bool SELF = false>
__device__ __forceinline__ void tile_pairs(const float *sx, const int j0, const int j1,
                                           const float2 eps2,
                                           const float2 (&nx)[IR], const float2 (&ny)[IR],
                                           const float2 (&nz)[IR], const float2 (&nxl)[IR],
                                           const float2 (&nyl)[IR], const float2 (&nzl)[IR],
                                           float2 (&ax)[IR], float2 (&ay)[IR], float2 (&az)[IR],
                                           float2 (&ph)[IR], const int *kr = nullptr) {
    using dev::f2;
    const float *sy = sx + TJ, *sz = sx + 2 * TJ, *sm = sx + 3 * TJ;
    const float *sxl = sx + 4 * TJ, *syl = sx + 5 * TJ, *szl = sx + 6 * TJ;
#pragma unroll 2
    for (int jj = j0; jj < j1; jj += 4) {
        const float4 X = *reinterpret_cast<const float4 *>(sx + jj);
        const float4 Y = *reinterpret_cast<const float4 *>(sy + jj);
        const float4 Z = *reinterpret_cast<const float4 *>(sz + jj);
        const float4 M = *reinterpret_cast<const float4 *>(sm + jj);
        float4 XL = make_float4(0.f, 0.f, 0.f, 0.f), YL = XL, ZL = XL;
        if (SPLIT) {
            XL = *reinterpret_cast<const float4 *>(sxl + jj);
            YL = *reinterpret_cast<const float4 *>(syl + jj);
            ZL = *reinterpret_cast<const float4 *>(szl + jj);
        }
        pair2<IR, GUARD, SPLIT, SELF>(f2(X.x, X.y), f2(Y.x, Y.y), f2(Z.x, Z.y),
                                      f2(XL.x, XL.y), f2(YL.x, YL.y), f2(ZL.x, ZL.y),
                                      f2(M.x, M.y), eps2, nx, ny, nz, nxl, nyl, nzl, ax, ay, az,
                                      ph, kr, jj);
        pair2<IR, GUARD, SPLIT, SELF>(f2(X.z, X.w), f2(Y.z, Y.w), f2(Z.z, Z.w),
                                      f2(XL.z, XL.w), f2(YL.z, YL.w), f2(ZL.z, ZL.w),
                                      f2(M.z, M.w), eps2, nx, ny, nz, nxl, nyl, nzl, ax, ay, az,
                                      ph, kr, jj + 2);
    }
}

// Near test of an (i-block, j-tile) pair of boxes: the gap between the
// boxes is below gamma times the largest coordinate magnitude of either.
__device__ __forceinline__ bool boxes_near(const float *bb, const float *tb, float gamma) {
    float g2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gap = fmaxf(0.f, fmaxf(__ldg(tb + c) - bb[3 + c], bb[c] - __ldg(tb + 3 + c)));
        g2 = fmaf(gap, gap, g2);
    }
    const float X = gamma * fmaxf(bb[6], __ldg(tb + 6));
    return g2 < X * X;
}

template <int NT, int IR, int TJ, int ST, int POL, bool GUARD, bool SPLIT, bool NF>
__global__ void __launch_bounds__(NT) force_sk_kernel(const ForceParams p) {
    using namespace dev;
    constexpr int BI = NT * IR;
    constexpr int NC = SPLIT ? 7 : 4;  // SoA arrays staged per j-tile
    static_assert(TJ % 4 == 0 && (TJ * 4) % 16 == 0, "tile must be 16-byte granular");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + ST * NC * 4 * TJ);
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
        for (int comp = 0; comp < NC; ++comp)
            bulk_g2s(dst + comp * TJ, p.soa + comp * p.Np + jt * TJ, 4 * TJ, &full[s]);
    };
    if (tid == 0) {
        for (int64_t q = 0; q < nq && q < ST; ++q) issue(q);
    }

    float2 nx[IR], ny[IR], nz[IR], nxl[IR], nyl[IR], nzl[IR];
    float bb[8];
    Acc<POL> acc[IR][4];
    const float2 eps2 = f2(p.eps2, p.eps2);
    int64_t b = 0, seg_begin = 0;
    const int64_t first_block = L0 / p.ntiles;

    for (int64_t q = 0; q < nq; ++q) {
        const int64_t t = L0 + q;
        const int64_t jt = t % p.ntiles;
        if (q == 0 || jt == 0) {
            b = t / p.ntiles;
            seg_begin = jt;
            if (NF) {
                const int64_t u = b * (NT / 32) + (tid >> 5);  // this warp's box
#pragma unroll
                for (int e = 0; e < 8; ++e) bb[e] = __ldg(p.block_box + u * 8 + e);
            }
#pragma unroll
            for (int k = 0; k < IR; ++k) {
                const int64_t sl = slot_of<NT, IR, NF>(b, k, tid);
                const bool live = sl < p.ni;  // past the rows: a zero particle
                const int64_t i = p.i0 + (live ? sl : 0);
                const float x = live ? p.soa[i] : 0.f, y = live ? p.soa[p.Np + i] : 0.f,
                            z = live ? p.soa[2 * p.Np + i] : 0.f;
                nx[k] = f2(-x, -x);
                ny[k] = f2(-y, -y);
                nz[k] = f2(-z, -z);
                if (SPLIT) {
                    const float xl = live ? p.soa[4 * p.Np + i] : 0.f,
                                yl = live ? p.soa[5 * p.Np + i] : 0.f,
                                zl = live ? p.soa[6 * p.Np + i] : 0.f;
                    nxl[k] = f2(-xl, -xl);
                    nyl[k] = f2(-yl, -yl);
                    nzl[k] = f2(-zl, -zl);
                } else {
                    nxl[k] = nyl[k] = nzl[k] = f2(0.f, 0.f);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[k][e].zero();
            }
        }
        const int s = (int)(q % ST);
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((q / ST) & 1), p.timeout);
        const float *sx = stages + s * NC * TJ;
        float2 ax[IR], ay[IR], az[IR], ph[IR];
#pragma unroll
        for (int k = 0; k < IR; ++k) ax[k] = ay[k] = az[k] = ph[k] = f2(0.f, 0.f);
        // a tile that holds some of block b's slots has the self pairs: they
        // take the masked loop (exact j != i); every other tile the plain one
        const int64_t r0 = p.i0 + b * BI;  // packed index of the block's first row
        const bool diag = jt * TJ < r0 + BI && (jt + 1) * TJ > r0;
        if (diag) {
            int kr[IR];
#pragma unroll
            for (int k = 0; k < IR; ++k)
                kr[k] = (int)(p.i0 + slot_of<NT, IR, NF>(b, k, tid) - jt * TJ);
            tile_pairs<IR, TJ, GUARD, SPLIT, true>(sx, 0, TJ, eps2, nx, ny, nz, nxl, nyl, nzl, ax,
                                                   ay, az, ph, kr);
        } else if (NF) {
            // per (warp, 64-particle sub-tile): warp-uniform choice
#pragma unroll 1
            for (int c = 0; c < TJ / 64; ++c) {
                const float *tb = p.tile_box + (jt * (TJ / 64) + c) * 8;
                if (boxes_near(bb, tb, p.gamma))
                    tile_pairs<IR, TJ, GUARD, true>(sx, 64 * c, 64 * c + 64, eps2, nx, ny, nz,
                                                    nxl, nyl, nzl, ax, ay, az, ph);
                else
                    tile_pairs<IR, TJ, GUARD, false>(sx, 64 * c, 64 * c + 64, eps2, nx, ny, nz,
                                                     nxl, nyl, nzl, ax, ay, az, ph);
            }
        } else {
            tile_pairs<IR, TJ, GUARD, SPLIT>(sx, 0, TJ, eps2, nx, ny, nz, nxl, nyl, nzl, ax, ay,
                                             az, ph);
        }
#pragma unroll
        for (int k = 0; k < IR; ++k) {
            acc[k][0].add(ax[k].x + ax[k].y);
            acc[k][1].add(ay[k].x + ay[k].y);
            acc[k][2].add(az[k].x + az[k].y);
            acc[k][3].add(ph[k].x + ph[k].y);
        }

        if (__syncthreads_or(!ok)) {
            // A stage never arrived: latch the error, let the copies that are
            // still in flight land (bounded), and leave together.
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
            // end of this CTA's segment of i-block b: tiles [seg_begin, jt]
            if (seg_begin == 0 && jt == p.ntiles - 1) {
                force_epilogue<NT, IR, POL, GUARD, NF>(p, b, acc);
            } else {
                const int slot = (b == first_block) ? 0 : 1;
                Record *rec = p.records + (2 * c + slot) * BI;
#pragma unroll
                for (int k = 0; k < IR; ++k) store_record<POL>(rec + k * NT + tid, acc[k]);
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
                        for (int e = 0; e < 4; ++e) acc[k][e].zero();
                    for (int64_t cc = cf; cc <= cl; ++cc) {
                        const int sl = (b == sk_lo(p.total, C, cc) / p.ntiles) ? 0 : 1;
                        const Record *r = p.records + (2 * cc + sl) * BI;
#pragma unroll
                        for (int k = 0; k < IR; ++k) merge_record<POL>(acc[k], r + k * NT + tid);
                    }
                    force_epilogue<NT, IR, POL, GUARD, NF>(p, b, acc);
                    if (tid == 0) p.counters[b] = 0u;
                }
            }
        }
    }
}

// ------------------------------------------------------------ FP64 pairs
// One i per thread, j-tiles of NT particles staged through shared memory by
// the whole CTA; the pair j == i is skipped by index, and with eps == 0 so
// are coincident pairs.
template <int NT, bool GUARD>
__global__ void __launch_bounds__(NT)
    force_fp64_kernel(const double *__restrict__ pos, const double *__restrict__ mass, int64_t N,
                      int64_t i0, int64_t ni, double eps2, double G, double *acc, double *pot,
                      double *vel, double kick, uint32_t *status) {
    __shared__ double sx[NT], sy[NT], sz[NT], sm[NT];
    const int64_t row = blockIdx.x * (int64_t)NT + threadIdx.x;  // output row
    const int64_t i = i0 + row;                                   // particle
    const bool live = row < ni;
    const double xi = live ? pos[3 * i] : 0.0;
    const double yi = live ? pos[3 * i + 1] : 0.0;
    const double zi = live ? pos[3 * i + 2] : 0.0;
    double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
    for (int64_t j0 = 0; j0 < N; j0 += NT) {
        const int64_t j = j0 + threadIdx.x;
        if (j < N) {
            sx[threadIdx.x] = pos[3 * j];
            sy[threadIdx.x] = pos[3 * j + 1];
            sz[threadIdx.x] = pos[3 * j + 2];
            sm[threadIdx.x] = mass[j];
        }
        __syncthreads();
        const int nj = (int)((N - j0) < NT ? (N - j0) : NT);
        for (int jj = 0; jj < nj; ++jj) {
            if (j0 + jj == i) continue;
            const double dx = sx[jj] - xi, dy = sy[jj] - yi, dz = sz[jj] - zi;
            const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
            if (GUARD && r2 == 0.0) continue;
            const double ri = rsqrt(r2);
            const double s = sm[jj] * ri;
            const double s3 = s * (ri * ri);
            ax = fma(s3, dx, ax);
            ay = fma(s3, dy, ay);
            az = fma(s3, dz, az);
            ph += s;
        }
        __syncthreads();
    }
    if (live) {
        const double gx = G * ax, gy = G * ay, gz = G * az, gp = -G * ph;
        acc[3 * row] = gx;
        acc[3 * row + 1] = gy;
        acc[3 * row + 2] = gz;
        if (pot) pot[row] = gp;
        if (vel) {
            vel[3 * row] += kick * gx;
            vel[3 * row + 1] += kick * gy;
            vel[3 * row + 2] += kick * gz;
        }
        if (!(isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(gp)))
            dev::set_status(status, kStatusNonFinite);
    }
}

// ---------------------------------------------------------- dispatch
// Shapes compiled into this build: (threads, i per thread, tile_j, stages).
#define NB_FORCE_SHAPES(X) \
    X(512, 2, 1024, 2)     \
    X(512, 2, 512, 2)      \
    X(256, 2, 512, 2)      \
    X(256, 2, 256, 3)      \
    X(256, 4, 256, 3)      \
    X(128, 2, 128, 3)      \
    X(128, 1, 64, 2)

bool force_shape_compiled(const Shape &s) {
#define NB_MATCH(NT, IR, TJ, ST) \
    if (s.threads == NT && s.ipt == IR && s.tile_j == TJ && s.stages == ST) return true;
    NB_FORCE_SHAPES(NB_MATCH)
#undef NB_MATCH
    return false;
}

template <int NT, int IR, int TJ, int ST, int POL, bool GUARD, bool SPLIT, bool NF>
static int launch_sk(const ForceParams &p, int cps, cudaStream_t st) {
    auto kern = force_sk_kernel<NT, IR, TJ, ST, POL, GUARD, SPLIT, NF>;
    const size_t smem = (size_t)ST * (SPLIT ? 7 : 4) * 4 * TJ + (size_t)ST * 8;
    // stages above 48 KB need the opt-in (up to 227 KB per CTA)
    if (smem > 48 * 1024) {
        const int rc = smem_optin(reinterpret_cast<const void *>(kern), smem);
        if (rc != NB_OK) return rc;
    }
    static const int occ = occupancy(reinterpret_cast<const void *>(kern), NT, smem);
    const int grid = persistent_grid(cps, occ, p.total);
    kern<<<grid, NT, smem, st>>>(p);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// mode: 0 single positions, 1 split, 2 adaptive (split near, single far;
// never with the eps = 0 guard)
template <int NT, int IR, int TJ, int ST, int POL>
static int launch_sk_gs(const ForceParams &p, bool guard, int mode, int cps, cudaStream_t st) {
    if (guard)
        return mode ? launch_sk<NT, IR, TJ, ST, POL, true, true, false>(p, cps, st)
                    : launch_sk<NT, IR, TJ, ST, POL, true, false, false>(p, cps, st);
    if (mode == 2) return launch_sk<NT, IR, TJ, ST, POL, false, true, true>(p, cps, st);
    return mode ? launch_sk<NT, IR, TJ, ST, POL, false, true, false>(p, cps, st)
                : launch_sk<NT, IR, TJ, ST, POL, false, false, false>(p, cps, st);
}

template <int NT, int IR, int TJ, int ST>
static int launch_sk_pol(const ForceParams &p, int pol, bool guard, int mode, int cps,
                         cudaStream_t st) {
    switch (pol) {
        case NB_PREC_FP32: return launch_sk_gs<NT, IR, TJ, ST, NB_PREC_FP32>(p, guard, mode, cps, st);
        case NB_PREC_KAHAN: return launch_sk_gs<NT, IR, TJ, ST, NB_PREC_KAHAN>(p, guard, mode, cps, st);
        case NB_PREC_F64ACC: return launch_sk_gs<NT, IR, TJ, ST, NB_PREC_F64ACC>(p, guard, mode, cps, st);
    }
    return fail(NB_ERR_UNSUPPORTED, "precision %d has no FP32-pair kernel", pol);
}

int occupancy(const void *kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

int persistent_grid(int cps, int occ, int64_t total) {
    const int64_t per_sm = std::min(cps, occ);
    const int64_t slots = per_sm * device_sm_count();
    return (int)std::max<int64_t>(1, std::min<int64_t>(slots, total));
}

int launch_force(const ForceJob &j) {
    const bool guard = (j.eps == 0.0);
    uint32_t *status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    if (j.precision == NB_PREC_FP64) {
        if (j.sym) {
            if (guard) return fail(NB_ERR_UNSUPPORTED, "symmetric pairs need eps > 0");
            return launch_force_sym(j, false);
        }
        constexpr int NT = 128;
        const int64_t grid = cdiv(j.ni, NT);
        count_launch();
        if (guard)
            force_fp64_kernel<NT, true><<<(unsigned)grid, NT, 0, j.stream>>>(
                j.pos, j.mass, j.N, j.i0, j.ni, 0.0, j.G, j.acc, j.pot, j.vel, j.kick, status);
        else
            force_fp64_kernel<NT, false><<<(unsigned)grid, NT, 0, j.stream>>>(
                j.pos, j.mass, j.N, j.i0, j.ni, j.eps * j.eps, j.G, j.acc, j.pot, j.vel, j.kick,
                status);
        NB_CUDA(cudaGetLastError());
        return NB_OK;
    }
    float *soa = reinterpret_cast<float *>(j.ws + j.L.packA);
    const Shape &sh0 = j.shape;
    const bool adaptive = j.adaptive && !guard;
    char *sb = j.ws + j.L.sortbuf;
    if (j.sym && guard) return fail(NB_ERR_UNSUPPORTED, "symmetric pairs need eps > 0");
    if (adaptive) {
        // boxes per 64 j-slots and per warp of i-slots (direct kernel: 32 IR
        // slots; symmetric FP32 kernel: 256 slots)
        const int tile_unit = 64;
        const int block_unit = j.sym ? 256 : 32 * sh0.ipt;
        int rc = launch_sorted_pack(j.pos, j.mass, j.N, j.L.Np, soa, sort_perm(sb, j.L),
                                    sort_keys(sb), sort_box6(sb, j.L), sort_tile_boxes(sb, j.L),
                                    tile_unit, sort_block_boxes(sb, j.L), block_unit,
                                    j.reuse_order, j.stream);
        if (rc) return rc;
    } else if (!j.packed_ready) {
        int rc = launch_pack(j.pos, j.mass, j.N, j.L.Np, soa, j.stream);
        if (rc) return rc;
    }
    if (j.sym) return launch_force_sym(j, adaptive);
    const Shape &sh = j.shape;
    ForceParams p;
    p.soa = soa;
    p.Np = j.L.Np;
    p.i0 = j.i0;
    p.ni = j.ni;
    p.nblocks = (int32_t)cdiv(j.ni, sh.block_i());
    p.ntiles = (int32_t)cdiv(j.N, sh.tile_j);
    p.total = (int64_t)p.nblocks * p.ntiles;
    const float eps_f = (float)j.eps;
    p.eps2 = eps_f * eps_f;
    p.G = j.G;
    p.acc = j.acc;
    p.pot = j.pot;
    p.vel = j.vel;
    p.kick = j.kick;
    p.records = reinterpret_cast<Record *>(j.ws + j.L.records);
    p.counters = reinterpret_cast<uint32_t *>(j.ws + j.L.counters);
    p.status = status;
    p.timeout = j.timeout;
    p.unissued = j.unissued;
    p.tile_box = adaptive ? sort_tile_boxes(sb, j.L) : nullptr;   // per 64 j-slots
    p.block_box = adaptive ? sort_block_boxes(sb, j.L) : nullptr; // per warp (32 IR i-slots)
    p.perm = adaptive ? sort_perm(sb, j.L) : nullptr;
    p.gamma = j.gamma;
    const int mode = adaptive ? 2 : (j.split ? 1 : 0);
#define NB_DISPATCH(NT, IR, TJ, ST)                                                   \
    if (sh.threads == NT && sh.ipt == IR && sh.tile_j == TJ && sh.stages == ST)      \
        return launch_sk_pol<NT, IR, TJ, ST>(p, j.precision, guard, mode, sh.ctas_per_sm, \
                                             j.stream);
    NB_FORCE_SHAPES(NB_DISPATCH)
#undef NB_DISPATCH
    return fail(NB_ERR_UNSUPPORTED, "force kernel shape (%d,%d,%d,%d) not compiled", sh.threads,
                sh.ipt, sh.tile_j, sh.stages);
}

}  // namespace nb
