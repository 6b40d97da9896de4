// Symmetric-pair force evaluation (Eq. 1 with Newton's third law).
//
// The pair term of Eq. 1 is antisymmetric up to the masses: with
// d = x_j - x_i and r^-3 = (|d|^2 + eps^2)^-3/2,
//     a_i += m_j r^-3 d,   a_j -= m_i r^-3 d,
//     phi_i += m_j r^-1,   phi_j += m_i r^-1,
// so one evaluation of d, r^2, r^-1 and r^-3 serves both particles.  Per
// unordered pair that is 18 FP32 operations (single-float displacement) in
// place of 2 x 13, about 9 per directed interaction.
//
// Decomposition.  The (padded) slots are cut into row blocks of 2048; the
// work items are the block pairs (I, J) with J >= I, in row-major order,
// cut into units of 2 j-sets and split over one persistent CTA per SM into
// contiguous ranges of equal estimated cost (stream-K: a range may start or
// end inside an item).  The estimate counts FP32 operations per (warp,
// j-set) from the same near/far box tests the pair kernel makes; three small
// kernels compute it, scan it and cut the ranges.
// A CTA of 8 warps keeps block I in registers: warp w holds the 256 slots
// I*2048 + w*256 + [0, 256), lane l the eight slots  + 32k + l  (k = 0..7),
// each pre-broadcast as an (x, x) pair.  A j-set is 64 slots of block J;
// lane l loads two of them, j-slots l and 32 + l, into the .x / .y halves
// of packed f32x2 registers, so every FP32 operation of the pair term is a
// packed one (one rotation step: 8 i-slots x 2 j = 16 pairs, 148 packed
// FP32 instructions, 16 MUFU rsqrt, 16 shuffles).  The set rotates through
// the lanes with shuffles: at step s lane l holds j-slots (l + s) mod 32 and
// 32 + (l + s) mod 32, so in 32 steps every lane meets every j once, and the
// j-particles' own sums (a_j, phi_j) travel with them and come home to lane
// l.  Each step's eight j-side terms go into fresh registers and then into
// the travelling sums with one add, so a strong close pair's term meets
// ~47 later FP32 roundings within an item, not ~260.
//
//   * Off-diagonal items (I < J): both halves of every pair.  The 8 warps'
//     j-side sums of 2 j-sets are added in warp order in shared memory (one
//     barrier per 2 j-sets), giving the FP32 partial of the J-block
//     particles from block I.
//   * Diagonal items (I = J): the i-side only, over all ordered pairs of
//     the block; the self pairs (j-set 4w + h at rotation step 0: i-slot 2h
//     against the .x j, 2h + 1 against the .y j) get a zero mass, so Eq. 1's
//     j != i holds exactly.
//
// The i-side FP32 register sums, kept per j-stream (.x, .y), are folded into
// the accumulation policy (FP32, Kahan or FP64; totals kept in shared
// memory) every 4 j-sets (128 terms per stream and particle; for F64ACC
// through an FP32 middle sum in shared memory that goes into FP64 every 8
// j-sets, FP64 adds being slow on this part) over the CTA's segment of a
// row.  In Hilbert order a particle's strongest, mutually cancelling terms
// (its spatial neighbours) arrive together; with 512-term FP32 chains the
// running sums of central particles of a log-normal Plummer sphere
// (N = 300001, eps = 1e-3) lost up to 1e-5 of |a|, with 128-term chains they
// stay at the 2e-6 of the unsorted order.  (Flushing every 2 j-sets was
// measured 0.8 % slower at 2^20 for 2.08e-6 -> 1.94e-6 worst error.)
//
// Combining across CTAs.  Every particle's sum collects one j-side FP32
// partial per block above it and one i-side total per CTA that worked on its
// row.  Both go, as they are produced, into two-word fixed-point
// accumulators (nb_fixed.cuh) with integer atomic adds: exact and
// independent of arrival order, so results are bitwise reproducible, and the
// scratch is O(N) (64 B per particle) -- not a partial per block pair.  A
// one-block kernel picks the fixed-point exponent from the a-priori bound
// N max|m| max(0.385 / eps^2, 1 / eps) on every partial and total (the
// largest value of |d| (|d|^2 + eps^2)^-3/2 is 0.385 / eps^2 at
// |d| = eps / sqrt 2).  The fold kernel reads each particle's accumulators
// once (and zeroes them for the next call), applies G, scatters through the
// Hilbert permutation and optionally kicks the velocity.
//
// Displacements: single floats, hi/lo pairs (x_j.hi - x_i.hi) +
// (x_j.lo - x_i.lo), or adaptive: per (warp i-set, j-set) the hi/lo form
// only when the bounding boxes are closer than gamma * max|x| (a 32-bit
// mask per warp and item, from the Hilbert-sorted pack's boxes of 256 i-
// and 64 j-slots).
//
// FP64 pairs (force_sym64_kernel) keep the first form of this kernel: 16
// warps of 128 slots (4 per lane, doubles), 32-slot j-sets of one particle
// per lane, scalar j-side sums.
#include <cuda_runtime.h>

#include <stdlib.h>

#include <algorithm>
#include <cmath>

#include "nb_device.cuh"
#include "nb_fixed.cuh"
#include "nb_internal.h"
#include "nb_sym_core.cuh"
#include "nb_symj.cuh"

namespace nb {

using dev::Acc;
using dev::add2;
using dev::f2;
using dev::fma2;
using dev::mul2;
using dev::rsqrt_approx;

namespace {

using namespace symcore;
using namespace symj;

#define NB_TRY_SYM(...)                \
    do {                               \
        const int rc_ = (__VA_ARGS__); \
        if (rc_ != NB_OK) return rc_;  \
    } while (0)

constexpr int BI = 2048;            // slots per row block
static_assert(BI == kSymBlock, "row block size");
constexpr int CPS = 1;              // resident CTAs per SM
constexpr int US = 16;              // stream-K units per item (both kernels)
// FP32 pairs (force_sym_kernel)
constexpr int NW = 8;               // warps per CTA
constexpr int NT = NW * 32;         // threads per CTA
constexpr int IRP = 8;              // i-slots per lane
constexpr int WS = 32 * IRP;        // i-slots per warp
constexpr int JSP = 64;             // slots per j-set (two per lane)
constexpr int NJSP = BI / JSP;      // j-sets per block: one 32-bit near mask
constexpr int KBP = 2;              // j-sets per cross-warp reduction (128 slots)
constexpr int FLP = 4;              // j-sets per i-side flush (128 terms per j-stream)
constexpr int FL2P = 16;            // F64ACC: j-sets per FP64 add of the FP32 middle sums
                                    // (1024 pair terms; 8 j-sets: 341.4 ms at 2^20, 16: 334.5)
static_assert(NW * WS == BI && NJSP == 32 && NJSP / KBP == US, "FP32 kernel shape");
constexpr size_t kRedBytes = 2 * KBP * 2 * NW * 32 * sizeof(float4);
// FP64 pairs (force_sym64_kernel)
constexpr int SW = 16;              // warps per CTA
constexpr int SNT = SW * 32;        // threads per CTA
constexpr int NJS = BI / JS;        // 32-slot j-sets per block
constexpr int KB = 4;               // j-sets per cross-warp reduction
static_assert(SW * 32 * IR == BI && NJS / KB == US, "FP64 kernel shape");

struct SymParams {
    const float *soa;   // packed SoA [7][Np]
    int64_t Np;
    int64_t nb;         // row blocks
    int64_t T;          // items nb (nb + 1) / 2
    int64_t U;          // stream-K units T * US (KB j-sets of one item each)
    int64_t ctas;       // grid size of the pair kernel
    float eps2;
    float gamma;        // adaptive threshold; the mode decides whether it is used
    const float *jbox;  // per 32 slots: lo[3], hi[3], max|x|, pad
    const float *wbox;  // per 128 slots
    unsigned long long *acc_fx;  // [4 components][2 words][Np] fixed-point totals
    const int *fx_exp;           // the call's fixed-point exponent F
    const int64_t *lo;  // [ctas + 1]: CTA c owns units [lo[c], lo[c + 1])
    uint32_t *status;
};

// FP64 pairs: the common layout plus positions [N][3] and masses in
// particle order.
struct SymParams64 : SymParams {
    const double *pos64, *mass64;
    int64_t N;
    double eps2_64;
};

__host__ __device__ inline int64_t row_start(int64_t I, int64_t nb) {
    return I * nb - I * (I - 1) / 2;
}

// Adds v to component e of slot s's fixed-point total.
__device__ __forceinline__ void add_fixed(const SymParams &p, int e, int64_t s, double v, int F) {
    unsigned long long *w = p.acc_fx + (int64_t)(2 * e) * p.Np + s;
    if (!fx::add(w, w + p.Np, v, F)) dev::set_status(p.status, kStatusNonFinite);
}
__device__ __forceinline__ void add_fixed(const SymParams &p, int e, int64_t s, float v, int F) {
    unsigned long long *w = p.acc_fx + (int64_t)(2 * e) * p.Np + s;
    if (!fx::add_f32(w, w + p.Np, v, F)) dev::set_status(p.status, kStatusNonFinite);
}

// ------------------------------------------------------------- FP32 pairs
__device__ __forceinline__ void load_jp(const SymParams &p, int64_t s, float (&j)[14]) {
    symj::load_pair(p.soa, p.Np, s, j);
}

// MODE: 0 single-float displacement, 1 hi/lo, 2 adaptive.  POT: the
// potential sums too (the caller wants phi).  The i-slots' lo parts stay in
// registers for MODE 1 (every j-set is near) and come from shared memory
// for MODE 2 (only near j-sets use them; 245 of 255 registers are taken).
template <int POL, int MODE, bool POT>
__global__ void __launch_bounds__(NT, CPS) force_sym_kernel(const SymParams p) {
    constexpr int NWJ = NW, IRJ = IRP, SNTJ = NT;
    constexpr bool LOSM = MODE == 2;
    constexpr int HW = IRJ / 2;  // j-sets per warp i-set
    constexpr size_t kRedBytesJ = kRedBytes;
    extern __shared__ __align__(16) unsigned char smemj[];
    float4 *red = reinterpret_cast<float4 *>(smemj);  // [2][KBP][2 halves][NWJ][32]
    Acc<POL> *tot = reinterpret_cast<Acc<POL> *>(smemj + kRedBytesJ);  // [IRJ * 4][SNTJ]
    constexpr bool MID = POL == NB_PREC_F64ACC;
    float *mid = reinterpret_cast<float *>(smemj + kRedBytesJ + 4 * IRJ * SNTJ * sizeof(Acc<POL>));
    // LOSM: (-x.lo, -x.lo) pairs [3][IRJ][SNTJ] after the F64ACC middle sums
    float2 *lo2 = reinterpret_cast<float2 *>(smemj + kRedBytesJ +
                                             4 * IRJ * SNTJ * sizeof(Acc<POL>) +
                                             (MID ? 4 * IRJ * SNTJ * sizeof(float) : 0)) +
                  threadIdx.x;
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int64_t c = blockIdx.x;
    int64_t u = __ldg(p.lo + c);
    const int64_t u_end = __ldg(p.lo + c + 1);
    if (u >= u_end) return;
    const int F = __ldg(p.fx_exp);
    const int64_t t0 = u / US;
    int64_t I = 0;
    while (row_start(I + 1, p.nb) <= t0) ++I;
    int64_t J = I + (t0 - row_start(I, p.nb));
    const float2 e2 = f2(p.eps2, p.eps2);
    ISetJ<IRJ> S;
    int half = 0;
    bool row_open = false;
    while (u < u_end) {
        const int qa = (int)(u % US) * KBP;
        const int64_t item_end = (u / US + 1) * US;
        const int64_t seg_end = item_end < u_end ? item_end : u_end;
        const int qb = qa + (int)(seg_end - u) * KBP;
        const int64_t ib = I * BI + w * (32 * IRJ);  // this warp's i-set
        if (!row_open) {
#pragma unroll
            for (int k = 0; k < IRJ; ++k) {
                const int64_t sl = ib + 32 * k + l;
                const float x = __ldg(p.soa + sl), y = __ldg(p.soa + p.Np + sl),
                            z = __ldg(p.soa + 2 * p.Np + sl), m = __ldg(p.soa + 3 * p.Np + sl);
                S.nx[k] = f2(-x, -x);
                S.ny[k] = f2(-y, -y);
                S.nz[k] = f2(-z, -z);
                S.m[k] = f2(m, m);
                const float xl = __ldg(p.soa + 4 * p.Np + sl), yl = __ldg(p.soa + 5 * p.Np + sl),
                            zl = __ldg(p.soa + 6 * p.Np + sl);
                if (LOSM) {
                    if (MODE != 0) {
                        lo2[(0 * IRJ + k) * SNTJ] = f2(-xl, -xl);
                        lo2[(1 * IRJ + k) * SNTJ] = f2(-yl, -yl);
                        lo2[(2 * IRJ + k) * SNTJ] = f2(-zl, -zl);
                    }
                } else {
                    S.nxl[k] = -xl;
                    S.nyl[k] = -yl;
                    S.nzl[k] = -zl;
                }
                S.ax[k] = S.ay[k] = S.az[k] = S.ph[k] = f2(0.f, 0.f);
            }
#pragma unroll
            for (int v = 0; v < 4 * IRJ; ++v) {
                tot[v * SNTJ + tid].zero();
                if (MID) mid[v * SNTJ + tid] = 0.f;
            }
            row_open = true;
        }
        const bool sym = J != I;
        const int64_t jb = J * BI;
        unsigned near = 0u;
        if (MODE == 2) {
            float wb[7], tb[7];
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                wb[a] = __ldg(p.wbox + (ib / (32 * IRJ)) * 8 + a);
                tb[a] = __ldg(p.jbox + (jb / JSP + l) * 8 + a);
            }
            near = __ballot_sync(0xffffffffu, boxes_near(wb, tb, p.gamma));
        }
        float jn[14];
        load_jp(p, jb + qa * JSP + l, jn);
        for (int q = qa; q < qb; ++q) {
            float jc[14];
#pragma unroll
            for (int a = 0; a < 14; ++a) jc[a] = jn[a];
            if (q + 1 < qb) load_jp(p, jb + (q + 1) * JSP + l, jn);
            const bool nq = (near >> q) & 1u;
            float4 b0, b1;
            if (sym) {
                run_setj<IRJ, MODE, true, POT, LOSM>(S, e2, jc, nq, b0, b1, -1, lo2, SNTJ);
                float4 *r = red + (((half * KBP + (q % KBP)) * 2) * NWJ + w) * 32 + l;
                r[0] = b0;
                r[NWJ * 32] = b1;
            } else {
                // the warp's own slots are j-sets HW w .. HW w + HW - 1 of the block
                run_setj<IRJ, MODE, false, POT, LOSM>(S, e2, jc, nq, b0, b1,
                                                  q / HW == w ? q % HW : -1, lo2, SNTJ);
            }
            if ((q + 1) % FLP == 0 || q + 1 == qb) {
#pragma unroll
                for (int k = 0; k < IRJ; ++k) {
                    const float2 v4[4] = {S.ax[k], S.ay[k], S.az[k], S.ph[k]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int v = (k * 4 + e) * SNTJ + tid;
                        const float val = v4[e].x + v4[e].y;
                        if (MID)
                            mid[v] += val;
                        else
                            tot[v].add(val);
                    }
                    S.ax[k] = S.ay[k] = S.az[k] = S.ph[k] = f2(0.f, 0.f);
                }
                if (MID && ((q + 1) % FL2P == 0 || q + 1 == qb)) {
#pragma unroll
                    for (int v = 0; v < 4 * IRJ; ++v) {
                        tot[v * SNTJ + tid].add(mid[v * SNTJ + tid]);
                        mid[v * SNTJ + tid] = 0.f;
                    }
                }
            }
            if (sym && (q + 1) % KBP == 0) {
                __syncthreads();
                for (int v = tid; v < KBP * JSP * 4; v += SNTJ) {
                    const int e = v & 3, js = (v >> 2) & (JSP - 1), qq = v >> 8;
                    const float *r = reinterpret_cast<const float *>(
                                         red + (((half * KBP + qq) * 2 + (js >> 5)) * NWJ) * 32 +
                                         (js & 31)) + e;
                    float sum = 0.f;
#pragma unroll
                    for (int w2 = 0; w2 < NWJ; ++w2) sum += r[w2 * 32 * 4];
                    if (POT || e < 3)
                        add_fixed(p, e, jb + (q + 1 - KBP + qq) * JSP + js, e < 3 ? -sum : sum, F);
                }
                half ^= 1;
            }
        }
        u = seg_end;
        if ((J == p.nb - 1 && qb == NJSP) || u == u_end) {
#pragma unroll
            for (int k = 0; k < IRJ; ++k) {
                const int64_t slot = ib + 32 * k + l;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (POT || e < 3) add_fixed(p, e, slot, tot[(k * 4 + e) * SNTJ + tid].value(), F);
            }
            row_open = false;
        }
        if (qb == NJSP && ++J == p.nb) {
            ++I;
            J = I;
        }
    }
}

// Reads and zeroes every slot's fixed-point totals (padding slots too: they
// collect j-side sums as zero-mass test particles); for real particles,
// applies G, writes acc / pot through the permutation (NULL = identity) and
// optionally kicks the velocity.
__global__ void __launch_bounds__(256) sym_fold_kernel(const SymParams p, int64_t N,
                                                       const int *__restrict__ perm, double G,
                                                       double *__restrict__ acc,
                                                       double *__restrict__ pot,
                                                       double *__restrict__ vel, double kick) {
    const int F = __ldg(p.fx_exp);
    uint32_t bad = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < p.Np;
         s += (int64_t)gridDim.x * blockDim.x) {
        double a[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            unsigned long long *wd = p.acc_fx + (int64_t)(2 * e) * p.Np + s;
            const unsigned long long hi = __ldcs(wd), lo = __ldcs(wd + p.Np);
            if (hi) wd[0] = 0ull;
            if (lo) wd[p.Np] = 0ull;
            a[e] = fx::value(hi, lo, F);
        }
        if (s >= N) continue;
        const double ax = G * a[0], ay = G * a[1], az = G * a[2];
        const double gp = -G * a[3];
        const int64_t i = perm ? (int64_t)perm[s] : s;
        acc[3 * i] = ax;
        acc[3 * i + 1] = ay;
        acc[3 * i + 2] = az;
        if (vel) {
            vel[3 * i] += kick * ax;
            vel[3 * i + 1] += kick * ay;
            vel[3 * i + 2] += kick * az;
        }
        if (pot) pot[i] = gp;
        if (!(isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(gp))) bad = 1;
    }
    if (bad) dev::set_status(p.status, kStatusNonFinite);
}

// The call's fixed-point exponent from the bound N max|m| max(0.385 / eps^2,
// 1 / eps) (x 1.02 for the rounding of FP32 partial sums) on every partial
// and total.  Every block takes the maximum of its share of the masses
// (independent loads, four per thread in flight) and folds it into one word
// with an integer atomicMax on the bits (non-negative doubles order like
// their bit patterns, so the maximum is exact and F reproducible); the last
// block to finish (arrival counter) computes F and resets both words.
__global__ void __launch_bounds__(256) sym_exponent_kernel(const double *__restrict__ mass,
                                                           int64_t N, double eps,
                                                           int *__restrict__ F,
                                                           unsigned long long *mmax_bits,
                                                           unsigned *arrivals) {
    __shared__ double part[8];
    __shared__ bool last;
    double m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += 4 * stride) {
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = i + k * stride < N ? fabs(__ldg(mass + i + k * stride)) : 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) m = fmax(m, v[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) m = fmax(m, part[k]);
        atomicMax(mmax_bits, (unsigned long long)__double_as_longlong(m));
        __threadfence();
        last = atomicAdd(arrivals, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double mm = __longlong_as_double((long long)atomicAdd(mmax_bits, 0ull));
        const double per = fmax(0.3849002 / (eps * eps), 1.0 / eps);
        *F = fx::exponent_for(1.02 * (double)N * mm * per);
        *mmax_bits = 0ull;
        *arrivals = 0u;
    }
}

// ------------------------------------------------------------- FP64 pairs
// The same decomposition with FP64 arithmetic throughout (positions, pairs,
// sums), for the FP64 policy: each unordered pair once, its j-side sums
// rotated through the lanes as doubles.  The slots are the particles in
// their own order (no packing, no near/far choice); one rsqrt per unordered
// pair instead of two.
struct alignas(16) D4 {
    double x, y, z, w;
};

struct ISet64 {
    double x[IR], y[IR], z[IR], m[IR];
    double ax[IR], ay[IR], az[IR], ph[IR];
};

template <bool SYM, bool SELF, bool POT>
__device__ __forceinline__ void step64(ISet64 &S, double eps2, double jx, double jy, double jz,
                                       double jm, double &bx, double &by, double &bz, double &bp,
                                       int self_k) {
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        const double mj = (SELF && k == self_k) ? 0.0 : jm;
        const double dx = jx - S.x[k], dy = jy - S.y[k], dz = jz - S.z[k];
        const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
        const double ri = rsqrt(r2);
        const double ri3 = ri * ri * ri;
        const double sj = mj * ri3;
        S.ax[k] = fma(sj, dx, S.ax[k]);
        S.ay[k] = fma(sj, dy, S.ay[k]);
        S.az[k] = fma(sj, dz, S.az[k]);
        if (POT) S.ph[k] = fma(mj, ri, S.ph[k]);
        if (SYM) {
            const double si = S.m[k] * ri3;
            bx = fma(-si, dx, bx);
            by = fma(-si, dy, by);
            bz = fma(-si, dz, bz);
            if (POT) bp = fma(S.m[k], ri, bp);
        }
    }
}

template <bool SYM, bool POT>
__device__ __forceinline__ void rotate_set64(ISet64 &S, double eps2, const double (&j)[4],
                                             D4 &b, int self_k) {
    const int src = (threadIdx.x + 1) & 31;
    double jx = j[0], jy = j[1], jz = j[2], jm = j[3];
    double bx = 0.0, by = 0.0, bz = 0.0, bp = 0.0;
    auto rotate = [&]() {
        jx = __shfl_sync(0xffffffffu, jx, src);
        jy = __shfl_sync(0xffffffffu, jy, src);
        jz = __shfl_sync(0xffffffffu, jz, src);
        jm = __shfl_sync(0xffffffffu, jm, src);
        if (SYM) {
            bx = __shfl_sync(0xffffffffu, bx, src);
            by = __shfl_sync(0xffffffffu, by, src);
            bz = __shfl_sync(0xffffffffu, bz, src);
            if (POT) bp = __shfl_sync(0xffffffffu, bp, src);
        }
    };
    int s0 = 0;
    if (self_k >= 0) {
        step64<SYM, true, POT>(S, eps2, jx, jy, jz, jm, bx, by, bz, bp, self_k);
        rotate();
        s0 = 1;
    }
#pragma unroll 2
    for (int st = s0; st < JS; ++st) {
        step64<SYM, false, POT>(S, eps2, jx, jy, jz, jm, bx, by, bz, bp, -1);
        rotate();
    }
    b = D4{bx, by, bz, bp};
}

__device__ __forceinline__ void load_j64(const SymParams64 &p, int64_t s, double (&j)[4]) {
    if (s < p.N) {
        j[0] = __ldg(p.pos64 + 3 * s);
        j[1] = __ldg(p.pos64 + 3 * s + 1);
        j[2] = __ldg(p.pos64 + 3 * s + 2);
        j[3] = __ldg(p.mass64 + s);
    } else {
        j[0] = j[1] = j[2] = j[3] = 0.0;  // padding: zero mass at the origin
    }
}

constexpr size_t kRed64Bytes = 2 * KB * SW * 32 * sizeof(D4);

template <bool POT>
__global__ void __launch_bounds__(SNT, CPS) force_sym64_kernel(const SymParams64 p) {
    extern __shared__ __align__(16) unsigned char smem64[];
    D4 *red = reinterpret_cast<D4 *>(smem64);  // [2][KB][SW][32]
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int64_t c = blockIdx.x;
    int64_t u = __ldg(p.lo + c);
    const int64_t u_end = __ldg(p.lo + c + 1);
    if (u >= u_end) return;
    const int F = __ldg(p.fx_exp);
    const int64_t t0 = u / US;
    int64_t I = 0;
    while (row_start(I + 1, p.nb) <= t0) ++I;
    int64_t J = I + (t0 - row_start(I, p.nb));
    ISet64 S;
    int half = 0;
    bool row_open = false;
    while (u < u_end) {
        const int qa = (int)(u % US) * KB;
        const int64_t item_end = (u / US + 1) * US;
        const int64_t seg_end = item_end < u_end ? item_end : u_end;
        const int qb = qa + (int)(seg_end - u) * KB;
        const int64_t ib = I * BI + w * 128;
        if (!row_open) {
#pragma unroll
            for (int k = 0; k < IR; ++k) {
                double v[4];
                load_j64(p, ib + 32 * k + l, v);
                S.x[k] = v[0];
                S.y[k] = v[1];
                S.z[k] = v[2];
                S.m[k] = v[3];
                S.ax[k] = S.ay[k] = S.az[k] = S.ph[k] = 0.0;
            }
            row_open = true;
        }
        const bool sym = J != I;
        const int64_t jb = J * BI;
        double jn[4];
        load_j64(p, jb + qa * JS + l, jn);
        for (int q = qa; q < qb; ++q) {
            double jc[4] = {jn[0], jn[1], jn[2], jn[3]};
            if (q + 1 < qb) load_j64(p, jb + (q + 1) * JS + l, jn);
            D4 b;
            if (sym) {
                rotate_set64<true, POT>(S, p.eps2_64, jc, b, -1);
                red[((half * KB + (q % KB)) * SW + w) * 32 + l] = b;
            } else {
                rotate_set64<false, POT>(S, p.eps2_64, jc, b, (q >> 2) == w ? (q & 3) : -1);
            }
            if (sym && (q + 1) % KB == 0) {
                __syncthreads();
                for (int v = tid; v < KB * JS * 4; v += SNT) {
                    const int qq = v >> 7, ll = (v >> 2) & 31, e = v & 3;
                    const double *r = reinterpret_cast<const double *>(red) +
                                      ((half * KB + qq) * SW * 32 + ll) * 4 + e;
                    double sum = 0.0;
#pragma unroll
                    for (int w2 = 0; w2 < SW; ++w2) sum += r[w2 * 32 * 4];
                    if (POT || e < 3) add_fixed(p, e, jb + (q + 1 - KB + qq) * JS + ll, sum, F);
                }
                half ^= 1;
            }
        }
        u = seg_end;
        if ((J == p.nb - 1 && qb == NJS) || u == u_end) {
#pragma unroll
            for (int kk = 0; kk < IR; ++kk) {
                const int64_t slot = I * BI + w * 128 + 32 * kk + l;
                add_fixed(p, 0, slot, S.ax[kk], F);
                add_fixed(p, 1, slot, S.ay[kk], F);
                add_fixed(p, 2, slot, S.az[kk], F);
                if (POT) add_fixed(p, 3, slot, S.ph[kk], F);
            }
            row_open = false;
        }
        if (qb == NJS && ++J == p.nb) {
            ++I;
            J = I;
        }
    }
}

// ------------------------------------------------ cost-weighted stream-K
// Relative cost of a stream-K unit (KBP j-sets of an item, at whose end
// the CTA's warps meet at a barrier): the slowest warp's FP32-pipe cycles
// per lane and step over the unit's j-sets -- far pairs 18 off the diagonal
// (13 on it: i-side only), near pairs 24 (19) -- plus 28 that every unit
// costs alike.  That constant was fitted to per-CTA timers: with 1 the CTAs'
// times grew with their number of units (regression slope ~40 % of a
// unit's mean time); with 28 the last CTA of a 2^20 Plummer evaluation ends
// 0.2 % after the mean (0.9 % with the earlier per-item sum of all warps'
// j-sets), of a 2^18 one 1.1 %.  The FP64 kernel's units all cost the same.
constexpr uint32_t kCostSymFar = 18, kCostSymNear = 24, kCostDiagFar = 13, kCostDiagNear = 19;
constexpr uint32_t kCostSymUnit = 28;

__device__ __forceinline__ void item_of(int64_t t, int64_t nb, int64_t &I, int64_t &J) {
    const double b = 2.0 * (double)nb + 1.0;
    int64_t r = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
    if (r < 0) r = 0;
    if (r > nb - 1) r = nb - 1;
    while (r > 0 && row_start(r, nb) > t) --r;
    while (r + 1 < nb && row_start(r + 1, nb) <= t) ++r;
    I = r;
    J = r + (t - row_start(r, nb));
}

// The adaptive FP32 kernel's unit costs of item t, one thread: the same
// sums as sym_cost_kernel<2, NW, JSP> (which adds them up per item).
__device__ void item_unit_costs(const SymParams &p, int64_t t, uint32_t (&uc)[US]) {
    int64_t I, J;
    item_of(t, p.nb, I, J);
    const bool sym = I != J;
    const uint32_t cn = sym ? kCostSymNear : kCostDiagNear;
    const uint32_t cf = sym ? kCostSymFar : kCostDiagFar;
    for (int u = 0; u < US; ++u) uc[u] = 0;
    for (int w = 0; w < NW; ++w) {
        float wb[7];
        for (int a = 0; a < 7; ++a) wb[a] = __ldg(p.wbox + (I * NW + w) * 8 + a);
        for (int u = 0; u < US; ++u) {
            uint32_t sum = 0;
            for (int k = 0; k < KBP; ++k) {
                float tb[7];
                for (int a = 0; a < 7; ++a) tb[a] = __ldg(p.jbox + (J * NJSP + u * KBP + k) * 8 + a);
                sum += boxes_near(wb, tb, p.gamma) ? cn : cf;
            }
            uc[u] = sum > uc[u] ? sum : uc[u];
        }
    }
    for (int u = 0; u < US; ++u) uc[u] += kCostSymUnit;
}

// One warp per item: the near/far decisions the pair kernel will take.  For
// the adaptive FP32 kernel lane l takes j-set l (unit l / 2): the unit's
// cost is the maximum over the warps of its two j-sets' sum; other modes
// give every unit the same cost.
template <int MODE, int NWK, int JSET>
__global__ void __launch_bounds__(256) sym_cost_kernel(const SymParams p, uint32_t *cost) {
    constexpr int NJ = BI / JSET;  // j-sets per block
    constexpr int WS = BI / NWK;   // i-slots per warp
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (t >= p.T) return;  // whole warps
    int64_t I, J;
    item_of(t, p.nb, I, J);
    const bool sym = I != J;
    const uint32_t cn = sym ? kCostSymNear : kCostDiagNear;
    const uint32_t cf = sym ? kCostSymFar : kCostDiagFar;
    uint32_t c = 0;
    if constexpr (MODE != 2) {
        // every unit of the item alike (every j-set near for MODE 1)
        c = (l & 1) ? 0u : 2 * (MODE == 1 ? cn : cf) + kCostSymUnit;
    } else {
        static_assert(NJ == 32 && KBP == 2 && NWK == NW, "lane l: j-set l, unit l / 2");
        float tb[7];
#pragma unroll
        for (int a = 0; a < 7; ++a) tb[a] = __ldg(p.jbox + (J * NJ + l) * 8 + a);
        uint32_t m = 0;
        for (int w = 0; w < NWK; ++w) {
            float wb[7];
#pragma unroll
            for (int a = 0; a < 7; ++a) wb[a] = __ldg(p.wbox + ((I * BI + w * WS) / WS) * 8 + a);
            const uint32_t v = boxes_near(wb, tb, p.gamma) ? cn : cf;
            const uint32_t pair = v + __shfl_xor_sync(0xffffffffu, v, 1);
            m = pair > m ? pair : m;
        }
        c = (l & 1) ? 0u : m + kCostSymUnit;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (l == 0) cost[t] = c;
}

// prefix[t] = sum of cost[0, t), prefix[T] = total (one block, fixed order).
__global__ void __launch_bounds__(1024) sym_scan_kernel(const uint32_t *cost, int64_t T,
                                                        unsigned long long *prefix) {
    __shared__ unsigned long long part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (T + 1023) / 1024;
    const int64_t a = tid * per, b = (a + per) < T ? (a + per) : T;
    unsigned long long s = 0;
    for (int64_t t = a; t < b; ++t) s += cost[t];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < 1024; ++i) {
            const unsigned long long v = part[i];
            part[i] = run;
            run += v;
        }
        prefix[T] = run;
    }
    __syncthreads();
    unsigned long long run = part[tid];
    for (int64_t t = a; t < b; ++t) {
        prefix[t] = run;
        run += cost[t];
    }
}

// lo[c] = the unit where the cumulative cost reaches c / ctas of the total
// (the nearest unit boundary, from the item's unit costs for the adaptive
// kernel, linearly inside an item otherwise); lo[0] = 0, lo[ctas] = U,
// non-decreasing.
template <int MODE>
__global__ void sym_ranges_kernel(const SymParams p, const uint32_t *cost,
                                  const unsigned long long *prefix, int64_t T, int64_t ctas,
                                  int64_t *lo) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= ctas;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c == 0 || c == ctas) {
            lo[c] = c == 0 ? 0 : T * US;
            continue;
        }
        const unsigned long long target = prefix[T] * (unsigned long long)c / (unsigned long long)ctas;
        int64_t a = 0, b = T - 1;
        while (a < b) {
            const int64_t m = (a + b + 1) / 2;
            if (prefix[m] <= target)
                a = m;
            else
                b = m - 1;
        }
        const unsigned long long r = target - prefix[a];
        int64_t off;
        if (MODE == 2) {
            uint32_t uc[US];
            item_unit_costs(p, a, uc);
            unsigned long long run = 0;
            off = 0;
            while (off < US && run + uc[off] <= r) run += uc[off++];
            if (off < US && 2 * (r - run) > uc[off]) ++off;  // the nearer boundary
        } else {
            off = (int64_t)(r * (unsigned long long)US / cost[a]);
            if (off > US) off = US;
        }
        lo[c] = a * US + off;
    }
}

template <int POL, int MODE, bool POT>
int launch_pair(const SymParams &p, cudaStream_t st) {
    auto kern = force_sym_kernel<POL, MODE, POT>;
    const size_t smem = kRedBytes + 4 * BI * sizeof(Acc<POL>) +
                        (POL == NB_PREC_F64ACC ? 4 * BI * sizeof(float) : 0) +
                        (MODE == 2 ? 3 * BI * sizeof(float2) : 0);
    const int rc = smem_optin(reinterpret_cast<const void *>(kern), smem);
    if (rc != NB_OK) return rc;
    kernel_timer_begin(st);
    kern<<<(unsigned)p.ctas, NT, smem, st>>>(p);
    kernel_timer_end(st);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// FP64: the cost estimate per (16 warps x 32-slot j-sets), else per
// (8 warps x 64-slot j-sets).
template <int MODE, bool FP64 = false>
int launch_split(const SymParams &p, const ForceJob &j, const SymLayout &y) {
    if constexpr (FP64)
        sym_cost_kernel<0, SW, JS><<<(unsigned)cdiv(p.T * 32, 256), 256, 0, j.stream>>>(p, y.cost);
    else
        sym_cost_kernel<MODE, NW, JSP><<<(unsigned)cdiv(p.T * 32, 256), 256, 0, j.stream>>>(p, y.cost);
    sym_scan_kernel<<<1, 1024, 0, j.stream>>>(y.cost, p.T, y.prefix);
    sym_ranges_kernel<FP64 ? 0 : MODE><<<(unsigned)cdiv(p.ctas + 1, 256), 256, 0, j.stream>>>(
        p, y.cost, y.prefix, p.T, p.ctas, y.lo);
    sym_exponent_kernel<<<(unsigned)std::min<int64_t>(cdiv(j.N, 4 * 256), 1024), 256, 0,
                          j.stream>>>(j.mass, j.N, j.eps, y.fx_exp, y.mmax_bits, y.arrivals);
    count_launch(4);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

int launch_fold(const SymParams &p, const ForceJob &j, const int *perm) {
    const int64_t fold_blocks = std::min<int64_t>(cdiv(p.Np, 256), 64 * (int64_t)device_sm_count());
    sym_fold_kernel<<<(unsigned)fold_blocks, 256, 0, j.stream>>>(p, j.N, perm, j.G, j.acc, j.pot,
                                                                 j.vel, j.kick);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int POL, int MODE>
int launch_sym_mode(const SymParams &p, const ForceJob &j, const SymLayout &y, const int *perm) {
    NB_TRY_SYM(launch_split<MODE>(p, j, y));
    NB_TRY_SYM(j.pot ? launch_pair<POL, MODE, true>(p, j.stream)
                     : launch_pair<POL, MODE, false>(p, j.stream));
    return launch_fold(p, j, perm);
}

template <bool POT>
int launch_pair64(const SymParams64 &p, cudaStream_t st) {
    auto kern = force_sym64_kernel<POT>;
    const int rc = smem_optin(reinterpret_cast<const void *>(kern), kRed64Bytes);
    if (rc != NB_OK) return rc;
    kern<<<(unsigned)p.ctas, SNT, kRed64Bytes, st>>>(p);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

int launch_sym64(const SymParams64 &p, const ForceJob &j, const SymLayout &y) {
    NB_TRY_SYM(launch_split<0, true>(p, j, y));
    NB_TRY_SYM(j.pot ? launch_pair64<true>(p, j.stream) : launch_pair64<false>(p, j.stream));
    return launch_fold(p, j, nullptr);
}

template <int POL>
int launch_sym_pol(const SymParams &p, const ForceJob &j, const SymLayout &y, int mode,
                   const int *perm) {
    switch (mode) {
        case 0: return launch_sym_mode<POL, 0>(p, j, y, perm);
        case 1: return launch_sym_mode<POL, 1>(p, j, y, perm);
        default: return launch_sym_mode<POL, 2>(p, j, y, perm);
    }
}

}  // namespace

SymSizes sym_sizes(int64_t Np) {
    SymSizes z{};
    z.nb = cdiv(Np, kSymBlock);
    z.T = z.nb * (z.nb + 1) / 2;
    z.U = z.T * US;
    z.ctas = std::min<int64_t>(CPS * (int64_t)device_sm_count(), z.U);
    z.fx_bytes = 8 * 8 * (size_t)(z.nb * kSymBlock);  // 4 components x 2 words per slot
    z.cost_bytes = 256 + align_up(4 * (size_t)z.T, 256) + align_up(8 * (size_t)(z.T + 1), 256) +
                   8 * (size_t)(z.ctas + 1);
    return z;
}

SymLayout sym_layout(char *ws, const WsLayout &L) {
    const SymSizes z = sym_sizes(L.Np);
    SymLayout y;
    char *c = ws + L.sym_cost;
    y.fx_exp = reinterpret_cast<int *>(c);
    y.mmax_bits = reinterpret_cast<unsigned long long *>(c + 8);
    y.arrivals = reinterpret_cast<unsigned *>(c + 16);
    y.cost = reinterpret_cast<uint32_t *>(c + 256);
    y.prefix = reinterpret_cast<unsigned long long *>(c + 256 + align_up(4 * (size_t)z.T, 256));
    y.lo = reinterpret_cast<int64_t *>(c + 256 + align_up(4 * (size_t)z.T, 256) +
                                       align_up(8 * (size_t)(z.T + 1), 256));
    y.acc_fx = reinterpret_cast<unsigned long long *>(ws + L.sym_fx);
    return y;
}

int launch_force_sym(const ForceJob &j, bool adaptive) {
    if (j.eps <= 0.0) return fail(NB_ERR_UNSUPPORTED, "symmetric pairs need eps > 0");
    if (j.L.sym_fx_bytes == 0)
        return fail(NB_ERR_WORKSPACE, "workspace has no symmetric-pair buffers");
    const SymSizes z = sym_sizes(j.L.Np);
    const SymLayout y = sym_layout(j.ws, j.L);
    SymParams p;
    char *sb = j.ws + j.L.sortbuf;
    p.soa = reinterpret_cast<const float *>(j.ws + j.L.packA);
    p.Np = z.nb * kSymBlock;
    p.nb = z.nb;
    p.T = z.T;
    p.U = z.U;
    p.ctas = z.ctas;
    const float ef = (float)j.eps;
    p.eps2 = ef * ef;
    p.gamma = j.gamma;
    p.jbox = adaptive ? sort_tile_boxes(sb, j.L) : nullptr;
    p.wbox = adaptive ? sort_block_boxes(sb, j.L) : nullptr;
    p.acc_fx = y.acc_fx;
    p.fx_exp = y.fx_exp;
    p.lo = y.lo;
    const int *perm = adaptive ? sort_perm(sb, j.L) : nullptr;
    p.status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    const int mode = adaptive ? 2 : (j.split ? 1 : 0);
    if (j.precision == NB_PREC_FP64) {
        SymParams64 p64;
        static_cast<SymParams &>(p64) = p;
        p64.pos64 = j.pos;
        p64.mass64 = j.mass;
        p64.N = j.N;
        p64.eps2_64 = j.eps * j.eps;
        return launch_sym64(p64, j, y);
    }
    switch (j.precision) {
        case NB_PREC_FP32: return launch_sym_pol<NB_PREC_FP32>(p, j, y, mode, perm);
        case NB_PREC_KAHAN: return launch_sym_pol<NB_PREC_KAHAN>(p, j, y, mode, perm);
        case NB_PREC_F64ACC: return launch_sym_pol<NB_PREC_F64ACC>(p, j, y, mode, perm);
    }
    return fail(NB_ERR_INVALID, "unknown precision %d", j.precision);
}

}  // namespace nb
