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
// cut into units of 4 j-sets and split over one persistent CTA per SM into
// contiguous ranges of equal estimated cost (stream-K: a range may start or
// end inside an item).  The estimate counts FP32 operations per (warp,
// j-set) from the same near/far box tests the pair kernel makes; three small
// kernels compute it, scan it and cut the ranges.
// A CTA keeps block I in registers: warp w holds the 128 slots
// I*2048 + w*128 + [0, 128), lane l the four slots  + 32k + l  (k = 0..3,
// two packed f32x2 pairs).  For every 32-slot j-set of block J each warp
// loads one j-particle per lane and rotates the set through its lanes with
// shuffles: at step s lane l holds j-slot (l + s) mod 32, so in 32 steps
// every lane meets every j once, and the j-particle's own sums (a_j, phi_j)
// travel with it and come home to lane l.
//
//   * Off-diagonal items (I < J): both halves of every pair.  The 16 warps'
//     j-side sums of 4 j-sets are added in warp order in shared memory (one
//     barrier per 4 j-sets) and stored as the FP32 partial P[I, J] of the
//     J-block particles.
//   * Diagonal items (I = J): the i-side only, over all ordered pairs of
//     the block; the self pair (j-set 4w + k at rotation step 0 for lane
//     slot k of warp w) gets a zero mass, so Eq. 1's j != i holds exactly.
//
// The i-side FP32 register sums are folded into the accumulation policy
// (FP32, Kahan or FP64; totals kept in shared memory) every 4 j-sets (128
// terms per running sum; for F64ACC through an FP32 middle sum in shared
// memory that goes into FP64 every 16 j-sets, FP64 adds being slow on this
// part), and stored once per row segment as an FP64 record.  In
// Morton order a particle's strongest, mutually cancelling terms (its
// spatial neighbours) arrive together; with 16 j-sets per flush the FP32
// running sums of central particles of a log-normal Plummer sphere
// (N = 300001, eps = 1e-3) lost up to 1e-5 of |a|, with 4 they stay at the
// 2e-6 of the unsorted order.  A second kernel adds, slot by
// slot in a fixed order, the records of the row's CTAs and the partials
// P[I', I] for I' < I, applies G, scatters through the Morton permutation
// and optionally kicks the velocity.  Every
// sum runs in a fixed order: results are bitwise reproducible.
//
// Displacements: single floats, hi/lo pairs (x_j.hi - x_i.hi) +
// (x_j.lo - x_i.lo), or adaptive: per (warp i-set, j-set) the hi/lo form
// only when the bounding boxes are closer than gamma * max|x| (a 64-bit
// mask per warp and item, from the Morton-sorted pack's boxes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {

using dev::Acc;
using dev::add2;
using dev::f2;
using dev::fma2;
using dev::mul2;
using dev::rsqrt_approx;

namespace {

constexpr int NW = 16;              // warps per CTA
constexpr int NT = NW * 32;         // threads per CTA
constexpr int IR = 4;               // i-slots per lane (two packed pairs)
constexpr int BI = NW * 32 * IR;    // slots per row block
constexpr int JS = 32;              // slots per j-set (one per lane)
constexpr int NJS = BI / JS;        // j-sets per block
constexpr int KB = 4;               // j-sets per cross-warp reduction
constexpr int FL = 4;               // j-sets per i-side flush of the register sums
constexpr int FL2 = 16;             // F64ACC: j-sets per flush of the FP32 middle sums
constexpr int US = NJS / KB;        // stream-K units (KB j-sets) per item
static_assert(BI == kSymBlock, "row block size");
static_assert(KB * JS * 4 == NT, "one reduced value per thread");
static_assert(NJS % KB == 0 && NJS % FL2 == 0 && FL2 % FL == 0, "groups tile a block");
constexpr size_t kRedBytes = 2 * KB * NW * 32 * sizeof(float4);

struct SymParams {
    const float *soa;   // packed SoA [7][Np]
    int64_t Np;
    int64_t nb;         // row blocks
    int64_t T;          // items nb (nb + 1) / 2
    int64_t U;          // stream-K units T * US (KB j-sets of one item each)
    int64_t ctas;       // grid size of the pair kernel
    int64_t K;          // record slots per row
    float eps2;
    float gamma;        // adaptive threshold; the mode decides whether it is used
    const float *jbox;  // per 32 slots: lo[3], hi[3], max|x|, pad
    const float *wbox;  // per 128 slots
    float *P;           // [nb (nb - 1) / 2][BI][4]
    double *rec;        // [nb][K][BI][4]
    const int64_t *lo;  // [ctas + 1]: CTA c owns units [lo[c], lo[c + 1])
    uint32_t *status;
};

__host__ __device__ inline int64_t row_start(int64_t I, int64_t nb) {
    return I * nb - I * (I - 1) / 2;
}

// The CTA whose unit range holds unit u: the last c with lo[c] <= u (the
// ranges are contiguous and ordered; empty ranges are never the answer).
__device__ __forceinline__ int64_t range_owner(const int64_t *lo, int64_t ctas, int64_t u) {
    int64_t a = 0, b = ctas - 1;
    while (a < b) {
        const int64_t m = (a + b + 1) / 2;
        if (__ldg(lo + m) <= u)
            a = m;
        else
            b = m - 1;
    }
    return a;
}

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

// One rotation step: the lane's four i-slots against its current j.  With
// SELF, i-slot self_k is the j-particle itself: its half of the pair gets a
// zero mass (Eq. 1 leaves out j = i).
template <bool NEAR, bool SYM, bool SELF>
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
        if (NEAR) {
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
        S.ph[g] = fma2(M, ri, S.ph[g]);
        if (SYM) {
            const float2 si = mul2(S.nm[g], ri3);  // -m_i r^-3
            bx = fmaf(si.x, dx.x, bx);
            bx = fmaf(si.y, dx.y, bx);
            by = fmaf(si.x, dy.x, by);
            by = fmaf(si.y, dy.y, by);
            bz = fmaf(si.x, dz.x, bz);
            bz = fmaf(si.y, dz.y, bz);
            bp = fmaf(S.m[g].x, ri.x, bp);
            bp = fmaf(S.m[g].y, ri.y, bp);
        }
    }
}

// 32 steps over one j-set; the j values (and sums) end on their home lane.
// self_k >= 0 (diagonal items only): the j-set is the warp's own i-slots
// 32 self_k + [0, 32), so step 0 pairs every lane with itself.
template <bool NEAR, bool SYM>
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
        if (NEAR) {
            jxl = __shfl_sync(0xffffffffu, jxl, src);
            jyl = __shfl_sync(0xffffffffu, jyl, src);
            jzl = __shfl_sync(0xffffffffu, jzl, src);
        }
        if (SYM) {
            bx = __shfl_sync(0xffffffffu, bx, src);
            by = __shfl_sync(0xffffffffu, by, src);
            bz = __shfl_sync(0xffffffffu, bz, src);
            bp = __shfl_sync(0xffffffffu, bp, src);
        }
    };
    int s0 = 0;
    if (self_k >= 0) {
        step<NEAR, SYM, true>(S, e2, jx, jy, jz, jm, jxl, jyl, jzl, bx, by, bz, bp, self_k);
        rotate();
        s0 = 1;
    }
#pragma unroll 4
    for (int s = s0; s < JS; ++s) {
        step<NEAR, SYM, false>(S, e2, jx, jy, jz, jm, jxl, jyl, jzl, bx, by, bz, bp);
        rotate();
    }
    b = make_float4(bx, by, bz, bp);
}

template <int MODE, bool SYM>
__device__ __forceinline__ void run_set(ISet &S, const float2 e2, const float (&j)[7], bool near,
                                        float4 &b, int self_k) {
    if (MODE == 1 || (MODE == 2 && near))
        rotate_set<true, SYM>(S, e2, j, b, self_k);
    else
        rotate_set<false, SYM>(S, e2, j, b, self_k);
}

__device__ __forceinline__ void load_j(const SymParams &p, int64_t s, float (&j)[7]) {
#pragma unroll
    for (int a = 0; a < 7; ++a) j[a] = __ldg(p.soa + a * p.Np + s);
}

// MODE: 0 single-float displacement, 1 hi/lo, 2 adaptive.
template <int POL, int MODE>
__global__ void __launch_bounds__(NT, 1) force_sym_kernel(const SymParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *red = reinterpret_cast<float4 *>(smem);                   // [2][KB][NW][32]
    Acc<POL> *tot = reinterpret_cast<Acc<POL> *>(smem + kRedBytes);   // [16][NT]
    constexpr bool MID = POL == NB_PREC_F64ACC;
    float *mid = reinterpret_cast<float *>(smem + kRedBytes + 16 * NT * sizeof(Acc<POL>));
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int64_t c = blockIdx.x;
    int64_t u = __ldg(p.lo + c);
    const int64_t u_end = __ldg(p.lo + c + 1);
    if (u >= u_end) return;
    const int64_t t0 = u / US;
    int64_t I = 0;
    while (row_start(I + 1, p.nb) <= t0) ++I;
    int64_t J = I + (t0 - row_start(I, p.nb));
    const float2 e2 = f2(p.eps2, p.eps2);
    ISet S;
    int half = 0;
    bool row_open = false;
    while (u < u_end) {
        // this CTA's j-sets [qa, qb) of item (I, J)
        const int qa = (int)(u % US) * KB;
        const int64_t item_end = (u / US + 1) * US;
        const int64_t seg_end = item_end < u_end ? item_end : u_end;
        const int qb = qa + (int)(seg_end - u) * KB;
        const int64_t ib = I * BI + w * 128;  // this warp's i-set
        if (!row_open) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                float v[2][7];
#pragma unroll
                for (int h = 0; h < 2; ++h) load_j(p, ib + 32 * (2 * g + h) + l, v[h]);
                S.nx[g] = f2(-v[0][0], -v[1][0]);
                S.ny[g] = f2(-v[0][1], -v[1][1]);
                S.nz[g] = f2(-v[0][2], -v[1][2]);
                S.m[g] = f2(v[0][3], v[1][3]);
                S.nm[g] = f2(-v[0][3], -v[1][3]);
                S.nxl[g] = f2(-v[0][4], -v[1][4]);
                S.nyl[g] = f2(-v[0][5], -v[1][5]);
                S.nzl[g] = f2(-v[0][6], -v[1][6]);
                S.ax[g] = S.ay[g] = S.az[g] = S.ph[g] = f2(0.f, 0.f);
            }
#pragma unroll
            for (int v = 0; v < 16; ++v) {
                tot[v * NT + tid].zero();
                if (MID) mid[v * NT + tid] = 0.f;
            }
            row_open = true;
        }
        const bool sym = J != I;
        const int64_t jb = J * BI;
        // near mask of this warp's i-set against the block's 64 j-sets
        unsigned long long near = 0ull;
        if (MODE == 2) {
            float wb[7];
#pragma unroll
            for (int a = 0; a < 7; ++a) wb[a] = __ldg(p.wbox + (ib / 128) * 8 + a);
            float tb[2][7];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int a = 0; a < 7; ++a) tb[h][a] = __ldg(p.jbox + (jb / JS + l + 32 * h) * 8 + a);
            const unsigned lo = __ballot_sync(0xffffffffu, boxes_near(wb, tb[0], p.gamma));
            const unsigned hi = __ballot_sync(0xffffffffu, boxes_near(wb, tb[1], p.gamma));
            near = ((unsigned long long)hi << 32) | lo;
        }
        const int64_t pidx = J * (J - 1) / 2 + I;
        float jn[7];
        load_j(p, jb + qa * JS + l, jn);
        for (int q = qa; q < qb; ++q) {
            float jc[7];
#pragma unroll
            for (int a = 0; a < 7; ++a) jc[a] = jn[a];
            if (q + 1 < qb) load_j(p, jb + (q + 1) * JS + l, jn);
            const bool nq = (near >> q) & 1ull;
            float4 b;
            if (sym) {
                run_set<MODE, true>(S, e2, jc, nq, b, -1);
                red[((half * KB + (q % KB)) * NW + w) * 32 + l] = b;
            } else {
                run_set<MODE, false>(S, e2, jc, nq, b, (q >> 2) == w ? (q & 3) : -1);
            }
            if ((q + 1) % FL == 0 || q + 1 == qb) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float2 v4[4] = {S.ax[g], S.ay[g], S.az[g], S.ph[g]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int v0 = ((2 * g) * 4 + e) * NT + tid;
                        const int v1 = ((2 * g + 1) * 4 + e) * NT + tid;
                        if (MID) {
                            mid[v0] += v4[e].x;
                            mid[v1] += v4[e].y;
                        } else {
                            tot[v0].add(v4[e].x);
                            tot[v1].add(v4[e].y);
                        }
                    }
                    S.ax[g] = S.ay[g] = S.az[g] = S.ph[g] = f2(0.f, 0.f);
                }
                if (MID && ((q + 1) % FL2 == 0 || q + 1 == qb)) {
#pragma unroll
                    for (int v = 0; v < 16; ++v) {
                        tot[v * NT + tid].add(mid[v * NT + tid]);
                        mid[v * NT + tid] = 0.f;
                    }
                }
            }
            if (sym && (q + 1) % KB == 0) {
                __syncthreads();
                const int qq = tid >> 7, ll = (tid >> 2) & 31, e = tid & 3;
                const float *r =
                    reinterpret_cast<const float *>(red) + ((half * KB + qq) * NW * 32 + ll) * 4 + e;
                float s = 0.f;
#pragma unroll
                for (int w2 = 0; w2 < NW; ++w2) s += r[w2 * 32 * 4];
                // streaming store: the partials are read once, by the fold, and must
                // not evict the packed positions that every CTA re-reads from L2
                __stcs(p.P + ((pidx * BI) + (q + 1 - KB + qq) * JS + ll) * 4 + e, s);
                half ^= 1;
            }
        }
        u = seg_end;
        if ((J == p.nb - 1 && qb == NJS) || u == u_end) {
            // row segment done: FP64 record of the policy totals
            const int64_t k = c - range_owner(p.lo, p.ctas, row_start(I, p.nb) * US);
            // k < K by the bound of sym_sizes; never write past it
            if (k >= p.K && tid == 0) dev::set_status(p.status, kStatusInvalid);
#pragma unroll
            for (int kk = 0; kk < IR; ++kk) {
                if (k >= p.K) break;
                const int64_t slot = w * 128 + 32 * kk + l;
                double *r = p.rec + (((I * p.K + k) * BI) + slot) * 4;
                __stcs(reinterpret_cast<double2 *>(r),
                       make_double2(tot[(kk * 4 + 0) * NT + tid].value(),
                                    tot[(kk * 4 + 1) * NT + tid].value()));
                __stcs(reinterpret_cast<double2 *>(r) + 1,
                       make_double2(tot[(kk * 4 + 2) * NT + tid].value(),
                                    tot[(kk * 4 + 3) * NT + tid].value()));
            }
            row_open = false;
        }
        if (qb == NJS && ++J == p.nb) {
            ++I;
            J = I;
        }
    }
}

// Adds an FP64 record value in the policy's arithmetic.
template <int POL>
__device__ __forceinline__ void add_record(Acc<POL> &a, double v);
template <>
__device__ __forceinline__ void add_record<NB_PREC_FP32>(Acc<NB_PREC_FP32> &a, double v) {
    a.add((float)v);
}
template <>
__device__ __forceinline__ void add_record<NB_PREC_KAHAN>(Acc<NB_PREC_KAHAN> &a, double v) {
    const float h = (float)v;
    a.add(h);
    a.add((float)(v - (double)h));
}
template <>
__device__ __forceinline__ void add_record<NB_PREC_F64ACC>(Acc<NB_PREC_F64ACC> &a, double v) {
    a.s += v;
}

// Adds `count` FP32 partials (stride `stride` float4s) in order.  F64ACC adds
// groups of 8 in FP32 first (8 x 128 or 8 x 2048 pair terms, the size of one
// direct-kernel tile of FP32 sums) and each group's sum in FP64: FP64 adds are
// slow on this part and one per partial made the fold FP64-bound.
template <int POL>
__device__ __forceinline__ void add_partials(Acc<POL> (&a)[4], const float4 *P4, int64_t count,
                                             int64_t stride) {
    if (POL == NB_PREC_F64ACC) {
        for (int64_t k0 = 0; k0 < count; k0 += 8) {
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            const int64_t k1 = (k0 + 8) < count ? (k0 + 8) : count;
            for (int64_t k = k0; k < k1; ++k) {
                const float4 v = __ldcs(P4 + k * stride);
                g.x += v.x;
                g.y += v.y;
                g.z += v.z;
                g.w += v.w;
            }
            a[0].add(g.x);
            a[1].add(g.y);
            a[2].add(g.z);
            a[3].add(g.w);
        }
    } else {
        for (int64_t k = 0; k < count; ++k) {
            const float4 v = __ldcs(P4 + k * stride);
            a[0].add(v.x);
            a[1].add(v.y);
            a[2].add(v.z);
            a[3].add(v.w);
        }
    }
}

template <int POL>
__global__ void __launch_bounds__(256) sym_fold_kernel(const SymParams p, int64_t N,
                                                       const int *__restrict__ perm, double G,
                                                       double *__restrict__ acc,
                                                       double *__restrict__ pot,
                                                       double *__restrict__ vel, double kick,
                                                       uint32_t *status) {
    uint32_t bad = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = s / BI, r = s % BI;
        Acc<POL> a[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) a[e].zero();
        const int64_t rs = row_start(I, p.nb);
        const int64_t c0 = range_owner(p.lo, p.ctas, rs * US);
        const int64_t c1 = range_owner(p.lo, p.ctas, (rs + (p.nb - I)) * US - 1);
        for (int64_t k = 0; k <= c1 - c0 && k < p.K; ++k) {
            if (__ldg(p.lo + c0 + k) == __ldg(p.lo + c0 + k + 1)) continue;  // empty range
            const double2 *rr = reinterpret_cast<const double2 *>(p.rec + (((I * p.K + k) * BI) + r) * 4);
            const double2 u = __ldg(rr), v = __ldg(rr + 1);
            add_record<POL>(a[0], u.x);
            add_record<POL>(a[1], u.y);
            add_record<POL>(a[2], v.x);
            add_record<POL>(a[3], v.y);
        }
        add_partials<POL>(a, reinterpret_cast<const float4 *>(p.P) + (I * (I - 1) / 2) * BI + r, I,
                          BI);
        const double ph = a[3].value();
        const double ax = G * a[0].value(), ay = G * a[1].value(), az = G * a[2].value();
        const double gp = -G * ph;
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
    if (bad) dev::set_status(status, kStatusNonFinite);
}

// ------------------------------------------------ cost-weighted stream-K
// Relative cost of one (warp, j-set) of an item.  Far pairs: the FP32 pipe
// cycles per lane and step (off-diagonal 18, diagonal i-side only 13).  Near
// pairs take 24 / 19 pipe cycles, but a near j-set of one warp also holds
// its 15 siblings at the next barrier; weighted 36 / 28 the per-CTA timers
// of a 2^20 Plummer evaluation end within 1 % of each other (24 / 19: the
// last CTA 3.5 % after the median).
constexpr uint32_t kCostSymFar = 18, kCostSymNear = 36, kCostDiagFar = 13, kCostDiagNear = 28;
constexpr uint32_t kUnitCostMin = KB * NW * kCostDiagFar;
constexpr uint32_t kUnitCostMax = KB * NW * kCostSymNear;

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

// One warp per item: the near/far decisions the pair kernel will take.
template <int MODE>
__global__ void __launch_bounds__(256) sym_cost_kernel(const SymParams p, uint32_t *cost) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (t >= p.T) return;  // whole warps
    int64_t I, J;
    item_of(t, p.nb, I, J);
    const bool sym = I != J;
    const uint32_t cn = sym ? kCostSymNear : kCostDiagNear;
    const uint32_t cf = sym ? kCostSymFar : kCostDiagFar;
    uint32_t c = 0;
    if (MODE != 2) {
        c = (MODE == 1 ? cn : cf) * 2 * NW;  // this lane's 2 j-sets x 16 warps
    } else {
        float tb[2][7];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int a = 0; a < 7; ++a) tb[h][a] = __ldg(p.jbox + (J * BI / JS + l + 32 * h) * 8 + a);
        for (int w = 0; w < NW; ++w) {
            float wb[7];
#pragma unroll
            for (int a = 0; a < 7; ++a) wb[a] = __ldg(p.wbox + ((I * BI + w * 128) / 128) * 8 + a);
#pragma unroll
            for (int h = 0; h < 2; ++h) c += boxes_near(wb, tb[h], p.gamma) ? cn : cf;
        }
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
// (linear inside an item); lo[0] = 0, lo[ctas] = U, non-decreasing.
__global__ void sym_ranges_kernel(const uint32_t *cost, const unsigned long long *prefix,
                                  int64_t T, int64_t ctas, int64_t *lo) {
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
        int64_t off = (int64_t)((target - prefix[a]) * (unsigned long long)US / cost[a]);
        if (off > US) off = US;
        lo[c] = a * US + off;
    }
}

template <int POL, int MODE>
int launch_sym_mode(const SymParams &p, const ForceJob &j, const int *perm, uint32_t *status) {
    {
        uint32_t *cost = reinterpret_cast<uint32_t *>(j.ws + j.L.sym_cost);
        unsigned long long *prefix = reinterpret_cast<unsigned long long *>(
            j.ws + j.L.sym_cost + align_up(4 * (size_t)p.T, 256));
        int64_t *lo = const_cast<int64_t *>(p.lo);
        sym_cost_kernel<MODE><<<(unsigned)cdiv(p.T * 32, 256), 256, 0, j.stream>>>(p, cost);
        sym_scan_kernel<<<1, 1024, 0, j.stream>>>(cost, p.T, prefix);
        sym_ranges_kernel<<<(unsigned)cdiv(p.ctas + 1, 256), 256, 0, j.stream>>>(cost, prefix, p.T,
                                                                                 p.ctas, lo);
        count_launch(3);
        NB_CUDA(cudaGetLastError());
    }
    auto kern = force_sym_kernel<POL, MODE>;
    const size_t smem = kRedBytes + 16 * NT * sizeof(Acc<POL>) +
                        (POL == NB_PREC_F64ACC ? 16 * NT * sizeof(float) : 0);
    static const cudaError_t optin =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    NB_CUDA(optin);
    kern<<<(unsigned)p.ctas, NT, smem, j.stream>>>(p);
    count_launch();
    NB_CUDA(cudaGetLastError());
    const int64_t fold_blocks = std::min<int64_t>(cdiv(j.N, 256), 64 * (int64_t)device_sm_count());
    sym_fold_kernel<POL><<<(unsigned)fold_blocks, 256, 0, j.stream>>>(
        p, j.N, perm, j.G, j.acc, j.pot, j.vel, j.kick, status);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int POL>
int launch_sym_pol(const SymParams &p, const ForceJob &j, int mode, const int *perm,
                   uint32_t *status) {
    switch (mode) {
        case 0: return launch_sym_mode<POL, 0>(p, j, perm, status);
        case 1: return launch_sym_mode<POL, 1>(p, j, perm, status);
        default: return launch_sym_mode<POL, 2>(p, j, perm, status);
    }
}

// ================================================================ batched
// Many independent systems (offsets [B+1], eps [B]), each unordered pair of
// a system evaluated once as above, at warp granularity.  Every system is
// padded to whole 128-slot blocks in Morton order (re-sorted every 16 steps);
// a work item is (system c, i-block a, j-blocks [b0, b1)) with b0 >= a and at
// most 8 j-blocks.  Persistent warps take items from an atomic queue ordered
// largest first; a warp holds its i-block in registers (4 slots per lane),
// rotates each 32-slot j-set through its lanes (j-side sums travelling with
// the particle) and writes, per off-diagonal block pair (a, b), the FP32
// j-side partial of block b's 128 slots, and per item the i-side total as
// an FP64 record.  A fold adds, per slot and in a fixed order, the records of
// its row and the partials of the blocks a' < a, so results do not depend on
// which warp took which item.
constexpr int BW = 128;           // slots per warp block
constexpr int BG = 8;             // j-blocks per item at most
constexpr int kBsMaxN = 8192;     // particles per system (64 blocks)
constexpr int kBsResort = 16;     // steps between Morton re-sorts

struct BsParams {
    int32_t B;
    const int64_t *offsets;
    const double *eps;
    double G;
    const double *mass;
    double *pos, *vel, *acc, *pot;
    int64_t *sbase;      // [B + 1] first slot of each system (multiples of 128)
    int64_t *ibase;      // [B + 1] first item of each system
    int64_t *pbase;      // [B + 1] first block pair of each system
    int32_t *rstart;     // [blocks + 1] first item of each row (global block index)
    int32_t *bsys;       // [blocks] system of each block
    int4 *items;         // [items] (c, a, b0, b1)
    int32_t *order;      // [items] largest first
    unsigned *counter;   // queue head
    int64_t *totals;     // slots, items, block pairs, blocks
    float *soa;          // [7][Ns]
    int64_t Ns;          // slot capacity
    int *perm;           // [Ns] slot -> particle, -1 for padding
    float *box32;        // [Ns / 32][8]
    float *box128;       // [Ns / 128][8]
    float *P;            // [block pairs][128][4]
    double *rec;         // [items][128][4]
    int64_t items_cap, pairs_cap;
    float gamma;
    uint32_t *status;
    // FP64 state in slot order for the whole call (contiguous kick, drift,
    // pack and fold): two buffers of 10 arrays [Ns] (x y z vx vy vz ax ay az m)
    // -- a re-sort permutes one into the other -- and the potential
    double *st[2];
    double *pots;
    int cur;
};

__device__ __forceinline__ double *st_arr(const BsParams &p, int b, int k) {
    return p.st[b] + (int64_t)k * p.Ns;
}

__device__ __forceinline__ int64_t bs_items_of_row(int64_t nblk, int64_t a) {
    return (nblk - a + BG - 1) / BG;
}

// Validation, padded layout, item list and its largest-first order (one
// block of 1024 threads; the systems' sizes are fixed for the whole call).
__global__ void __launch_bounds__(1024) bsym_setup_kernel(BsParams p, int64_t N) {
    __shared__ int64_t s_tot[4];
    __shared__ int32_t cnt[1024][BG];
    const int tid = threadIdx.x;
    if (tid == 0) {
        if (p.offsets[0] != 0 || p.offsets[p.B] != N) dev::set_status(p.status, kStatusInvalid);
        // prefix sums over systems (serial: once per call)
        int64_t sb = 0, ib = 0, pb = 0, blk = 0;
        for (int c = 0; c < p.B; ++c) {
            const int64_t n = p.offsets[c + 1] - p.offsets[c];
            const double e = p.eps[c];
            int64_t nblk = 0;
            if (n >= 1 && n <= kBsMaxN && e > 0.0 && isfinite(e))
                nblk = (n + BW - 1) / BW;
            else
                dev::set_status(p.status, kStatusInvalid);
            p.sbase[c] = sb;
            p.ibase[c] = ib;
            p.pbase[c] = pb;
            int64_t it = 0;
            for (int64_t a = 0; a < nblk; ++a) {
                p.rstart[blk + a] = (int32_t)(ib + it);
                p.bsys[blk + a] = c;
                it += bs_items_of_row(nblk, a);
            }
            sb += nblk * BW;
            ib += it;
            pb += nblk * (nblk - 1) / 2;
            blk += nblk;
        }
        p.sbase[p.B] = sb;
        p.ibase[p.B] = ib;
        p.pbase[p.B] = pb;
        p.rstart[blk] = (int32_t)ib;
        if (sb > p.Ns || ib > p.items_cap || pb > p.pairs_cap) {
            dev::set_status(p.status, kStatusInvalid);  // cannot happen: bounds of bsym_layout
            sb = ib = pb = blk = 0;
            p.sbase[p.B] = 0;
        }
        s_tot[0] = sb;
        s_tot[1] = ib;
        s_tot[2] = pb;
        s_tot[3] = blk;
        p.totals[0] = sb;
        p.totals[1] = ib;
        p.totals[2] = pb;
        p.totals[3] = blk;
        *p.counter = 0u;
    }
    __syncthreads();
    const int64_t nitems = s_tot[1];
    if (s_tot[0] == 0) return;
    // items, one system per thread
    for (int c = tid; c < p.B; c += blockDim.x) {
        const int64_t nblk = (p.sbase[c + 1] - p.sbase[c]) / BW;
        int64_t idx = p.ibase[c];
        for (int64_t a = 0; a < nblk; ++a)
            for (int64_t b0 = a; b0 < nblk; b0 += BG)
                p.items[idx++] = make_int4(c, (int)a, (int)b0, (int)(b0 + BG < nblk ? b0 + BG : nblk));
    }
    __syncthreads();
    // stable counting sort by size (j-blocks), largest first: per-thread
    // contiguous chunks, counts per size, exclusive prefix in (size desc,
    // thread) order
    const int64_t per = (nitems + 1023) / 1024;
    const int64_t lo = tid * per, hi = (lo + per) < nitems ? (lo + per) : nitems;
    for (int k = 0; k < BG; ++k) cnt[tid][k] = 0;
    for (int64_t i = lo; i < hi; ++i) {
        const int4 it = p.items[i];
        cnt[tid][it.w - it.z - 1] += 1;
    }
    __syncthreads();
    if (tid == 0) {
        int32_t run = 0;
        for (int k = BG - 1; k >= 0; --k)
            for (int t = 0; t < 1024; ++t) {
                const int32_t v = cnt[t][k];
                cnt[t][k] = run;
                run += v;
            }
    }
    __syncthreads();
    for (int64_t i = lo; i < hi; ++i) {
        const int4 it = p.items[i];
        p.order[cnt[tid][it.w - it.z - 1]++] = (int32_t)i;
    }
}

// Morton order of each system (one CTA per system): FP64 bounding box,
// 30-bit codes, keys code << 13 | source index, shared-memory bitonic sort;
// then the state is gathered into the other buffer in the new order: from
// the caller's arrays (from_user: particle order) or from the current
// slot-order buffer (a re-sort).  The real particles of a system always fill
// its first n slots; the padding slots hold zeros and perm = -1.
__global__ void __launch_bounds__(512) bsym_sort_kernel(BsParams p, int from_user) {
    extern __shared__ unsigned long long keys[];  // kBsMaxN keys, then kBsMaxN old perm entries
    int *old_perm = reinterpret_cast<int *>(keys + kBsMaxN);
    __shared__ double red[6][16];
    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t sb = p.sbase[c], ns = p.sbase[c + 1] - sb;
    if (ns == 0) return;
    const int64_t o0 = p.offsets[c];
    const int n = (int)(p.offsets[c + 1] - o0);
    const int src = p.cur, dst = 1 - p.cur;
    auto xsrc = [&](int e, int d) -> double {
        return from_user ? p.pos[3 * (o0 + e) + d] : st_arr(p, src, d)[sb + e];
    };
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int e = tid; e < n; e += blockDim.x)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = xsrc(e, d);
            lo[d] = fmin(lo[d], x);
            hi[d] = fmax(hi[d], x);
        }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    if (lane == 0)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            red[d][w] = lo[d];
            red[3 + d][w] = hi[d];
        }
    if (!from_user)
        for (int e = tid; e < n; e += blockDim.x) old_perm[e] = p.perm[sb + e];
    __syncthreads();
    double blo[3], scale[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double a = 1e308, b = -1e308;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) {
            a = fmin(a, red[d][k]);
            b = fmax(b, red[3 + d][k]);
        }
        blo[d] = a;
        scale[d] = b > a ? 1023.0 / (b - a) : 0.0;
    }
    int P2 = 1;
    while (P2 < n) P2 <<= 1;
    for (int e = tid; e < P2; e += blockDim.x) {
        unsigned long long k = ~0ull;
        if (e < n) {
            uint32_t code = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double q = (xsrc(e, d) - blo[d]) * scale[d];
                q = q < 0.0 ? 0.0 : (q > 1023.0 ? 1023.0 : q);
                uint32_t v = (uint32_t)q, r = 0;
#pragma unroll
                for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
                code |= r << d;
            }
            k = ((unsigned long long)code << 13) | (unsigned long long)e;
        }
        keys[e] = k;
    }
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = tid; e < P2; e += blockDim.x) {
                const int x = e ^ j;
                if (x > e) {
                    const bool asc = (e & k) == 0;
                    const unsigned long long a = keys[e], b = keys[x];
                    if ((a > b) == asc) {
                        keys[e] = b;
                        keys[x] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int64_t s = tid; s < ns; s += blockDim.x) {
        double v[10];
        int pi = -1;
        if (s < n) {
            const int e = (int)(keys[s] & 0x1fffull);
            if (from_user) {
                const int64_t i = o0 + e;
                pi = (int)i;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    v[d] = p.pos[3 * i + d];
                    v[3 + d] = p.vel ? p.vel[3 * i + d] : 0.0;
                    v[6 + d] = p.acc[3 * i + d];
                }
                v[9] = p.mass[i];
            } else {
                pi = old_perm[e];
#pragma unroll
                for (int k = 0; k < 10; ++k) v[k] = st_arr(p, src, k)[sb + e];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 10; ++k) v[k] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) st_arr(p, dst, k)[sb + s] = v[k];
        p.perm[sb + s] = pi;
    }
}

// End of a call: the slot-order state back to the caller's arrays.
__global__ void __launch_bounds__(256) bsym_scatter_kernel(BsParams p, int moved) {
    const int64_t ns = __ldg(p.totals);
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int i = p.perm[s];
        if (i < 0) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (moved) {
                p.pos[3 * (int64_t)i + d] = st_arr(p, p.cur, d)[s];
                p.vel[3 * (int64_t)i + d] = st_arr(p, p.cur, 3 + d)[s];
            }
            p.acc[3 * (int64_t)i + d] = st_arr(p, p.cur, 6 + d)[s];
        }
        if (p.pot) p.pot[i] = p.pots[s];
    }
}

// One block per 128-slot block: optional kick (v += kick a) and drift
// (x += dt v) of the block's particles (slot-order FP64 state), the hi/lo pack, and the
// boxes of its four 32-slot j-sets and of the whole block (real slots only).
__global__ void __launch_bounds__(BW) bsym_pack_kernel(BsParams p, double kick, double dt) {
    const int64_t s = (int64_t)blockIdx.x * BW + threadIdx.x;
    if ((int64_t)blockIdx.x * BW >= __ldg(p.totals)) return;  // whole block
    const int i = p.perm[s];
    float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f}, m = 0.f;
    if (i >= 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = st_arr(p, p.cur, d)[s];
            if (dt != 0.0) {
                const double v = st_arr(p, p.cur, 3 + d)[s] + kick * st_arr(p, p.cur, 6 + d)[s];
                x += dt * v;
                st_arr(p, p.cur, 3 + d)[s] = v;
                st_arr(p, p.cur, d)[s] = x;
            }
            hi[d] = __double2float_rn(x);
            lo[d] = __double2float_rn(x - (double)hi[d]);
        }
        m = __double2float_rn(st_arr(p, p.cur, 9)[s]);
    }
    store_packed(p.soa, p.Ns, s, hi, lo, m);
    // boxes
    float bl[3], bh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bl[d] = i >= 0 ? hi[d] : 3e38f;
        bh[d] = i >= 0 ? hi[d] : -3e38f;
        for (int o = 16; o > 0; o >>= 1) {
            bl[d] = fminf(bl[d], __shfl_xor_sync(0xffffffffu, bl[d], o));
            bh[d] = fmaxf(bh[d], __shfl_xor_sync(0xffffffffu, bh[d], o));
        }
    }
    __shared__ float wb[4][6];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        float amax = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.box32[(s / 32) * 8 + d] = bl[d];
            p.box32[(s / 32) * 8 + 3 + d] = bh[d];
            wb[w][d] = bl[d];
            wb[w][3 + d] = bh[d];
            amax = fmaxf(amax, fmaxf(fabsf(bl[d]), fabsf(bh[d])));
        }
        p.box32[(s / 32) * 8 + 6] = bh[0] < bl[0] ? 0.f : amax;
        p.box32[(s / 32) * 8 + 7] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float l3[3] = {3e38f, 3e38f, 3e38f}, h3[3] = {-3e38f, -3e38f, -3e38f}, amax = 0.f;
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                l3[d] = fminf(l3[d], wb[k][d]);
                h3[d] = fmaxf(h3[d], wb[k][3 + d]);
            }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.box128[blockIdx.x * 8 + d] = l3[d];
            p.box128[blockIdx.x * 8 + 3 + d] = h3[d];
            amax = fmaxf(amax, fmaxf(fabsf(l3[d]), fabsf(h3[d])));
        }
        p.box128[blockIdx.x * 8 + 6] = h3[0] < l3[0] ? 0.f : amax;
        p.box128[blockIdx.x * 8 + 7] = 0.f;
    }
}

// Persistent warps over the item queue.
template <int POL, int MODE>
__global__ void __launch_bounds__(NT, 1) bsym_item_kernel(BsParams p) {
    // per-warp i-side totals of the current item (FP64 policy: FP32 within
    // an item of <= 8 blocks, FP64 in the record and the fold)
    constexpr int IPOL = POL == NB_PREC_F64ACC ? NB_PREC_FP32 : POL;
    extern __shared__ __align__(16) unsigned char bs_smem[];
    auto tot = reinterpret_cast<Acc<IPOL>(*)[16][32]>(bs_smem);  // [NW][16][32]
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t nitems = __ldg(p.totals + 1);
    ISet S;
    while (true) {
        unsigned q0 = 0;
        if (l == 0) q0 = atomicAdd(p.counter, 1u);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if ((int64_t)q0 >= nitems) break;
        const int idx = __ldg(p.order + q0);
        const int4 it = p.items[idx];
        const int c = it.x, a = it.y, b0 = it.z, b1 = it.w;
        const int64_t sb = p.sbase[c];
        const int64_t ib = sb + (int64_t)BW * a;
        const float ef = (float)__ldg(p.eps + c);
        const float2 e2 = f2(ef * ef, ef * ef);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float v[2][7];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int d = 0; d < 7; ++d) v[h][d] = __ldg(p.soa + d * p.Ns + ib + 32 * (2 * g + h) + l);
            S.nx[g] = f2(-v[0][0], -v[1][0]);
            S.ny[g] = f2(-v[0][1], -v[1][1]);
            S.nz[g] = f2(-v[0][2], -v[1][2]);
            S.m[g] = f2(v[0][3], v[1][3]);
            S.nm[g] = f2(-v[0][3], -v[1][3]);
            S.nxl[g] = f2(-v[0][4], -v[1][4]);
            S.nyl[g] = f2(-v[0][5], -v[1][5]);
            S.nzl[g] = f2(-v[0][6], -v[1][6]);
            S.ax[g] = S.ay[g] = S.az[g] = S.ph[g] = f2(0.f, 0.f);
        }
#pragma unroll
        for (int v = 0; v < 16; ++v) tot[w][v][l].zero();
        const int nq = (b1 - b0) * 4;  // j-sets of the item (<= 32)
        unsigned near = 0u;
        if (MODE == 2) {
            float wbx[7], tb[7];
#pragma unroll
            for (int d = 0; d < 7; ++d) wbx[d] = __ldg(p.box128 + (ib / BW) * 8 + d);
            const int64_t js = (sb + (int64_t)BW * b0) / JS + (l < nq ? l : 0);
#pragma unroll
            for (int d = 0; d < 7; ++d) tb[d] = __ldg(p.box32 + js * 8 + d);
            near = __ballot_sync(0xffffffffu, l < nq && boxes_near(wbx, tb, p.gamma));
        }
        float jn[7];
        const int64_t jb0 = sb + (int64_t)BW * b0;
#pragma unroll
        for (int d = 0; d < 7; ++d) jn[d] = __ldg(p.soa + d * p.Ns + jb0 + l);
        for (int q = 0; q < nq; ++q) {
            float jc[7];
#pragma unroll
            for (int d = 0; d < 7; ++d) jc[d] = jn[d];
            if (q + 1 < nq)
#pragma unroll
                for (int d = 0; d < 7; ++d) jn[d] = __ldg(p.soa + d * p.Ns + jb0 + JS * (q + 1) + l);
            const int b = b0 + (q >> 2);
            const bool nqb = (near >> q) & 1u;
            float4 bs;
            if (b != a) {
                run_set<MODE, true>(S, e2, jc, nqb, bs, -1);
                const int64_t pair = p.pbase[c] + (int64_t)b * (b - 1) / 2 + a;
                __stcs(reinterpret_cast<float4 *>(p.P) + pair * BW + 32 * (q & 3) + l, bs);
            } else {
                run_set<MODE, false>(S, e2, jc, nqb, bs, q & 3);
            }
            if ((q & 3) == 3) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float2 v4[4] = {S.ax[g], S.ay[g], S.az[g], S.ph[g]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        tot[w][(2 * g) * 4 + e][l].add(v4[e].x);
                        tot[w][(2 * g + 1) * 4 + e][l].add(v4[e].y);
                    }
                    S.ax[g] = S.ay[g] = S.az[g] = S.ph[g] = f2(0.f, 0.f);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < IR; ++k) {
            double *r = p.rec + ((int64_t)idx * BW + 32 * k + l) * 4;
            __stcs(reinterpret_cast<double2 *>(r),
                   make_double2(tot[w][k * 4 + 0][l].value(), tot[w][k * 4 + 1][l].value()));
            __stcs(reinterpret_cast<double2 *>(r) + 1,
                   make_double2(tot[w][k * 4 + 2][l].value(), tot[w][k * 4 + 3][l].value()));
        }
    }
}

// Per slot: the records of its row and the partials of blocks a' < a (fixed
// order), x G, closing kick, store; resets the queue for the next step.
template <int POL>
__global__ void __launch_bounds__(256) bsym_fold_kernel(BsParams p, double kick) {
    const int64_t ns = __ldg(p.totals);
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.counter = 0u;
    uint32_t bad = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (p.perm[s] < 0) continue;
        const int64_t blk = s / BW, r = s % BW;
        const int c = p.bsys[blk];
        const int64_t a = blk - p.sbase[c] / BW;
        Acc<POL> acc4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc4[e].zero();
        for (int32_t it = p.rstart[blk]; it < p.rstart[blk + 1]; ++it) {
            const double2 *rr = reinterpret_cast<const double2 *>(p.rec + ((int64_t)it * BW + r) * 4);
            const double2 u = __ldcs(rr), v = __ldcs(rr + 1);
            add_record<POL>(acc4[0], u.x);
            add_record<POL>(acc4[1], u.y);
            add_record<POL>(acc4[2], v.x);
            add_record<POL>(acc4[3], v.y);
        }
        add_partials<POL>(acc4,
                          reinterpret_cast<const float4 *>(p.P) + (p.pbase[c] + a * (a - 1) / 2) * BW + r,
                          a, BW);
        const double ax = p.G * acc4[0].value(), ay = p.G * acc4[1].value(),
                     az = p.G * acc4[2].value();
        const double gp = -p.G * acc4[3].value();
        st_arr(p, p.cur, 6)[s] = ax;
        st_arr(p, p.cur, 7)[s] = ay;
        st_arr(p, p.cur, 8)[s] = az;
        if (kick != 0.0) {
            st_arr(p, p.cur, 3)[s] += kick * ax;
            st_arr(p, p.cur, 4)[s] += kick * ay;
            st_arr(p, p.cur, 5)[s] += kick * az;
        }
        p.pots[s] = gp;
        if (!(isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(gp))) bad = 1;
    }
    if (bad) dev::set_status(p.status, kStatusNonFinite);
}

template <int POL, int MODE>
int launch_bsym_steps(BsParams p, const BatchedJob &j, int64_t nb_max) {
    const cudaStream_t st = j.stream;
    const unsigned pack_grid = (unsigned)nb_max;
    const unsigned fold_grid = (unsigned)std::min<int64_t>(cdiv(nb_max * BW, 256), 64 * (int64_t)device_sm_count());
    const unsigned item_grid = (unsigned)device_sm_count();
    constexpr int sort_smem = 12 * kBsMaxN;  // keys and the old permutation
    static const cudaError_t optin = cudaFuncSetAttribute(
        bsym_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sort_smem);
    NB_CUDA(optin);
    p.cur = 0;
    auto sort = [&](int from_user) {
        bsym_sort_kernel<<<(unsigned)p.B, 512, sort_smem, st>>>(p, from_user);
        p.cur ^= 1;
        count_launch();
    };
    constexpr int IPOL = POL == NB_PREC_F64ACC ? NB_PREC_FP32 : POL;
    const size_t item_smem = (size_t)NW * 16 * 32 * sizeof(Acc<IPOL>);
    static const cudaError_t optin_item = cudaFuncSetAttribute(
        bsym_item_kernel<POL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)item_smem);
    NB_CUDA(optin_item);
    auto force = [&](double kick) {
        bsym_item_kernel<POL, MODE><<<item_grid, NT, item_smem, st>>>(p);
        bsym_fold_kernel<POL><<<fold_grid, 256, 0, st>>>(p, kick);
        count_launch(2);
    };
    bsym_setup_kernel<<<1, 1024, 0, st>>>(p, j.N);
    count_launch();
    sort(1);
    if (!j.acc_valid || j.nsteps == 0) {
        bsym_pack_kernel<<<pack_grid, BW, 0, st>>>(p, 0.0, 0.0);
        count_launch();
        force(0.0);
    }
    for (int64_t n = 0; n < j.nsteps; ++n) {
        if (n > 0 && n % kBsResort == 0) sort(0);
        bsym_pack_kernel<<<pack_grid, BW, 0, st>>>(p, 0.5 * j.dt, j.dt);
        count_launch();
        force(0.5 * j.dt);
    }
    bsym_scatter_kernel<<<fold_grid, 256, 0, st>>>(p, j.nsteps > 0 ? 1 : 0);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int POL>
int launch_bsym_pol(BsParams p, const BatchedJob &j, int mode, int64_t nb_max) {
    switch (mode) {
        case 0: return launch_bsym_steps<POL, 0>(p, j, nb_max);
        case 1: return launch_bsym_steps<POL, 1>(p, j, nb_max);
        default: return launch_bsym_steps<POL, 2>(p, j, nb_max);
    }
}

}  // namespace

SymSizes sym_sizes(int64_t Np) {
    SymSizes z{};
    z.nb = cdiv(Np, kSymBlock);
    z.T = z.nb * (z.nb + 1) / 2;
    z.U = z.T * US;
    z.ctas = std::min<int64_t>(device_sm_count(), z.U);
    // Records per row: a cost-balanced range holds at least
    // (U / ctas) * (min unit cost / max unit cost) - 2 units, so a row of
    // nb * US units meets at most that many ranges plus 2; with short ranges
    // (empty ones possible) every CTA gets a slot.
    const double min_len =
        (double)z.U / (double)z.ctas * (double)kUnitCostMin / (double)kUnitCostMax - 2.0;
    int64_t K = z.ctas;
    if (min_len >= 1.0)
        K = std::min<int64_t>(z.ctas, (int64_t)std::ceil((double)(z.nb * US) / min_len) + 2);
    z.K = K;
    z.p_bytes = (size_t)(z.nb * (z.nb - 1) / 2) * kSymBlock * 16;
    z.rec_bytes = (size_t)z.nb * (size_t)K * kSymBlock * 32;
    z.cost_bytes = align_up(4 * (size_t)z.T, 256) + align_up(8 * (size_t)(z.T + 1), 256) +
                   8 * (size_t)(z.ctas + 1);
    return z;
}

int launch_force_sym(const ForceJob &j, bool adaptive) {
    if (j.eps <= 0.0) return fail(NB_ERR_UNSUPPORTED, "symmetric pairs need eps > 0");
    if (j.L.sym_rec_bytes == 0)
        return fail(NB_ERR_WORKSPACE, "workspace has no symmetric-pair buffers");
    const SymSizes z = sym_sizes(j.L.Np);
    SymParams p;
    char *sb = j.ws + j.L.sortbuf;
    p.soa = reinterpret_cast<const float *>(j.ws + j.L.packA);
    p.Np = j.L.Np;
    p.nb = z.nb;
    p.T = z.T;
    p.U = z.U;
    p.ctas = z.ctas;
    p.K = z.K;
    const float ef = (float)j.eps;
    p.eps2 = ef * ef;
    p.gamma = j.gamma;
    p.jbox = adaptive ? sort_tile_boxes(sb, j.L) : nullptr;
    p.wbox = adaptive ? sort_block_boxes(sb, j.L) : nullptr;
    p.P = reinterpret_cast<float *>(j.ws + j.L.sym_p);
    p.rec = reinterpret_cast<double *>(j.ws + j.L.sym_rec);
    p.lo = reinterpret_cast<const int64_t *>(j.ws + j.L.sym_cost + align_up(4 * (size_t)z.T, 256) +
                                             align_up(8 * (size_t)(z.T + 1), 256));
    const int *perm = adaptive ? sort_perm(sb, j.L) : nullptr;
    uint32_t *status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    p.status = status;
    const int mode = adaptive ? 2 : (j.split ? 1 : 0);
    switch (j.precision) {
        case NB_PREC_FP32: return launch_sym_pol<NB_PREC_FP32>(p, j, mode, perm, status);
        case NB_PREC_KAHAN: return launch_sym_pol<NB_PREC_KAHAN>(p, j, mode, perm, status);
        case NB_PREC_F64ACC: return launch_sym_pol<NB_PREC_F64ACC>(p, j, mode, perm, status);
    }
    return fail(NB_ERR_UNSUPPORTED, "symmetric pairs compute FP32 pairs (FP32, KAHAN, F64ACC)");
}


// ------------------------------------------------------------ batched host
BsymLayout bsym_layout(int64_t N, int32_t B) {
    BsymLayout z{};
    z.Ns = round_up(N + (int64_t)BW * B, BW);
    z.blocks = z.Ns / BW;
    z.items = 6 * z.blocks;                 // per system <= nblk (1 + 65 / 16) items
    z.pairs = (int64_t)(BW / 2) * z.blocks;  // per system nblk (nblk - 1) / 2 <= 32 nblk
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    z.o_sbase = take(8 * (size_t)(B + 1));
    z.o_ibase = take(8 * (size_t)(B + 1));
    z.o_pbase = take(8 * (size_t)(B + 1));
    z.o_rstart = take(4 * (size_t)(z.blocks + 1));
    z.o_bsys = take(4 * (size_t)z.blocks);
    z.o_items = take(16 * (size_t)z.items);
    z.o_order = take(4 * (size_t)z.items);
    z.o_misc = take(256);  // counter, totals
    z.o_soa = take(4 * (size_t)kPackArrays * z.Ns);
    z.o_perm = take(4 * (size_t)z.Ns);
    z.o_box32 = take(32 * (size_t)(z.Ns / 32));
    z.o_box128 = take(32 * (size_t)z.blocks);
    z.o_P = take(16 * (size_t)BW * z.pairs);
    z.o_rec = take(32 * (size_t)BW * z.items);
    z.o_st0 = take(80 * (size_t)z.Ns);
    z.o_st1 = take(80 * (size_t)z.Ns);
    z.o_pots = take(8 * (size_t)z.Ns);
    z.bytes = off;
    return z;
}

int launch_batched_sym(const BatchedJob &j) {
    if (j.L.bsym_bytes == 0) return fail(NB_ERR_WORKSPACE, "workspace has no batched symmetric buffers");
    const BsymLayout z = bsym_layout(j.N, j.B);
    char *base = j.ws + j.L.bsym;
    BsParams p;
    p.B = j.B;
    p.offsets = j.offsets;
    p.eps = j.eps;
    p.G = j.G;
    p.mass = j.mass;
    p.pos = j.pos;
    p.vel = j.vel;
    p.acc = j.acc;
    p.pot = j.pot;
    p.sbase = reinterpret_cast<int64_t *>(base + z.o_sbase);
    p.ibase = reinterpret_cast<int64_t *>(base + z.o_ibase);
    p.pbase = reinterpret_cast<int64_t *>(base + z.o_pbase);
    p.rstart = reinterpret_cast<int32_t *>(base + z.o_rstart);
    p.bsys = reinterpret_cast<int32_t *>(base + z.o_bsys);
    p.items = reinterpret_cast<int4 *>(base + z.o_items);
    p.order = reinterpret_cast<int32_t *>(base + z.o_order);
    p.counter = reinterpret_cast<unsigned *>(base + z.o_misc);
    p.totals = reinterpret_cast<int64_t *>(base + z.o_misc + 64);
    p.soa = reinterpret_cast<float *>(base + z.o_soa);
    p.Ns = z.Ns;
    p.perm = reinterpret_cast<int *>(base + z.o_perm);
    p.box32 = reinterpret_cast<float *>(base + z.o_box32);
    p.box128 = reinterpret_cast<float *>(base + z.o_box128);
    p.P = reinterpret_cast<float *>(base + z.o_P);
    p.rec = reinterpret_cast<double *>(base + z.o_rec);
    p.st[0] = reinterpret_cast<double *>(base + z.o_st0);
    p.st[1] = reinterpret_cast<double *>(base + z.o_st1);
    p.pots = reinterpret_cast<double *>(base + z.o_pots);
    p.cur = 0;
    p.items_cap = z.items;
    p.pairs_cap = z.pairs;
    p.gamma = j.gamma > 0.f ? j.gamma : kNearFarGamma;
    p.status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    const int mode = j.positions == NB_POS_SPLIT ? 1 : (j.positions == NB_POS_SINGLE ? 0 : 2);
    switch (j.precision) {
        case NB_PREC_FP32: return launch_bsym_pol<NB_PREC_FP32>(p, j, mode, z.blocks);
        case NB_PREC_KAHAN: return launch_bsym_pol<NB_PREC_KAHAN>(p, j, mode, z.blocks);
        case NB_PREC_F64ACC: return launch_bsym_pol<NB_PREC_F64ACC>(p, j, mode, z.blocks);
    }
    return fail(NB_ERR_UNSUPPORTED, "symmetric pairs compute FP32 pairs (FP32, KAHAN, F64ACC)");
}

}  // namespace nb
