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
// Hilbert order a particle's strongest, mutually cancelling terms (its
// spatial neighbours) arrive together; with 16 j-sets per flush the FP32
// running sums of central particles of a log-normal Plummer sphere
// (N = 300001, eps = 1e-3) lost up to 1e-5 of |a|, with 4 they stay at the
// 2e-6 of the unsorted order.  A second kernel adds, slot by
// slot in a fixed order, the records of the row's CTAs and the partials
// P[I', I] for I' < I, applies G, scatters through the Hilbert permutation
// and optionally kicks the velocity.  Every
// sum runs in a fixed order: results are bitwise reproducible.
//
// Displacements: single floats, hi/lo pairs (x_j.hi - x_i.hi) +
// (x_j.lo - x_i.lo), or adaptive: per (warp i-set, j-set) the hi/lo form
// only when the bounding boxes are closer than gamma * max|x| (a 64-bit
// mask per warp and item, from the Hilbert-sorted pack's boxes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "nb_device.cuh"
#include "nb_internal.h"
#include "nb_sym_core.cuh"

namespace nb {

using dev::Acc;
using dev::add2;
using dev::f2;
using dev::fma2;
using dev::mul2;
using dev::rsqrt_approx;

namespace {

using namespace symcore;

constexpr int SW = 16;              // warps per CTA of the pair kernel
constexpr int SNT = SW * 32;        // threads per CTA
constexpr int CPS = 1;              // resident CTAs per SM
constexpr int BI = SW * 32 * IR;    // slots per row block
constexpr int NJS = BI / JS;        // j-sets per block
constexpr int KB = 4;               // j-sets per cross-warp reduction
constexpr int FL = 4;               // j-sets per i-side flush of the register sums
constexpr int FL2 = 16;             // F64ACC: j-sets per flush of the FP32 middle sums
constexpr int US = NJS / KB;        // stream-K units (KB j-sets) per item
static_assert(BI == kSymBlock, "row block size");
static_assert(NJS % KB == 0 && NJS % FL2 == 0 && FL2 % FL == 0, "groups tile a block");
constexpr size_t kRedBytes = 2 * KB * SW * 32 * sizeof(float4);

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

// FP64 pairs: the common layout plus positions [N][3] and masses in
// particle order and FP64 partials.
struct SymParams64 : SymParams {
    const double *pos64, *mass64;
    int64_t N;
    double eps2_64;
    double *P64;        // [nb (nb - 1) / 2][BI][4]
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

__device__ __forceinline__ void load_j(const SymParams &p, int64_t s, float (&j)[7]) {
#pragma unroll
    for (int a = 0; a < 7; ++a) j[a] = __ldg(p.soa + a * p.Np + s);
}

// MODE: 0 single-float displacement, 1 hi/lo, 2 adaptive.  POT: the
// potential sums too (the caller wants phi).
template <int POL, int MODE, bool POT>
__global__ void __launch_bounds__(SNT, CPS) force_sym_kernel(const SymParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *red = reinterpret_cast<float4 *>(smem);                   // [2][KB][SW][32]
    Acc<POL> *tot = reinterpret_cast<Acc<POL> *>(smem + kRedBytes);   // [16][SNT]
    constexpr bool MID = POL == NB_PREC_F64ACC;
    float *mid = reinterpret_cast<float *>(smem + kRedBytes + 16 * SNT * sizeof(Acc<POL>));
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
                tot[v * SNT + tid].zero();
                if (MID) mid[v * SNT + tid] = 0.f;
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
            static_assert(NJS == 32 || NJS == 64, "one or two 32-bit ballots per block");
#pragma unroll
            for (int h = 0; h < NJS / 32; ++h) {
                float tb[7];
#pragma unroll
                for (int a = 0; a < 7; ++a) tb[a] = __ldg(p.jbox + (jb / JS + l + 32 * h) * 8 + a);
                const unsigned m = __ballot_sync(0xffffffffu, boxes_near(wb, tb, p.gamma));
                near |= (unsigned long long)m << (32 * h);
            }
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
                run_set<MODE, true, POT>(S, e2, jc, nq, b, -1);
                red[((half * KB + (q % KB)) * SW + w) * 32 + l] = b;
            } else {
                run_set<MODE, false, POT>(S, e2, jc, nq, b, (q >> 2) == w ? (q & 3) : -1);
            }
            if ((q + 1) % FL == 0 || q + 1 == qb) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float2 v4[4] = {S.ax[g], S.ay[g], S.az[g], S.ph[g]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int v0 = ((2 * g) * 4 + e) * SNT + tid;
                        const int v1 = ((2 * g + 1) * 4 + e) * SNT + tid;
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
                        tot[v * SNT + tid].add(mid[v * SNT + tid]);
                        mid[v * SNT + tid] = 0.f;
                    }
                }
            }
            if (sym && (q + 1) % KB == 0) {
                __syncthreads();
                for (int v = tid; v < KB * JS * 4; v += SNT) {
                    const int qq = v >> 7, ll = (v >> 2) & 31, e = v & 3;
                    const float *r = reinterpret_cast<const float *>(red) +
                                     ((half * KB + qq) * SW * 32 + ll) * 4 + e;
                    float s = 0.f;
#pragma unroll
                    for (int w2 = 0; w2 < SW; ++w2) s += r[w2 * 32 * 4];
                    // streaming store: the partials are read once, by the fold, and
                    // must not evict the packed positions every CTA re-reads from L2
                    __stcs(p.P + ((pidx * BI) + (q + 1 - KB + qq) * JS + ll) * 4 + e, s);
                }
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
                       make_double2(tot[(kk * 4 + 0) * SNT + tid].value(),
                                    tot[(kk * 4 + 1) * SNT + tid].value()));
                __stcs(reinterpret_cast<double2 *>(r) + 1,
                       make_double2(tot[(kk * 4 + 2) * SNT + tid].value(),
                                    tot[(kk * 4 + 3) * SNT + tid].value()));
            }
            row_open = false;
        }
        if (qb == NJS && ++J == p.nb) {
            ++I;
            J = I;
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
        const int64_t pidx = J * (J - 1) / 2 + I;
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
                    __stcs(p.P64 + ((pidx * BI) + (q + 1 - KB + qq) * JS + ll) * 4 + e, sum);
                }
                half ^= 1;
            }
        }
        u = seg_end;
        if ((J == p.nb - 1 && qb == NJS) || u == u_end) {
            const int64_t k = c - range_owner(p.lo, p.ctas, row_start(I, p.nb) * US);
            if (k >= p.K && tid == 0) dev::set_status(p.status, kStatusInvalid);
#pragma unroll
            for (int kk = 0; kk < IR; ++kk) {
                if (k >= p.K) break;
                double *r = p.rec + (((I * p.K + k) * BI) + w * 128 + 32 * kk + l) * 4;
                __stcs(reinterpret_cast<double2 *>(r), make_double2(S.ax[kk], S.ay[kk]));
                __stcs(reinterpret_cast<double2 *>(r) + 1, make_double2(S.az[kk], S.ph[kk]));
            }
            row_open = false;
        }
        if (qb == NJS && ++J == p.nb) {
            ++I;
            J = I;
        }
    }
}

__global__ void __launch_bounds__(256) sym_fold64_kernel(const SymParams64 p, double G,
                                                         double *__restrict__ acc,
                                                         double *__restrict__ pot,
                                                         double *__restrict__ vel, double kick,
                                                         uint32_t *status) {
    uint32_t bad = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < p.N;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = s / BI, r = s % BI;
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        const int64_t rs = row_start(I, p.nb);
        const int64_t c0 = range_owner(p.lo, p.ctas, rs * US);
        const int64_t c1 = range_owner(p.lo, p.ctas, (rs + (p.nb - I)) * US - 1);
        for (int64_t k = 0; k <= c1 - c0 && k < p.K; ++k) {
            if (__ldg(p.lo + c0 + k) == __ldg(p.lo + c0 + k + 1)) continue;  // empty range
            const double2 *rr = reinterpret_cast<const double2 *>(p.rec + (((I * p.K + k) * BI) + r) * 4);
            const double2 u = __ldg(rr), v = __ldg(rr + 1);
            a[0] += u.x;
            a[1] += u.y;
            a[2] += v.x;
            a[3] += v.y;
        }
        const D4 *P4 = reinterpret_cast<const D4 *>(p.P64) + (I * (I - 1) / 2) * BI + r;
        for (int64_t i2 = 0; i2 < I; ++i2) {
            const D4 v = P4[i2 * BI];
            a[0] += v.x;
            a[1] += v.y;
            a[2] += v.z;
            a[3] += v.w;
        }
        const double ax = G * a[0], ay = G * a[1], az = G * a[2], gp = -G * a[3];
        acc[3 * s] = ax;
        acc[3 * s + 1] = ay;
        acc[3 * s + 2] = az;
        if (vel) {
            vel[3 * s] += kick * ax;
            vel[3 * s + 1] += kick * ay;
            vel[3 * s + 2] += kick * az;
        }
        if (pot) pot[s] = gp;
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
constexpr uint32_t kUnitCostMin = KB * SW * kCostDiagFar;
constexpr uint32_t kUnitCostMax = KB * SW * kCostSymNear;

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
        c = (MODE == 1 ? cn : cf) * (NJS / 32) * SW;  // this lane's j-sets x the block's warps
    } else {
        constexpr int H = NJS / 32;  // j-sets of the block per lane
        float tb[H][7];
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
            for (int a = 0; a < 7; ++a) tb[h][a] = __ldg(p.jbox + (J * BI / JS + l + 32 * h) * 8 + a);
        for (int w = 0; w < SW; ++w) {
            float wb[7];
#pragma unroll
            for (int a = 0; a < 7; ++a) wb[a] = __ldg(p.wbox + ((I * BI + w * 128) / 128) * 8 + a);
#pragma unroll
            for (int h = 0; h < H; ++h) c += boxes_near(wb, tb[h], p.gamma) ? cn : cf;
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

template <int POL, int MODE, bool POT>
int launch_pair(const SymParams &p, cudaStream_t st) {
    auto kern = force_sym_kernel<POL, MODE, POT>;
    const size_t smem = kRedBytes + 16 * SNT * sizeof(Acc<POL>) +
                        (POL == NB_PREC_F64ACC ? 16 * SNT * sizeof(float) : 0);
    const int rc = smem_optin(reinterpret_cast<const void *>(kern), smem);
    if (rc != NB_OK) return rc;
    kernel_timer_begin(st);
    kern<<<(unsigned)p.ctas, SNT, smem, st>>>(p);
    kernel_timer_end(st);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
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
    const int rc_pair = j.pot ? launch_pair<POL, MODE, true>(p, j.stream)
                              : launch_pair<POL, MODE, false>(p, j.stream);
    if (rc_pair != NB_OK) return rc_pair;
    const int64_t fold_blocks = std::min<int64_t>(cdiv(j.N, 256), 64 * (int64_t)device_sm_count());
    sym_fold_kernel<POL><<<(unsigned)fold_blocks, 256, 0, j.stream>>>(
        p, j.N, perm, j.G, j.acc, j.pot, j.vel, j.kick, status);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
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

int launch_sym64(const SymParams64 &p, const ForceJob &j, uint32_t *status) {
    uint32_t *cost = reinterpret_cast<uint32_t *>(j.ws + j.L.sym_cost);
    unsigned long long *prefix = reinterpret_cast<unsigned long long *>(
        j.ws + j.L.sym_cost + align_up(4 * (size_t)p.T, 256));
    int64_t *lo = const_cast<int64_t *>(p.lo);
    sym_cost_kernel<0><<<(unsigned)cdiv(p.T * 32, 256), 256, 0, j.stream>>>(p, cost);
    sym_scan_kernel<<<1, 1024, 0, j.stream>>>(cost, p.T, prefix);
    sym_ranges_kernel<<<(unsigned)cdiv(p.ctas + 1, 256), 256, 0, j.stream>>>(cost, prefix, p.T,
                                                                             p.ctas, lo);
    count_launch(3);
    NB_CUDA(cudaGetLastError());
    const int rc = j.pot ? launch_pair64<true>(p, j.stream) : launch_pair64<false>(p, j.stream);
    if (rc != NB_OK) return rc;
    const int64_t fold_blocks = std::min<int64_t>(cdiv(j.N, 256), 64 * (int64_t)device_sm_count());
    sym_fold64_kernel<<<(unsigned)fold_blocks, 256, 0, j.stream>>>(p, j.G, j.acc, j.pot, j.vel,
                                                                   j.kick, status);
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

}  // namespace

SymSizes sym_sizes(int64_t Np) {
    SymSizes z{};
    z.nb = cdiv(Np, kSymBlock);
    z.T = z.nb * (z.nb + 1) / 2;
    z.U = z.T * US;
    z.ctas = std::min<int64_t>(CPS * (int64_t)device_sm_count(), z.U);
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
    if (j.precision == NB_PREC_FP64) {
        SymParams64 p64;
        static_cast<SymParams &>(p64) = p;
        p64.pos64 = j.pos;
        p64.mass64 = j.mass;
        p64.N = j.N;
        p64.eps2_64 = j.eps * j.eps;
        p64.P64 = reinterpret_cast<double *>(j.ws + j.L.sym_p);
        return launch_sym64(p64, j, status);
    }
    switch (j.precision) {
        case NB_PREC_FP32: return launch_sym_pol<NB_PREC_FP32>(p, j, mode, perm, status);
        case NB_PREC_KAHAN: return launch_sym_pol<NB_PREC_KAHAN>(p, j, mode, perm, status);
        case NB_PREC_F64ACC: return launch_sym_pol<NB_PREC_F64ACC>(p, j, mode, perm, status);
    }
    return fail(NB_ERR_INVALID, "unknown precision %d", j.precision);
}

}  // namespace nb
