// Many independent N-body clusters of uneven size in one persistent launch
// (the SPMD split of Sec. 3.1 applied to whole systems: each unit of work is
// an independent set of particles).
//
// The grid is a set of thread-block clusters of CS CTAs (hardware cluster
// barriers: every CTA of a cluster is co-resident, so there is no software
// spin-wait).  Each thread-block cluster pops N-body clusters from a queue
// ordered largest first (atomic counter; the order comes from a one-block
// bitonic sort of the sizes) and runs every leapfrog step of that system
// before taking the next.
//
// A system's particles are visited in Hilbert order: CTA 0 sorts them (FP64
// bounding box, 30-bit codes, shared-memory bitonic sort) when the system
// starts and every 16 steps; slot s of the order holds particle perm[s], and
// CTA r owns a 64-aligned range of slots.
//
//   per step, each CTA for its own slots:
//     v += (dt/2) a;  x += dt v;  pack x (hi/lo FP32) and m      (FP64 state)
//     bounding box of every owned 64-slot chunk
//     cluster barrier
//     a, phi of its slots against all slots of the system; v += (dt/2) a
//
// The packed positions and boxes are double-buffered (one barrier per step).
// j-tiles (and their 8 chunk boxes) are read through L2 (ld.global.cg: other
// CTAs of the cluster wrote them) into shared memory, the next tile
// prefetched into registers during the current one.  Each thread keeps 2
// consecutive slots in registers, so a warp's i-particles are a compact run
// of the Hilbert curve; per j-chunk of 64 slots a warp takes the single-float
// displacement when the chunk's box is at least gamma * max|x| away from the
// warp's box (rounding error of x_j - x_i at most 2^-24 max|x| per
// coordinate, so relative error <= 2^-24 / gamma), else the hi/lo one.  When
// a slice has fewer than two particles per thread, groups of L = 2..32 lanes
// share the same i-particles, split the j-pairs, and are summed with a fixed
// xor-shuffle tree (bitwise reproducible).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <mutex>

#include "nb_device.cuh"
#include "nb_order.cuh"
#include "nb_internal.h"

namespace cg = cooperative_groups;

namespace nb {

using dev::Acc;
using dev::f2;
using dev::pair2;

constexpr int kBTJ = 512;      // j-particles per shared-memory tile
constexpr int kBMaxN = 8192;   // particles per cluster (device-checked)
constexpr int kBSortMax = 8192;
constexpr int kBMaxSlots = 4096;

constexpr int kBMaxClusters = 320;  // resident thread-block clusters served
constexpr int kBChunk = 64;         // slots per box
constexpr int kBResort = 16;        // steps between Hilbert re-sorts of a system
constexpr size_t kBPermBytes = 4 * (size_t)kBMaxClusters * kBMaxN;
constexpr size_t kBBoxBytes = 4 * (size_t)kBMaxClusters * 2 * (kBMaxN / kBChunk) * 8;

size_t batched_scratch_bytes(int32_t B) {
    return 4 * (size_t)(B > 0 ? B : 1) + 4 * (size_t)kBMaxSlots + 256 + kBPermBytes + kBBoxBytes;
}

struct BatchedParams {
    const double *mass;
    const int64_t *offsets;
    int32_t B;
    int64_t N;
    const double *eps;
    double G;
    double *pos;
    double *vel;
    double *acc;
    double *pot;
    double dt;
    int64_t nsteps;
    int acc_valid;
    float *pack0;  // [7][Np]
    float *pack1;  // [7][Np]
    int64_t Np;
    const int *order;
    unsigned *counter;
    int *slots;
    uint32_t *status;
    // Hilbert order per thread-block cluster (adaptive displacement)
    int *perm;          // [clusters][kBMaxN]: sorted slot -> local particle index
    float *boxes;       // [clusters][2][kBMaxN / 64][8]: per 64-slot chunk boxes
    float gamma;        // far iff box gap >= gamma * max|x|; < 0: split everywhere
};

// ---------------------------------------------------------------- setup
// Resets the queue counter, validates the CSR layout and orders clusters by
// size, largest first (ties by index), with a shared-memory bitonic sort.
__global__ void batched_setup_kernel(const int64_t *__restrict__ offsets, int B, int64_t N,
                                     const double *__restrict__ eps, int *order,
                                     unsigned *counter, uint32_t *status) {
    extern __shared__ unsigned long long keys[];
    const int tid = threadIdx.x;
    if (tid == 0) {
        *counter = 0u;
        if (offsets[0] != 0 || offsets[B] != N) dev::set_status(status, kStatusInvalid);
    }
    for (int c = tid; c < B; c += blockDim.x) {
        const int64_t n = offsets[c + 1] - offsets[c];
        const double e = eps[c];
        if (n < 1 || n > kBMaxN || !(e > 0.0) || !isfinite(e))
            dev::set_status(status, kStatusInvalid);
    }
    if (B > kBSortMax) {
        for (int c = tid; c < B; c += blockDim.x) order[c] = c;
        return;
    }
    int P = 1;
    while (P < B) P <<= 1;
    for (int e = tid; e < P; e += blockDim.x) {
        unsigned long long k = ~0ull;
        if (e < B) {
            int64_t n = offsets[e + 1] - offsets[e];
            n = n < 0 ? 0 : (n > kBMaxN ? kBMaxN : n);
            k = ((unsigned long long)(kBMaxN - n) << 32) | (unsigned)e;
        }
        keys[e] = k;
    }
    __syncthreads();
    dev::block_bitonic_sort(keys, P);
    for (int c = tid; c < B; c += blockDim.x) order[c] = (int)(keys[c] & 0xffffffffu);
}

// ---------------------------------------------------------------- pieces
// Slots of a system are its particles in Hilbert order; CTA r of the cluster
// owns the 64-aligned slot range [slot_lo(r), slot_lo(r+1)), so every box
// chunk of 64 slots has exactly one owner.
template <int CS>
__device__ __forceinline__ int64_t slot_lo(int64_t n, int r) {
    const int64_t a = ((n * r / CS) + kBChunk - 1) / kBChunk * kBChunk;
    return a < n ? a : n;
}

// Hilbert order of the system's n particles (one CTA): FP64 bounding box,
// 30-bit codes, keys code << 13 | local index (unique), shared-memory
// bitonic sort, perm[slot] = local index.
template <int BT>
__device__ void sort_system(const BatchedParams &p, int64_t o0, int n, int *perm,
                            unsigned long long *keys) {
    __shared__ double red[6][32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int e = tid; e < n; e += BT)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double x = p.pos[3 * (o0 + e) + c];
            lo[c] = fmin(lo[c], x);
            hi[c] = fmax(hi[c], x);
        }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            red[c][w] = lo[c];
            red[3 + c][w] = hi[c];
        }
    __syncthreads();
    double blo[3], scale[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double a = 1e308, b = -1e308;
        for (int k = 0; k < BT / 32; ++k) {
            a = fmin(a, red[c][k]);
            b = fmax(b, red[3 + c][k]);
        }
        blo[c] = a;
        scale[c] = b > a ? 1023.0 / (b - a) : 0.0;
    }
    int P = 1;
    while (P < n) P <<= 1;
    for (int e = tid; e < P; e += BT) {
        unsigned long long k = ~0ull;
        if (e < n) {
            const uint32_t code = dev::hilbert30(dev::cell10(p.pos[3 * (o0 + e)], blo[0], scale[0]),
                                  dev::cell10(p.pos[3 * (o0 + e) + 1], blo[1], scale[1]),
                                  dev::cell10(p.pos[3 * (o0 + e) + 2], blo[2], scale[2]));
            k = ((unsigned long long)code << 13) | (unsigned long long)e;
        }
        keys[e] = k;
    }
    __syncthreads();
    dev::block_bitonic_sort(keys, P);
    for (int e = tid; e < n; e += BT) perm[e] = (int)(keys[e] & 0x1fffull);
}

// Own slots: optional kick + drift of the particle in each slot (FP64 state),
// split pack in slot order, then one box per owned 64-slot chunk.
template <int BT>
__device__ __forceinline__ void pack_slots(const BatchedParams &p, int64_t o0, int64_t a0,
                                           int64_t a1, const int *perm, float *pk, float *bx,
                                           bool kick_drift) {
    const double half = 0.5 * p.dt;
    for (int64_t s = a0 + threadIdx.x; s < a1; s += BT) {
        const int64_t i = o0 + perm[s];
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double x = p.pos[3 * i + c];
            if (kick_drift) {
                const double v = p.vel[3 * i + c] + half * p.acc[3 * i + c];
                x += p.dt * v;
                p.vel[3 * i + c] = v;
                p.pos[3 * i + c] = x;
            }
            hi[c] = __double2float_rn(x);
            lo[c] = __double2float_rn(x - (double)hi[c]);
        }
        store_packed(pk, p.Np, o0 + s, hi, lo, __double2float_rn(p.mass[i]));
    }
    __syncthreads();
    // boxes: warp per chunk, two slots per lane
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t ch = a0 / kBChunk + w; ch * kBChunk < a1; ch += BT / 32) {
        float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
        for (int64_t s = ch * kBChunk + lane; s < (ch + 1) * kBChunk && s < a1; s += 32)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float x = pk[c * p.Np + o0 + s];
                lo[c] = fminf(lo[c], x);
                hi[c] = fmaxf(hi[c], x);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
                hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
            }
        if (lane == 0) {
            float amax = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bx[ch * 8 + c] = lo[c];
                bx[ch * 8 + 3 + c] = hi[c];
                amax = fmaxf(amax, fmaxf(fabsf(lo[c]), fabsf(hi[c])));
            }
            bx[ch * 8 + 6] = amax;
            bx[ch * 8 + 7] = 0.f;
        }
    }
}

__device__ __forceinline__ bool near_boxes(const float *wb, const float *tb, float gamma) {
    float g2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gap = fmaxf(0.f, fmaxf(tb[c] - wb[3 + c], wb[c] - tb[3 + c]));
        g2 = fmaf(gap, gap, g2);
    }
    const float X = gamma * fmaxf(wb[6], tb[6]);
    return g2 < X * X;
}

// Forces on the slots of one chunk of the CTA's range [.., a1) from all
// slots of the system [0, n).  BT threads form G = BT / L groups of L lanes;
// group g holds the 2 consecutive slots c0 + 2g, c0 + 2g + 1 (so a warp's
// i-particles are contiguous in Hilbert order) and its lanes split the
// j-quads of every 64-slot chunk.  Per (warp, 64-slot j-chunk) the warp
// takes the single-float displacement when the boxes are well separated.
template <int BT, int POL>
__device__ __forceinline__ void force_chunk(const BatchedParams &p, int64_t o0, int64_t n,
                                            int64_t c0, int64_t a1, const int *perm,
                                            const float *pk, const float *bx, float eps2,
                                            double kick, int L, float (&tile)[7][kBTJ],
                                            float (&tbox)[kBTJ / kBChunk * 8]) {
    constexpr int IR = 2;
    constexpr int NCH = kBTJ / kBChunk;  // box chunks per j-tile
    constexpr int PER = 7 * kBTJ / BT;  // tile floats each thread stages
    static_assert(7 * kBTJ % BT == 0, "tile must split evenly over the CTA");
    const int tid = threadIdx.x;
    const int lane = tid % L;
    const int grp = tid / L;
    float2 nx[IR], ny[IR], nz[IR], nxl[IR], nyl[IR], nzl[IR];
    int64_t sl[IR];
    Acc<POL> tot[IR][4];
    float wlo[3] = {3e38f, 3e38f, 3e38f}, whi[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        sl[k] = c0 + 2 * grp + k;
        const bool live = sl[k] < a1;
        const int64_t i = o0 + (live ? sl[k] : 0);
        const float x = __ldcg(pk + i), y = __ldcg(pk + p.Np + i), z = __ldcg(pk + 2 * p.Np + i);
        const float xl = __ldcg(pk + 4 * p.Np + i), yl = __ldcg(pk + 5 * p.Np + i),
                    zl = __ldcg(pk + 6 * p.Np + i);
        if (live) {
            wlo[0] = fminf(wlo[0], x); whi[0] = fmaxf(whi[0], x);
            wlo[1] = fminf(wlo[1], y); whi[1] = fmaxf(whi[1], y);
            wlo[2] = fminf(wlo[2], z); whi[2] = fmaxf(whi[2], z);
        }
        nx[k] = f2(-x, -x);
        ny[k] = f2(-y, -y);
        nz[k] = f2(-z, -z);
        nxl[k] = f2(-xl, -xl);
        nyl[k] = f2(-yl, -yl);
        nzl[k] = f2(-zl, -zl);
#pragma unroll
        for (int e = 0; e < 4; ++e) tot[k][e].zero();
    }
    // this warp's i-box (the near/far test is warp-uniform), kept in shared memory
    __shared__ float s_wb[BT / 32][8];
    float *wb = s_wb[tid >> 5];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            wlo[c] = fminf(wlo[c], __shfl_xor_sync(0xffffffffu, wlo[c], o));
            whi[c] = fmaxf(whi[c], __shfl_xor_sync(0xffffffffu, whi[c], o));
        }
    if ((tid & 31) == 0) {
        float amax = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            wb[c] = wlo[c];
            wb[3 + c] = whi[c];
            amax = fmaxf(amax, fmaxf(fabsf(wlo[c]), fabsf(whi[c])));
        }
        wb[6] = whi[0] < wlo[0] ? 0.f : amax;  // no live slot in this warp: never near
    }
    __syncwarp();
    const float2 e2 = f2(eps2, eps2);
    float pre[PER], preb = 0.f;
    auto fetch = [&](int64_t t0) {
        const int64_t nj = (n - t0) < kBTJ ? (n - t0) : kBTJ;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * BT;
            const int arr = e / kBTJ, jj = e % kBTJ;
            pre[r] = jj < nj ? __ldcg(pk + arr * p.Np + o0 + t0 + jj) : 0.f;
        }
        // boxes of the tile's chunks (those past the system's end are never tested)
        if (tid < NCH * 8 && (int64_t)(tid / 8) * kBChunk < nj)
            preb = __ldcg(bx + (t0 / kBChunk) * 8 + tid);
    };
    fetch(0);
    for (int64_t t0 = 0; t0 < n; t0 += kBTJ) {
        const int nj = (int)((n - t0) < kBTJ ? (n - t0) : kBTJ);
        __syncthreads();  // the previous tile is no longer read
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * BT;
            tile[e / kBTJ][e % kBTJ] = pre[r];
        }
        if (tid < NCH * 8) tbox[tid] = preb;
        __syncthreads();
        if (t0 + kBTJ < n) fetch(t0 + kBTJ);  // in flight during the pairs below
        float2 ax[IR], ay[IR], az[IR], ph[IR];
#pragma unroll
        for (int k = 0; k < IR; ++k) ax[k] = ay[k] = az[k] = ph[k] = f2(0.f, 0.f);
        const int nquads = (nj + 3) / 4;  // a ragged tail reads the zero-mass pad
        // a tile that holds one of this warp's i-slots has self pairs: those
        // quads give the pair j == i a zero mass (exact j != i)
        bool own = false;
#pragma unroll
        for (int k = 0; k < IR; ++k) own |= sl[k] >= t0 && sl[k] < t0 + nj;
        const bool diag = __any_sync(0xffffffffu, own);
        auto quad = [&](int jq, bool split) {
            const float4 X = *reinterpret_cast<const float4 *>(&tile[0][4 * jq]);
            const float4 Y = *reinterpret_cast<const float4 *>(&tile[1][4 * jq]);
            const float4 Z = *reinterpret_cast<const float4 *>(&tile[2][4 * jq]);
            const float4 M = *reinterpret_cast<const float4 *>(&tile[3][4 * jq]);
            if (diag) {
                int kr[IR];
#pragma unroll
                for (int k = 0; k < IR; ++k) kr[k] = (int)(sl[k] - t0) - 4 * jq;
                const float4 XL = *reinterpret_cast<const float4 *>(&tile[4][4 * jq]);
                const float4 YL = *reinterpret_cast<const float4 *>(&tile[5][4 * jq]);
                const float4 ZL = *reinterpret_cast<const float4 *>(&tile[6][4 * jq]);
                pair2<IR, false, true, true>(f2(X.x, X.y), f2(Y.x, Y.y), f2(Z.x, Z.y),
                                             f2(XL.x, XL.y), f2(YL.x, YL.y), f2(ZL.x, ZL.y),
                                             f2(M.x, M.y), e2, nx, ny, nz, nxl, nyl, nzl, ax, ay,
                                             az, ph, kr, 0);
                pair2<IR, false, true, true>(f2(X.z, X.w), f2(Y.z, Y.w), f2(Z.z, Z.w),
                                             f2(XL.z, XL.w), f2(YL.z, YL.w), f2(ZL.z, ZL.w),
                                             f2(M.z, M.w), e2, nx, ny, nz, nxl, nyl, nzl, ax, ay,
                                             az, ph, kr, 2);
            } else if (split) {
                const float4 XL = *reinterpret_cast<const float4 *>(&tile[4][4 * jq]);
                const float4 YL = *reinterpret_cast<const float4 *>(&tile[5][4 * jq]);
                const float4 ZL = *reinterpret_cast<const float4 *>(&tile[6][4 * jq]);
                pair2<IR, false, true>(f2(X.x, X.y), f2(Y.x, Y.y), f2(Z.x, Z.y), f2(XL.x, XL.y),
                                       f2(YL.x, YL.y), f2(ZL.x, ZL.y), f2(M.x, M.y), e2, nx, ny,
                                       nz, nxl, nyl, nzl, ax, ay, az, ph);
                pair2<IR, false, true>(f2(X.z, X.w), f2(Y.z, Y.w), f2(Z.z, Z.w), f2(XL.z, XL.w),
                                       f2(YL.z, YL.w), f2(ZL.z, ZL.w), f2(M.z, M.w), e2, nx, ny,
                                       nz, nxl, nyl, nzl, ax, ay, az, ph);
            } else {
                const float2 zz = f2(0.f, 0.f);
                pair2<IR, false, false>(f2(X.x, X.y), f2(Y.x, Y.y), f2(Z.x, Z.y), zz, zz, zz,
                                        f2(M.x, M.y), e2, nx, ny, nz, nxl, nyl, nzl, ax, ay, az,
                                        ph);
                pair2<IR, false, false>(f2(X.z, X.w), f2(Y.z, Y.w), f2(Z.z, Z.w), zz, zz, zz,
                                        f2(M.z, M.w), e2, nx, ny, nz, nxl, nyl, nzl, ax, ay, az,
                                        ph);
            }
        };
        // near/far per 64-slot j-chunk of this tile against this warp's box
        constexpr int QC = kBChunk / 4;  // quads per chunk
        const int nch = (nquads + QC - 1) / QC;
        const unsigned all = (1u << nch) - 1u;
        unsigned near = all;
        if (p.gamma >= 0.f) {
            near = 0u;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                if (c < nch && near_boxes(wb, &tbox[8 * c], p.gamma)) near |= 1u << c;
        }
        if (L == 1) {
            if (near == all) {
#pragma unroll 2
                for (int jq = 0; jq < nquads; ++jq) quad(jq, true);
            } else if (near == 0u) {
#pragma unroll 2
                for (int jq = 0; jq < nquads; ++jq) quad(jq, false);
            } else {
#pragma unroll 1
                for (int c = 0; c < nch; ++c) {
                    const int q1 = (c + 1) * QC < nquads ? (c + 1) * QC : nquads;
                    if ((near >> c) & 1u) {
#pragma unroll 2
                        for (int jq = c * QC; jq < q1; ++jq) quad(jq, true);
                    } else {
#pragma unroll 2
                        for (int jq = c * QC; jq < q1; ++jq) quad(jq, false);
                    }
                }
            }
        } else {
            for (int jq = lane; jq < nquads; jq += L) quad(jq, (near >> (jq / QC)) & 1u);
        }
#pragma unroll
        for (int k = 0; k < IR; ++k) {
            tot[k][0].add(ax[k].x + ax[k].y);
            tot[k][1].add(ay[k].x + ay[k].y);
            tot[k][2].add(az[k].x + az[k].y);
            tot[k][3].add(ph[k].x + ph[k].y);
        }
    }
    double v[IR][4];
#pragma unroll
    for (int k = 0; k < IR; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) v[k][e] = tot[k][e].value();
    // lanes sharing a group: fixed butterfly over offsets L/2, L/4, ..., 1
    for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < IR; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) v[k][e] += __shfl_xor_sync(0xffffffffu, v[k][e], o);
    if (lane != 0) return;
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        if (sl[k] >= a1) continue;
        const int64_t i = o0 + perm[sl[k]];
        const double phs = v[k][3];
        const double a[3] = {p.G * v[k][0], p.G * v[k][1], p.G * v[k][2]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p.acc[3 * i + c] = a[c];
            if (kick != 0.0) p.vel[3 * i + c] += kick * a[c];
        }
        const double gp = -p.G * phs;
        if (p.pot) p.pot[i] = gp;
        if (!(isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]) && isfinite(gp))) bad = 1;
    }
    if (bad) dev::set_status(p.status, kStatusNonFinite);
}

// Two i-particles per group and as many lanes per group as the CTA's slot
// range leaves room for, so small ranges still fill the CTA.
template <int BT, int POL>
__device__ __forceinline__ void force_slots(const BatchedParams &p, int64_t o0, int64_t n,
                                            int64_t a0, int64_t a1, const int *perm,
                                            const float *pk, const float *bx, float eps2,
                                            double kick, float (&tile)[7][kBTJ],
                                            float (&tbox)[kBTJ / kBChunk * 8]) {
    const int64_t ns = a1 - a0;
    const int64_t groups = (ns + 1) / 2 > 0 ? (ns + 1) / 2 : 1;
    int L = 1;
    while (L < 32 && (int64_t)(2 * L) * groups <= BT) L <<= 1;
    const int64_t chunk = (int64_t)(BT / L) * 2;
    for (int64_t c0 = a0; c0 < a1; c0 += chunk)
        force_chunk<BT, POL>(p, o0, n, c0, a1, perm, pk, bx, eps2, kick, L, tile, tbox);
    // the epilogue's acc/vel writes (lane 0 of each group) are read by other
    // threads of this CTA in the next kick-drift-pack
    __syncthreads();
}

template <int CS, int BT, int POL>
__global__ void __launch_bounds__(BT, 1) batched_kernel(const BatchedParams p) {
    __shared__ __align__(16) float tile[7][kBTJ];
    __shared__ float tbox[kBTJ / kBChunk * 8];
    extern __shared__ unsigned long long sort_keys_smem[];  // kBMaxN keys, CTA rank 0 only
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int g = blockIdx.x / CS;
    int *perm = p.perm + (int64_t)g * kBMaxN;
    float *boxes = p.boxes + (int64_t)g * 2 * (kBMaxN / kBChunk) * 8;
    while (true) {
        if (r == 0 && threadIdx.x == 0) p.slots[g] = (int)atomicAdd(p.counter, 1u);
        cl.sync();
        const int q = __ldcg(&p.slots[g]);
        if (q >= p.B) break;
        const int c = p.order[q];
        const int64_t o0 = p.offsets[c], o1 = p.offsets[c + 1];
        const int64_t n = o1 - o0;
        const double epsd = p.eps[c];
        const bool valid = n >= 1 && n <= kBMaxN && epsd > 0.0 && isfinite(epsd) && o0 >= 0 &&
                           o1 <= p.N;
        if (valid) {
            const int64_t a0 = slot_lo<CS>(n, r), a1 = slot_lo<CS>(n, r + 1);
            const float ef = (float)epsd;
            const float eps2 = ef * ef;
            int buf = 0;
            float *bx[2] = {boxes, boxes + (kBMaxN / kBChunk) * 8};
            auto resort = [&]() {
                if (r == 0) sort_system<BT>(p, o0, (int)n, perm, sort_keys_smem);
                cl.sync();
            };
            resort();
            if (!p.acc_valid) {
                pack_slots<BT>(p, o0, a0, a1, perm, p.pack0, bx[0], false);
                cl.sync();
                force_slots<BT, POL>(p, o0, n, a0, a1, perm, p.pack0, bx[0], eps2, 0.0, tile, tbox);
            }
            for (int64_t step = 0; step < p.nsteps; ++step) {
                if (step > 0 && step % kBResort == 0) {
                    cl.sync();  // every CTA is done reading perm for the last step
                    resort();
                }
                buf ^= 1;
                float *pk = buf ? p.pack1 : p.pack0;
                pack_slots<BT>(p, o0, a0, a1, perm, pk, bx[buf], true);
                cl.sync();
                force_slots<BT, POL>(p, o0, n, a0, a1, perm, pk, bx[buf], eps2, 0.5 * p.dt, tile, tbox);
            }
        }
        cl.sync();
    }
}

// ---------------------------------------------------------------- launch
template <int CS, int BT, int POL>
static int launch_batched_cs(const BatchedParams &p, cudaStream_t st) {
    auto kern = batched_kernel<CS, BT, POL>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(BT, 1, 1);
    cfg.dynamicSmemBytes = 8 * kBMaxN;  // Hilbert keys of one system
    {
        const int rc = smem_optin(reinterpret_cast<const void *>(kern), 8 * (size_t)kBMaxN);
        if (rc != NB_OK) return rc;
    }
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters = -1;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (max_clusters < 0) {
            cfg.gridDim = dim3(CS * 1024, 1, 1);
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
                cudaGetLastError();
                n = device_sm_count() / CS;
            }
            max_clusters = n < 1 ? 1 : n;
        }
    }
    int nclusters = max_clusters;
    if (nclusters > p.B) nclusters = p.B;
    if (nclusters > kBMaxClusters) nclusters = kBMaxClusters;
    cfg.gridDim = dim3(CS * nclusters, 1, 1);
    NB_CUDA(cudaLaunchKernelEx(&cfg, kern, p));
    count_launch();
    return NB_OK;
}

template <int POL>
static int launch_batched_pol(const BatchedParams &p, int cs, int bt, cudaStream_t st) {
    switch (cs * 10000 + bt) {
        case 2 * 10000 + 256: return launch_batched_cs<2, 256, POL>(p, st);
        case 4 * 10000 + 256: return launch_batched_cs<4, 256, POL>(p, st);
        case 8 * 10000 + 256: return launch_batched_cs<8, 256, POL>(p, st);
        case 2 * 10000 + 512: return launch_batched_cs<2, 512, POL>(p, st);
        case 4 * 10000 + 512: return launch_batched_cs<4, 512, POL>(p, st);
        case 8 * 10000 + 512: return launch_batched_cs<8, 512, POL>(p, st);
    }
    return fail(NB_ERR_UNSUPPORTED,
                "batched shape (%d CTAs per cluster, %d threads) not compiled (2/4/8 x 256/512)",
                cs, bt);
}

int launch_batched(const BatchedJob &j) {
    if (j.precision == NB_PREC_FP64)
        return fail(NB_ERR_UNSUPPORTED, "the batched path computes FP32 pairs (FP32, KAHAN, F64ACC)");
    if (j.sym) return launch_batched_sym(j);
    if (j.B > kBMaxSlots * 1024) return fail(NB_ERR_UNSUPPORTED, "too many clusters");
    BatchedParams p;
    p.mass = j.mass;
    p.offsets = j.offsets;
    p.B = j.B;
    p.N = j.N;
    p.eps = j.eps;
    p.G = j.G;
    p.pos = j.pos;
    p.vel = j.vel;
    p.acc = j.acc;
    p.pot = j.pot;
    p.dt = j.dt;
    p.nsteps = j.nsteps;
    p.acc_valid = j.acc_valid ? 1 : 0;
    p.Np = j.L.Np;
    p.pack0 = reinterpret_cast<float *>(j.ws + j.L.packA);
    p.pack1 = p.pack0 + (size_t)kPackArrays * j.L.Np;
    char *scr = j.ws + j.L.scratch + 64 * 1024;
    p.order = reinterpret_cast<int *>(scr);
    p.slots = reinterpret_cast<int *>(scr + 4 * (size_t)j.B);
    p.counter = reinterpret_cast<unsigned *>(scr + 4 * (size_t)j.B + 4 * (size_t)kBMaxSlots);
    char *scr2 = scr + 4 * (size_t)j.B + 4 * (size_t)kBMaxSlots + 256;
    p.perm = reinterpret_cast<int *>(scr2);
    p.boxes = reinterpret_cast<float *>(scr2 + kBPermBytes);
    p.gamma = j.positions == NB_POS_SPLIT ? -1.f : (j.gamma > 0.f ? j.gamma : kNearFarGamma);
    p.status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    {
        int P = 1;
        while (P < j.B && P < kBSortMax) P <<= 1;
        const size_t smem = j.B <= kBSortMax ? (size_t)P * 8 : 0;
        const int rc = smem_optin(reinterpret_cast<const void *>(batched_setup_kernel),
                                  (size_t)kBSortMax * 8);
        if (rc != NB_OK) return rc;
        batched_setup_kernel<<<1, 1024, smem, j.stream>>>(j.offsets, j.B, j.N, j.eps,
                                                          const_cast<int *>(p.order), p.counter,
                                                          p.status);
        count_launch();
        NB_CUDA(cudaGetLastError());
    }
    const int cs = j.cluster > 0 ? j.cluster : 4;  // measured best on GB300 (4 x 256 threads)
    const int bt = j.threads > 0 ? j.threads : 256;
    switch (j.precision) {
        case NB_PREC_FP32: return launch_batched_pol<NB_PREC_FP32>(p, cs, bt, j.stream);
        case NB_PREC_KAHAN: return launch_batched_pol<NB_PREC_KAHAN>(p, cs, bt, j.stream);
        case NB_PREC_F64ACC: return launch_batched_pol<NB_PREC_F64ACC>(p, cs, bt, j.stream);
    }
    return fail(NB_ERR_INVALID, "unknown precision %d", j.precision);
}

}  // namespace nb
