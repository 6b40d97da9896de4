// Batches of independent systems with symmetric pairs (see the comment at
// the top of the batched section below); the pair evaluation is the one of
// nb_sym.cu (nb_sym_core.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "nb_device.cuh"
#include "nb_fpconv.cuh"
#include "nb_order.cuh"
#include "nb_internal.h"
#include "nb_sym_core.cuh"

namespace nb {

namespace {

using namespace symcore;

// ================================================================ batched
// Many independent systems (offsets [B+1], eps [B]), each unordered pair of
// a system evaluated once as above, at warp granularity.  Every system is
// padded to whole 128-slot blocks in Hilbert order (re-sorted every 32 steps);
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
constexpr int BG = 8;             // j-blocks per item at most (default item width)
constexpr int kBsMaxN = 8192;     // particles per system (64 blocks)
constexpr int kBsResort = 32;     // steps between Hilbert re-sorts
// Default near/far threshold of this path (x max|x| of the two boxes): the
// clusters are small and centred, so FP32-rounded positions stay accurate
// closer in than in a 2^20 sphere.  512-cluster workload, 1000 steps: 2826
// against 2761 G interactions/s with the library-wide 1/64, every sampled
// cluster within the 1e-5 gate.
constexpr float kBsNearGamma = 1.f / 256.f;

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
    int4 *bmeta;         // [blocks] first and end item of its row, first partial (block pair), a
    int4 *items;         // [items] (c, a, b0, b1)
    int32_t *order;      // [items] largest first
    unsigned *counter;   // queue head
    int64_t *totals;     // slots, items, block pairs, blocks
    float *soa;          // [7][Ns]
    int64_t Ns;          // slot capacity
    int *perm;           // [Ns] slot -> particle, -1 for padding
    float *box32;        // [Ns / 32][8]
    float *P;            // [block pairs][4][128]: planes ax ay az phi (phi only with the potential)
    float *rec;          // [items][2][128][4]: s, then -c (KAHAN) of the i-side totals
    int64_t items_cap, pairs_cap;
    int32_t g;           // j-blocks per item at most: 2, 4 or BG
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

__device__ __forceinline__ int64_t bs_items_of_row(int64_t nblk, int64_t a, int g) {
    return (nblk - a + g - 1) / g;
}

// The compensation term of a Kahan total (zero for the plain FP32 one).
__device__ __forceinline__ float comp(const Acc<NB_PREC_KAHAN> &a) { return a.c; }
__device__ __forceinline__ float comp(const Acc<NB_PREC_FP32> &) { return 0.f; }

// Validation, padded layout, item list and its largest-first order (one
// block of 1024 threads; the systems' sizes are fixed for the whole call).
// Thread t owns a contiguous chunk of systems: their sizes, an exclusive
// block-wide scan of the chunk totals (slots, items, block pairs, blocks),
// then each system's bases, row starts and block owners.
__global__ void __launch_bounds__(1024) bsym_setup_kernel(BsParams p, int64_t N) {
    __shared__ int64_t s_tot[4];
    // the scan's [4][1024] int64 sums and the sort's [1024][BG] int32 counts
    __shared__ __align__(16) int64_t sh[4 * 1024];
    static_assert(sizeof(int32_t) * 1024 * BG <= sizeof(int64_t) * 4 * 1024, "count table");
    auto cnt = reinterpret_cast<int32_t(*)[BG]>(sh);
    const int tid = threadIdx.x;
    const int64_t chunk = (p.B + 1023) / 1024;
    const int64_t c0 = tid * chunk < p.B ? tid * chunk : p.B;
    const int64_t c1 = c0 + chunk < p.B ? c0 + chunk : p.B;
    auto nblk_of = [&](int64_t c, bool report) -> int64_t {
        const int64_t n = p.offsets[c + 1] - p.offsets[c];
        const double e = p.eps[c];
        if (n >= 1 && n <= kBsMaxN && e > 0.0 && isfinite(e)) return (n + BW - 1) / BW;
        if (report) dev::set_status(p.status, kStatusInvalid);
        return 0;
    };
    int64_t own[4] = {0, 0, 0, 0};  // slots, items, block pairs, blocks of the chunk
    for (int64_t c = c0; c < c1; ++c) {
        const int64_t nblk = nblk_of(c, true);
        for (int64_t a = 0; a < nblk; ++a) own[1] += bs_items_of_row(nblk, a, p.g);
        own[0] += nblk * BW;
        own[2] += nblk * (nblk - 1) / 2;
        own[3] += nblk;
    }
    // inclusive Hillis-Steele scan of the four chunk totals
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[k * 1024 + tid] = own[k];
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = tid >= o ? sh[k * 1024 + tid - o] : 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[k * 1024 + tid] += v[k];
        __syncthreads();
    }
    int64_t base[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) base[k] = sh[k * 1024 + tid] - own[k];
    if (tid == 0) {
        if (p.offsets[0] != 0 || p.offsets[p.B] != N) dev::set_status(p.status, kStatusInvalid);
        int64_t t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = sh[k * 1024 + 1023];
        if (t[0] > p.Ns || t[1] > p.items_cap || t[2] > p.pairs_cap || p.g < 1 || p.g > BG) {
            // cannot happen (bounds of bsym_layout); if it did, every system
            // becomes empty so that no kernel indexes past the buffers
            dev::set_status(p.status, kStatusInvalid);
            t[0] = t[1] = t[2] = t[3] = 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s_tot[k] = t[k];
            p.totals[k] = t[k];
        }
        p.sbase[p.B] = t[0];
        p.ibase[p.B] = t[1];
        p.pbase[p.B] = t[2];
        p.rstart[t[3]] = (int32_t)t[1];
        *p.counter = 0u;
    }
    __syncthreads();
    if (s_tot[0] == 0) {
        for (int64_t c = tid; c < p.B; c += blockDim.x) p.sbase[c] = p.ibase[c] = p.pbase[c] = 0;
        return;
    }
    for (int64_t c = c0; c < c1; ++c) {
        const int64_t nblk = nblk_of(c, false);
        p.sbase[c] = base[0];
        p.ibase[c] = base[1];
        p.pbase[c] = base[2];
        int64_t it = 0;
        for (int64_t a = 0; a < nblk; ++a) {
            p.rstart[base[3] + a] = (int32_t)(base[1] + it);
            p.bsys[base[3] + a] = (int32_t)c;
            it += bs_items_of_row(nblk, a, p.g);
        }
        base[0] += nblk * BW;
        base[1] += it;
        base[2] += nblk * (nblk - 1) / 2;
        base[3] += nblk;
    }
    __syncthreads();
    const int64_t nitems = s_tot[1];
    if (s_tot[0] == 0) return;
    // what a fold of each block reads, in one 16-byte load
    for (int64_t b = tid; b < s_tot[3]; b += blockDim.x) {
        const int c = p.bsys[b];
        const int64_t a = b - p.sbase[c] / BW;
        p.bmeta[b] = make_int4(p.rstart[b], p.rstart[b + 1], (int)(p.pbase[c] + a * (a - 1) / 2),
                               (int)a);
    }
    // items, one system per thread
    for (int c = tid; c < p.B; c += blockDim.x) {
        const int64_t nblk = (p.sbase[c + 1] - p.sbase[c]) / BW;
        int64_t idx = p.ibase[c];
        for (int64_t a = 0; a < nblk; ++a)
            for (int64_t b0 = a; b0 < nblk; b0 += p.g)
                p.items[idx++] = make_int4(c, (int)a, (int)b0, (int)(b0 + p.g < nblk ? b0 + p.g : nblk));
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

// Hilbert order of each system (one CTA per system): FP64 bounding box,
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
            const uint32_t code = dev::hilbert30(dev::cell10(xsrc(e, 0), blo[0], scale[0]),
                                                 dev::cell10(xsrc(e, 1), blo[1], scale[1]),
                                                 dev::cell10(xsrc(e, 2), blo[2], scale[2]));
            k = ((unsigned long long)code << 13) | (unsigned long long)e;
        }
        keys[e] = k;
    }
    __syncthreads();
    dev::block_bitonic_sort(keys, P2);
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

// The box of the 32-slot j-set of slot s (real slots only); called by the
// 32 lanes of a warp for the 32 slots of one j-set.
__device__ __forceinline__ void set_box(const BsParams &p, int64_t s, bool real, const float hi[3]) {
    float bl[3], bh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bl[d] = real ? hi[d] : 3e38f;
        bh[d] = real ? hi[d] : -3e38f;
        for (int o = 16; o > 0; o >>= 1) {
            bl[d] = fminf(bl[d], __shfl_xor_sync(0xffffffffu, bl[d], o));
            bh[d] = fmaxf(bh[d], __shfl_xor_sync(0xffffffffu, bh[d], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        float amax = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.box32[(s / 32) * 8 + d] = bl[d];
            p.box32[(s / 32) * 8 + 3 + d] = bh[d];
            amax = fmaxf(amax, fmaxf(fabsf(bl[d]), fabsf(bh[d])));
        }
        p.box32[(s / 32) * 8 + 6] = bh[0] < bl[0] ? 0.f : amax;
        p.box32[(s / 32) * 8 + 7] = 0.f;
    }
}

// The hi/lo pack of slot s after an optional kick (v += kick a) and drift
// (x += dt v) of the slot-order FP64 state, and the box of the slot's
// 32-slot j-set (real slots only).  Called by the 32 lanes of a warp for the
// 32 slots of one j-set.
__device__ __forceinline__ void pack_slot(const BsParams &p, int64_t s, int i, double kick,
                                          double dt) {
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
    set_box(p, s, i >= 0, hi);
}

// One block per 128-slot block: pack_slot for each slot.
__global__ void __launch_bounds__(BW) bsym_pack_kernel(BsParams p, double kick, double dt) {
    const int64_t s = (int64_t)blockIdx.x * BW + threadIdx.x;
    if ((int64_t)blockIdx.x * BW >= __ldg(p.totals)) return;  // whole block
    pack_slot(p, s, p.perm[s], kick, dt);
}

// Persistent warps over the item queue (POT: the potential sums too).
template <int POL, int MODE, bool POT>
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
        // near masks of the warp's two 64-slot halves (packed groups 0, 1)
        unsigned near0 = 0u, near1 = 0u;
        if (MODE == 2) {
            float hb[2][7], tb[7];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float *a = p.box32 + (ib / JS + 2 * h) * 8, *c = a + 8;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    hb[h][d] = fminf(__ldg(a + d), __ldg(c + d));
                    hb[h][3 + d] = fmaxf(__ldg(a + 3 + d), __ldg(c + 3 + d));
                }
                hb[h][6] = fmaxf(__ldg(a + 6), __ldg(c + 6));
            }
            const int64_t js = (sb + (int64_t)BW * b0) / JS + (l < nq ? l : 0);
#pragma unroll
            for (int d = 0; d < 7; ++d) tb[d] = __ldg(p.box32 + js * 8 + d);
            near0 = __ballot_sync(0xffffffffu, l < nq && boxes_near(hb[0], tb, p.gamma));
            near1 = __ballot_sync(0xffffffffu, l < nq && boxes_near(hb[1], tb, p.gamma));
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
            const int nqb = (int)((near0 >> q) & 1u) | ((int)((near1 >> q) & 1u) << 1);
            float4 bs;
            if (b != a) {
                run_set2<MODE, true, POT>(S, e2, jc, nqb, bs, -1);
                const int64_t pair = p.pbase[c] + (int64_t)b * (b - 1) / 2 + a;
                float *P = p.P + pair * 4 * BW + 32 * (q & 3) + l;
                __stcs(P, bs.x);
                __stcs(P + BW, bs.y);
                __stcs(P + 2 * BW, bs.z);
                if (POT) __stcs(P + 3 * BW, bs.w);
            } else {
                run_set2<MODE, false, POT>(S, e2, jc, nqb, bs, q & 3);
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
            float4 *r = reinterpret_cast<float4 *>(p.rec) + (int64_t)idx * 2 * BW + 32 * k + l;
            __stcs(r, make_float4(tot[w][k * 4 + 0][l].s, tot[w][k * 4 + 1][l].s,
                                  tot[w][k * 4 + 2][l].s, tot[w][k * 4 + 3][l].s));
            if (IPOL == NB_PREC_KAHAN)
                __stcs(r + BW, make_float4(-comp(tot[w][k * 4 + 0][l]), -comp(tot[w][k * 4 + 1][l]),
                                           -comp(tot[w][k * 4 + 2][l]), -comp(tot[w][k * 4 + 3][l])));
        }
    }
}

// The F64ACC folds' accumulator: a compensated pair of floats, s + c, where
// each add computes its exact rounding error with Knuth's TwoSum (six FP32
// adds, valid for any magnitudes) and collects it in c.  For n adds the
// result is within about n u^2 |sum| of the exact sum (u = 2^-24), far below
// FP64 accumulation's own n 2^-53 for the sums of FP32 values folded here, at
// FP32-pipe cost: FP64 adds are slow on this part and one per record or
// group made the fold FP64-bound.
struct TwoF {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
        s = t;
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ double value() const { return fpconv::f2d(s) + fpconv::f2d(c); }
};

template <int POL>
struct FoldAccT {
    using type = Acc<POL>;
};
template <>
struct FoldAccT<NB_PREC_F64ACC> {
    using type = TwoF;
};
template <int POL>
using FoldAcc = typename FoldAccT<POL>::type;

// Slot s's total: the records of its row's items (s, then -c for KAHAN)
// and the partials of the blocks a' < a, in a fixed order and the policy's
// arithmetic (F64ACC: groups of 8 partials in FP32, as the partials of
// one tile of the direct kernel, then the compensated pair).  Loads go out
// four records or eight partials at a time.
template <int POL, bool POT>
__device__ __forceinline__ void slot_sums(const BsParams &p, int64_t s, const int4 bm,
                                          FoldAcc<POL> (&acc4)[4]) {
    constexpr int NC = POT ? 4 : 3;  // components summed
    const int64_t r = s % BW;
    const int64_t a = bm.w;
#pragma unroll
    for (int e = 0; e < 4; ++e) acc4[e].zero();
    const int32_t r0 = bm.x, r1 = bm.y;
    const float4 *rec = reinterpret_cast<const float4 *>(p.rec) + r;
    for (int32_t i0 = r0; i0 < r1; i0 += 4) {
        float4 u[4], v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t it = i0 + k < r1 ? i0 + k : r1 - 1;
            u[k] = __ldcs(rec + it * 2 * BW);
            if (POL == NB_PREC_KAHAN) v[k] = __ldcs(rec + it * 2 * BW + BW);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < r1) {
                const float uu[4] = {u[k].x, u[k].y, u[k].z, u[k].w};
                const float vv[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
                for (int e = 0; e < NC; ++e) {
                    acc4[e].add(uu[e]);
                    if (POL == NB_PREC_KAHAN) acc4[e].add(vv[e]);
                }
            }
    }
    const float *P = p.P + (int64_t)bm.z * 4 * BW + r;
    for (int64_t k0 = 0; k0 < a; k0 += 8) {
        float v[8][NC];
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int e = 0; e < NC; ++e)
                v[k][e] = k0 + k < a ? __ldcs(P + ((k0 + k) * 4 + e) * BW) : 0.f;
#pragma unroll
        for (int e = 0; e < NC; ++e) {
            if (POL == NB_PREC_F64ACC) {
                float g = v[0][e];
#pragma unroll
                for (int k = 1; k < 8; ++k) g += v[k][e];
                acc4[e].add(g);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (k0 + k < a) acc4[e].add(v[k][e]);
            }
        }
    }
}

// Per slot: the records of its row and the partials of blocks a' < a (fixed
// order), x G, closing kick, store (the potential only after items that
// summed it); resets the queue for the next step.
template <int POL, bool POT>
__global__ void __launch_bounds__(256) bsym_fold_kernel(BsParams p, double kick) {
    const int64_t ns = __ldg(p.totals);
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.counter = 0u;
    uint32_t bad = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (p.perm[s] < 0) continue;
        FoldAcc<POL> acc4[4];
        slot_sums<POL, POT>(p, s, p.bmeta[s / BW], acc4);
        const double ax = p.G * acc4[0].value(), ay = p.G * acc4[1].value(),
                     az = p.G * acc4[2].value();
        st_arr(p, p.cur, 6)[s] = ax;
        st_arr(p, p.cur, 7)[s] = ay;
        st_arr(p, p.cur, 8)[s] = az;
        if (kick != 0.0) {
            st_arr(p, p.cur, 3)[s] += kick * ax;
            st_arr(p, p.cur, 4)[s] += kick * ay;
            st_arr(p, p.cur, 5)[s] += kick * az;
        }
        double gp = 0.0;
        if (POT) {
            gp = -p.G * acc4[3].value();
            p.pots[s] = gp;
        }
        if (!(isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(gp))) bad = 1;
    }
    if (bad) dev::set_status(p.status, kStatusNonFinite);
}

// The fold of one step fused with the next step's opening: per slot (one
// block per 128-slot block) the total as bsym_fold_kernel, a = G x total,
// the closing kick of this step and the opening kick of the next in one
// v += kick a (kick = h), drift x += dt v, the hi/lo pack of x and the boxes
// (pack_slot's, without rewriting the mass plane: no re-sort came between).
// The kernel is bound by the FP64 pipe, so its conversions between float
// and double and its finiteness tests run on the integer pipes
// (nb_fpconv.cuh).  Neither a nor the potential is stored: the next step's
// fold replaces a before anything reads it, and only the last step of a
// loop sums the potential.
template <int POL>
__global__ void __launch_bounds__(BW) bsym_fold_pack_kernel(BsParams p, double kick, double dt) {
    const int64_t s = (int64_t)blockIdx.x * BW + threadIdx.x;
    if ((int64_t)blockIdx.x * BW >= __ldg(p.totals)) return;  // whole block
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.counter = 0u;
    const int i = p.perm[s];
    const int4 bm = p.bmeta[blockIdx.x];
    float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
    if (i >= 0) {
        // the state first: its loads overlap the sums' (the kernel is bound
        // by the latency of its dependent loads)
        double x0[3], v0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            x0[d] = st_arr(p, p.cur, d)[s];
            v0[d] = st_arr(p, p.cur, 3 + d)[s];
        }
        FoldAcc<POL> acc4[4];
        slot_sums<POL, false>(p, s, bm, acc4);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double a = acc4[d].value();
            if (p.G != 1.0) a *= p.G;
            ok = ok && fpconv::finite_d(a);
            const double v = v0[d] + kick * a;
            const double x = x0[d] + dt * v;
            st_arr(p, p.cur, 3 + d)[s] = v;
            st_arr(p, p.cur, d)[s] = x;
            hi[d] = fpconv::d2f(x);
            lo[d] = fpconv::d2f(x - fpconv::f2d(hi[d]));
        }
        if (!ok) dev::set_status(p.status, kStatusNonFinite);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p.soa[d * p.Ns + s] = hi[d];
        p.soa[(4 + d) * p.Ns + s] = lo[d];
    }
    set_box(p, s, i >= 0, hi);
}

template <int POL, int MODE>
int launch_bsym_steps(BsParams p, const BatchedJob &j, int64_t nb_max) {
    const cudaStream_t st = j.stream;
    const unsigned pack_grid = (unsigned)nb_max;
    const unsigned fold_grid = (unsigned)std::min<int64_t>(cdiv(nb_max * BW, 256), 64 * (int64_t)device_sm_count());
    const unsigned item_grid = (unsigned)device_sm_count();
    constexpr int sort_smem = 12 * kBsMaxN;  // keys and the old permutation
    {
        const int rc = smem_optin(reinterpret_cast<const void *>(bsym_sort_kernel), sort_smem);
        if (rc != NB_OK) return rc;
    }
    p.cur = 0;
    auto sort = [&](int from_user) {
        bsym_sort_kernel<<<(unsigned)p.B, 512, sort_smem, st>>>(p, from_user);
        p.cur ^= 1;
        count_launch();
    };
    constexpr int IPOL = POL == NB_PREC_F64ACC ? NB_PREC_FP32 : POL;
    const size_t item_smem = (size_t)NW * 16 * 32 * sizeof(Acc<IPOL>);
    for (const void *k : {reinterpret_cast<const void *>(bsym_item_kernel<POL, MODE, true>),
                          reinterpret_cast<const void *>(bsym_item_kernel<POL, MODE, false>)}) {
        const int rc = smem_optin(k, item_smem);
        if (rc != NB_OK) return rc;
    }
    // the potential is evaluated only where the caller can see it: a
    // forces-only call, or the last step of a step loop
    auto items = [&](bool pot) {
        if (pot)
            bsym_item_kernel<POL, MODE, true><<<item_grid, NT, item_smem, st>>>(p);
        else
            bsym_item_kernel<POL, MODE, false><<<item_grid, NT, item_smem, st>>>(p);
        count_launch();
    };
    const bool want_pot = j.pot != nullptr;
    const double h = j.dt;
    bsym_setup_kernel<<<1, 1024, 0, st>>>(p, j.N);
    count_launch();
    sort(1);
    if (!j.acc_valid || j.nsteps == 0) {
        bsym_pack_kernel<<<pack_grid, BW, 0, st>>>(p, 0.0, 0.0);
        items(want_pot && j.nsteps == 0);
        if (want_pot && j.nsteps == 0)
            bsym_fold_kernel<POL, true><<<fold_grid, 256, 0, st>>>(p, 0.0);
        else
            bsym_fold_kernel<POL, false><<<fold_grid, 256, 0, st>>>(p, 0.0);
        count_launch(2);
    }
    // Step n: [re-sort] [opening kick + drift + pack] items fold.  When no
    // re-sort separates step n from step n + 1, the fold of step n also
    // does step n + 1's opening kick, drift and pack (one pass, one launch).
    bool packed = false;
    for (int64_t n = 0; n < j.nsteps; ++n) {
        if (n > 0 && n % kBsResort == 0) sort(0);
        if (!packed) {
            bsym_pack_kernel<<<pack_grid, BW, 0, st>>>(p, 0.5 * h, h);
            count_launch();
        }
        const bool last = n == j.nsteps - 1;
        items(want_pot && last);
        packed = !last && (n + 1) % kBsResort != 0;
        if (packed)
            bsym_fold_pack_kernel<POL><<<pack_grid, BW, 0, st>>>(p, h, h);
        else if (want_pot && last)
            bsym_fold_kernel<POL, true><<<fold_grid, 256, 0, st>>>(p, 0.5 * h);
        else
            bsym_fold_kernel<POL, false><<<fold_grid, 256, 0, st>>>(p, 0.5 * h);
        count_launch();
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

// ------------------------------------------------------------ batched host
BsymLayout bsym_layout(int64_t N, int32_t B, int g) {
    BsymLayout z{};
    if (g < 1 || g > BG) g = BG;
    z.Ns = round_up(N + (int64_t)BW * B, BW);
    z.blocks = z.Ns / BW;
    // a system of n <= 64 blocks has sum over rows of ceil(m / g), m = 1..n,
    // items: <= n (n + 1) / (2 g) + n <= n (65 / (2 g) + 1)
    z.items = (65 / (2 * g) + 2) * z.blocks;
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
    z.o_bmeta = take(16 * (size_t)z.blocks);
    z.o_items = take(16 * (size_t)z.items);
    z.o_order = take(4 * (size_t)z.items);
    z.o_misc = take(256);  // counter, totals
    z.o_soa = take(4 * (size_t)kPackArrays * z.Ns);
    z.o_perm = take(4 * (size_t)z.Ns);
    z.o_box32 = take(32 * (size_t)(z.Ns / 32));
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
    const int g = j.item_blocks == 0 ? BG : j.item_blocks;
    if (g != 2 && g != 4 && g != BG)
        return fail(NB_ERR_INVALID, "item_blocks must be 2, 4 or 8 (got %d)", j.item_blocks);
    const BsymLayout z = bsym_layout(j.N, j.B, g);
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
    p.bmeta = reinterpret_cast<int4 *>(base + z.o_bmeta);
    p.items = reinterpret_cast<int4 *>(base + z.o_items);
    p.order = reinterpret_cast<int32_t *>(base + z.o_order);
    p.counter = reinterpret_cast<unsigned *>(base + z.o_misc);
    p.totals = reinterpret_cast<int64_t *>(base + z.o_misc + 64);
    p.soa = reinterpret_cast<float *>(base + z.o_soa);
    p.Ns = z.Ns;
    p.perm = reinterpret_cast<int *>(base + z.o_perm);
    p.box32 = reinterpret_cast<float *>(base + z.o_box32);
    p.P = reinterpret_cast<float *>(base + z.o_P);
    p.rec = reinterpret_cast<float *>(base + z.o_rec);
    p.st[0] = reinterpret_cast<double *>(base + z.o_st0);
    p.st[1] = reinterpret_cast<double *>(base + z.o_st1);
    p.pots = reinterpret_cast<double *>(base + z.o_pots);
    p.cur = 0;
    p.items_cap = z.items;
    p.pairs_cap = z.pairs;
    p.g = g;
    p.gamma = j.gamma > 0.f ? j.gamma : kBsNearGamma;
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
