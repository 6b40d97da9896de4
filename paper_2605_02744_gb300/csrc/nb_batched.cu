// Many independent N-body clusters of uneven size in one persistent launch
// (the SPMD split of Sec. 3.1 applied to whole systems: each unit of work is
// an independent set of particles).
//
// The grid is a set of thread-block clusters of CS CTAs (hardware cluster
// barriers: every CTA of a cluster is co-resident, so there is no software
// spin-wait).  Each thread-block cluster pops N-body clusters from a queue
// ordered largest first (atomic counter; the order comes from a one-block
// bitonic sort of the sizes) and runs every leapfrog step of that system
// before taking the next:
//
//   per step, each CTA for its own slice of the system's particles:
//     v += (dt/2) a;  x += dt v;  pack x (split hi/lo FP32) and m   (FP64 state)
//     cluster barrier
//     a, phi of its slice against all particles of the system; v += (dt/2) a
//
// The packed positions are double-buffered (one barrier per step).  j-tiles
// are read through L2 (ld.global.cg: other CTAs of the cluster wrote them) into
// shared memory, the next tile prefetched into registers during the current
// one.  Each thread keeps 2 i-particles in registers (independent FMA chains,
// <= 128 registers so a 512-thread CTA fits); when a slice has fewer than
// two particles per thread, groups of L = 2..32 lanes share the same
// i-particles, split the j-pairs, and are summed with a fixed xor-shuffle
// tree (bitwise reproducible).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <mutex>

#include "nb_device.cuh"
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

size_t batched_scratch_bytes(int32_t B) {
    return 4 * (size_t)(B > 0 ? B : 1) + 4 * (size_t)kBMaxSlots + 256;
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
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = tid; e < P; e += blockDim.x) {
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
    }
    for (int c = tid; c < B; c += blockDim.x) order[c] = (int)(keys[c] & 0xffffffffu);
}

// ---------------------------------------------------------------- pieces
__device__ __forceinline__ void pack_slice(const BatchedParams &p, int64_t s0, int64_t s1,
                                           float *pk, bool kick_drift) {
    const double half = 0.5 * p.dt;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
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
        store_packed(pk, p.Np, i, hi, lo, __double2float_rn(p.mass[i]));
    }
}

// Forces on the i of one chunk of the slice [.., s1) from all j of the
// system [o0, o1).  The CTA's BT threads form G = BT / L groups of L lanes;
// group g holds the IR particles c0 + k G + g (k < IR) and its lanes split
// the j-pairs of every tile (lane l takes pairs l, l + L, ...).  The next
// tile is loaded into registers while the current one is computed.
template <int BT, int IR, int POL>
__device__ __forceinline__ void force_chunk(const BatchedParams &p, int64_t o0, int64_t o1,
                                            int64_t c0, int64_t s1, const float *pk, float eps2,
                                            double kick, int L, float (&tile)[7][kBTJ]) {
    constexpr int PER = 7 * kBTJ / BT;  // tile floats each thread stages
    static_assert(7 * kBTJ % BT == 0, "tile must split evenly over the CTA");
    const int tid = threadIdx.x;
    const int lane = tid % L;
    const int G = BT / L;
    const int grp = tid / L;
    float2 nx[IR], ny[IR], nz[IR], nxl[IR], nyl[IR], nzl[IR];
    float mi[IR];
    int64_t ii[IR];
    Acc<POL> tot[IR][4];
#pragma unroll
    for (int k = 0; k < IR; ++k) {
        ii[k] = c0 + (int64_t)k * G + grp;
        const bool live = ii[k] < s1;
        const int64_t i = live ? ii[k] : o0;
        const float x = __ldcg(pk + i), y = __ldcg(pk + p.Np + i), z = __ldcg(pk + 2 * p.Np + i);
        const float xl = __ldcg(pk + 4 * p.Np + i), yl = __ldcg(pk + 5 * p.Np + i),
                    zl = __ldcg(pk + 6 * p.Np + i);
        mi[k] = __ldcg(pk + 3 * p.Np + i);
        nx[k] = f2(-x, -x);
        ny[k] = f2(-y, -y);
        nz[k] = f2(-z, -z);
        nxl[k] = f2(-xl, -xl);
        nyl[k] = f2(-yl, -yl);
        nzl[k] = f2(-zl, -zl);
#pragma unroll
        for (int e = 0; e < 4; ++e) tot[k][e].zero();
    }
    const float2 e2 = f2(eps2, eps2);
    float pre[PER];
    auto fetch = [&](int64_t jt0) {
        const int64_t nj = (o1 - jt0) < kBTJ ? (o1 - jt0) : kBTJ;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * BT;
            const int arr = e / kBTJ, jj = e % kBTJ;
            pre[r] = jj < nj ? __ldcg(pk + arr * p.Np + jt0 + jj) : 0.f;
        }
    };
    fetch(o0);
    for (int64_t jt0 = o0; jt0 < o1; jt0 += kBTJ) {
        const int nj = (int)((o1 - jt0) < kBTJ ? (o1 - jt0) : kBTJ);
        __syncthreads();  // the previous tile is no longer read
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * BT;
            tile[e / kBTJ][e % kBTJ] = pre[r];
        }
        __syncthreads();
        if (jt0 + kBTJ < o1) fetch(jt0 + kBTJ);  // in flight during the pairs below
        float2 ax[IR], ay[IR], az[IR], ph[IR];
#pragma unroll
        for (int k = 0; k < IR; ++k) ax[k] = ay[k] = az[k] = ph[k] = f2(0.f, 0.f);
        // quads of j (float4 loads); a ragged tail reads the zero-mass pad
        const int nquads = (nj + 3) / 4;
        auto quad = [&](int jq) {
            const float4 X = *reinterpret_cast<const float4 *>(&tile[0][4 * jq]);
            const float4 Y = *reinterpret_cast<const float4 *>(&tile[1][4 * jq]);
            const float4 Z = *reinterpret_cast<const float4 *>(&tile[2][4 * jq]);
            const float4 M = *reinterpret_cast<const float4 *>(&tile[3][4 * jq]);
            const float4 XL = *reinterpret_cast<const float4 *>(&tile[4][4 * jq]);
            const float4 YL = *reinterpret_cast<const float4 *>(&tile[5][4 * jq]);
            const float4 ZL = *reinterpret_cast<const float4 *>(&tile[6][4 * jq]);
            pair2<IR, false, true>(f2(X.x, X.y), f2(Y.x, Y.y), f2(Z.x, Z.y), f2(XL.x, XL.y),
                                   f2(YL.x, YL.y), f2(ZL.x, ZL.y), f2(M.x, M.y), e2, nx, ny, nz,
                                   nxl, nyl, nzl, ax, ay, az, ph);
            pair2<IR, false, true>(f2(X.z, X.w), f2(Y.z, Y.w), f2(Z.z, Z.w), f2(XL.z, XL.w),
                                   f2(YL.z, YL.w), f2(ZL.z, ZL.w), f2(M.z, M.w), e2, nx, ny, nz,
                                   nxl, nyl, nzl, ax, ay, az, ph);
        };
        if (L == 1) {
#pragma unroll 2
            for (int jq = 0; jq < nquads; ++jq) quad(jq);
        } else {
            for (int jq = lane; jq < nquads; jq += L) quad(jq);
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
        const int64_t i = ii[k];
        if (i >= s1) continue;
        const double phs = v[k][3] - (double)(mi[k] * dev::rsqrt_approx(eps2));  // self pair
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

// Two i-particles per group (independent FMA chains) and as many lanes per
// group as the slice leaves room for, so small slices still fill the CTA.
template <int BT, int POL>
__device__ __forceinline__ void force_slice(const BatchedParams &p, int64_t o0, int64_t o1,
                                            int64_t s0, int64_t s1, const float *pk, float eps2,
                                            double kick, float (&tile)[7][kBTJ]) {
    const int64_t ns = s1 - s0;
    const int64_t groups = (ns + 1) / 2 > 0 ? (ns + 1) / 2 : 1;
    int L = 1;
    while (L < 32 && (int64_t)(2 * L) * groups <= BT) L <<= 1;
    const int64_t chunk = (int64_t)(BT / L) * 2;
    for (int64_t c0 = s0; c0 < s1; c0 += chunk)
        force_chunk<BT, 2, POL>(p, o0, o1, c0, s1, pk, eps2, kick, L, tile);
    // the epilogue's acc/vel writes (lane 0 of each group) are read by other
    // threads of this CTA in the next kick-drift-pack
    __syncthreads();
}

template <int CS, int BT, int POL>
__global__ void __launch_bounds__(BT, 1) batched_kernel(const BatchedParams p) {
    __shared__ __align__(16) float tile[7][kBTJ];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int g = blockIdx.x / CS;
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
            const int64_t s0 = o0 + (n * r) / CS, s1 = o0 + (n * (r + 1)) / CS;
            const float ef = (float)epsd;
            const float eps2 = ef * ef;
            int buf = 0;
            if (!p.acc_valid) {
                pack_slice(p, s0, s1, p.pack0, false);
                cl.sync();
                force_slice<BT, POL>(p, o0, o1, s0, s1, p.pack0, eps2, 0.0, tile);
            }
            for (int64_t step = 0; step < p.nsteps; ++step) {
                buf ^= 1;
                float *pk = buf ? p.pack1 : p.pack0;
                pack_slice(p, s0, s1, pk, true);
                cl.sync();
                force_slice<BT, POL>(p, o0, o1, s0, s1, pk, eps2, 0.5 * p.dt, tile);
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
    cfg.dynamicSmemBytes = 0;
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
    if (nclusters > kBMaxSlots) nclusters = kBMaxSlots;
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
    p.status = reinterpret_cast<uint32_t *>(j.ws + j.L.status);
    {
        int P = 1;
        while (P < j.B && P < kBSortMax) P <<= 1;
        const size_t smem = j.B <= kBSortMax ? (size_t)P * 8 : 0;
        static std::once_flag once;
        std::call_once(once, [] {
            cudaFuncSetAttribute(batched_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kBSortMax * 8);
        });
        batched_setup_kernel<<<1, 1024, smem, j.stream>>>(j.offsets, j.B, j.N, j.eps,
                                                          const_cast<int *>(p.order), p.counter,
                                                          p.status);
        count_launch();
        NB_CUDA(cudaGetLastError());
    }
    const int cs = j.cluster > 0 ? j.cluster : 4;  // measured best on GB300 (4 x 512 threads)
    const int bt = j.threads > 0 ? j.threads : 512;
    switch (j.precision) {
        case NB_PREC_FP32: return launch_batched_pol<NB_PREC_FP32>(p, cs, bt, j.stream);
        case NB_PREC_KAHAN: return launch_batched_pol<NB_PREC_KAHAN>(p, cs, bt, j.stream);
        case NB_PREC_F64ACC: return launch_batched_pol<NB_PREC_F64ACC>(p, cs, bt, j.stream);
    }
    return fail(NB_ERR_INVALID, "unknown precision %d", j.precision);
}

}  // namespace nb
