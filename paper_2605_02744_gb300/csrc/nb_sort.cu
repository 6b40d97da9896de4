// Spatial ordering for the adaptive-displacement force path.
//
// Each evaluation sorts the particles along a Hilbert curve of their
// FP64 positions, packs them in that order, and records an axis-aligned box
// for every 64 consecutive j-slots and for every warp's i-slots.  Spatially
// compact groups let the force kernel pick, per (warp, 64-particle sub-tile)
// pair, the single-float displacement for well-separated pairs and the split
// hi/lo displacement only where the gap is small relative to the coordinates
// (where FP32 rounding of the positions matters).
//
//   bbox:     FP64 min/max of the positions (atomics on order-preserving
//             integer images; min/max do not depend on order)
//   keys:     30-bit Hilbert index of the position's cell in that box << 32 | index
//   sort:     bitonic network on 64-bit keys (shared-memory passes for
//             strides below 2048, global passes above); keys are unique, so
//             the order is fully determined
//   pack:     split hi/lo SoA in sorted order + permutation (slot -> index)
//   boxes:    per group of `unit` slots: lo[3], hi[3], max |coordinate|
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_order.cuh"
#include "nb_internal.h"

namespace nb {

constexpr int kSortChunk = 4096;  // keys per shared-memory bitonic block

__device__ __forceinline__ long long ordered_bits(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double from_ordered(long long b) {
    return __longlong_as_double(b >= 0 ? b : (b ^ 0x7fffffffffffffffLL));
}

__global__ void bbox_init_kernel(long long *box) {
    if (threadIdx.x < 3) {
        box[threadIdx.x] = ordered_bits(__longlong_as_double(0x7ff0000000000000LL));       // +inf
        box[3 + threadIdx.x] = ordered_bits(__longlong_as_double((long long)0xfff0000000000000ULL));  // -inf
    }
}

__global__ void bbox_kernel(const double *__restrict__ pos, int64_t N, long long *box) {
    __shared__ double smin[3][256], smax[3][256];
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double x = pos[3 * i + c];
            lo[c] = fmin(lo[c], x);
            hi[c] = fmax(hi[c], x);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        smin[c][threadIdx.x] = lo[c];
        smax[c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                smin[c][threadIdx.x] = fmin(smin[c][threadIdx.x], smin[c][threadIdx.x + h]);
                smax[c][threadIdx.x] = fmax(smax[c][threadIdx.x], smax[c][threadIdx.x + h]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        atomicMin(&box[threadIdx.x], ordered_bits(smin[threadIdx.x][0]));
        atomicMax(&box[3 + threadIdx.x], ordered_bits(smax[threadIdx.x][0]));
    }
}

__global__ void hilbert_keys_kernel(const double *__restrict__ pos, int64_t N, int64_t P,
                                   const long long *__restrict__ box,
                                   unsigned long long *__restrict__ keys) {
    double lo[3], scale[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = from_ordered(box[c]);
        const double ext = from_ordered(box[3 + c]) - lo[c];
        scale[c] = ext > 0.0 ? 1023.0 / ext : 0.0;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < N) {
            const uint32_t code = dev::hilbert30(dev::cell10(pos[3 * i], lo[0], scale[0]),
                                  dev::cell10(pos[3 * i + 1], lo[1], scale[1]),
                                  dev::cell10(pos[3 * i + 2], lo[2], scale[2]));
            k = ((unsigned long long)code << 32) | (unsigned long long)(uint32_t)i;
        }
        keys[i] = k;
    }
}

// All bitonic stages with stride < kSortChunk for keys [blk*C, (blk+1)*C):
// stage sizes k from k_lo to k_hi; with k_lo == k_hi only the strides of that
// one stage below the chunk size.  Direction follows the global index.
__global__ void bitonic_smem_kernel(unsigned long long *keys, int64_t k_lo, int64_t k_hi) {
    __shared__ unsigned long long s[kSortChunk];
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    for (int e = threadIdx.x; e < kSortChunk; e += blockDim.x) s[e] = keys[base + e];
    __syncthreads();
    for (int64_t k = k_lo; k <= k_hi; k <<= 1) {
        int64_t j0 = k >> 1;
        if (j0 >= kSortChunk) j0 = kSortChunk >> 1;
        for (int64_t j = j0; j > 0; j >>= 1) {
            for (int e = threadIdx.x; e < kSortChunk; e += blockDim.x) {
                const int x = e ^ (int)j;
                if (x > e) {
                    const bool asc = ((base + e) & k) == 0;
                    const unsigned long long a = s[e], b = s[x];
                    if ((a > b) == asc) {
                        s[e] = b;
                        s[x] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < kSortChunk; e += blockDim.x) keys[base + e] = s[e];
}

// One compare-exchange stride j (>= kSortChunk) of stage k over all P keys.
__global__ void bitonic_global_kernel(unsigned long long *keys, int64_t P, int64_t k, int64_t j) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P / 2;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = (t / j) * 2 * j + (t % j);
        const int64_t x = e + j;
        const bool asc = (e & k) == 0;
        const unsigned long long a = keys[e], b = keys[x];
        if ((a > b) == asc) {
            keys[e] = b;
            keys[x] = a;
        }
    }
}

__global__ void pack_sorted_kernel(const double *__restrict__ pos, const double *__restrict__ mass,
                                   const unsigned long long *__restrict__ keys, int64_t N,
                                   int64_t Np, float *__restrict__ soa, int *__restrict__ perm) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < Np;
         s += (int64_t)gridDim.x * blockDim.x) {
        float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f}, m = 0.f;
        int idx = -1;
        if (s < N) {
            idx = (int)(uint32_t)(keys[s] & 0xffffffffull);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double x = pos[3 * (int64_t)idx + c];
                hi[c] = __double2float_rn(x);
                lo[c] = __double2float_rn(x - (double)hi[c]);
            }
            m = __double2float_rn(mass[idx]);
        }
        store_packed(soa, Np, s, hi, lo, m);
        perm[s] = idx;
    }
}

// Box of the valid slots [u*unit, min((u+1)*unit, N)) of the sorted pack:
// out[u*8 + 0..2] = lo, 3..5 = hi, 6 = max |coordinate| over the box.
__global__ void slot_boxes_kernel(const float *__restrict__ soa, int64_t N, int64_t Np, int unit,
                                  float *__restrict__ out) {
    __shared__ float red[6][256];
    const int64_t u = blockIdx.x;
    const int64_t s0 = u * unit;
    const int64_t s1 = (s0 + unit) < N ? (s0 + unit) : N;
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = soa[c * Np + s];
            lo[c] = fminf(lo[c], x);
            hi[c] = fmaxf(hi[c], x);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        red[c][threadIdx.x] = lo[c];
        red[3 + c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                red[c][threadIdx.x] = fminf(red[c][threadIdx.x], red[c][threadIdx.x + h]);
                red[3 + c][threadIdx.x] = fmaxf(red[3 + c][threadIdx.x], red[3 + c][threadIdx.x + h]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float amax = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            out[u * 8 + c] = red[c][0];
            out[u * 8 + 3 + c] = red[3 + c][0];
            amax = fmaxf(amax, fmaxf(fabsf(red[c][0]), fabsf(red[3 + c][0])));
        }
        out[u * 8 + 6] = s1 > s0 ? amax : 0.f;
        out[u * 8 + 7] = 0.f;
    }
}

int64_t sort_keys_len(int64_t N) {
    int64_t P = kSortChunk;
    while (P < N) P <<= 1;
    return P;
}

int launch_sorted_pack(const double *pos, const double *mass, int64_t N, int64_t Np, float *soa,
                       int *perm, unsigned long long *keys, long long *box6, float *tile_boxes,
                       int tile_unit, float *block_boxes, int block_unit, bool reuse_order,
                       cudaStream_t st) {
    const int64_t P = sort_keys_len(N);
    const int threads = 256;
    if (reuse_order) goto pack;  // same particles as the last sorted call: keep its order
    {
    bbox_init_kernel<<<1, 32, 0, st>>>(box6);
    count_launch();
    const int64_t gb = std::min<int64_t>(cdiv(N, threads), 1024);
    bbox_kernel<<<(unsigned)gb, threads, 0, st>>>(pos, N, box6);
    count_launch();
    hilbert_keys_kernel<<<(unsigned)std::min<int64_t>(cdiv(P, threads), 8192), threads, 0, st>>>(
        pos, N, P, box6, keys);
    count_launch();
    const unsigned nchunks = (unsigned)(P / kSortChunk);
    bitonic_smem_kernel<<<nchunks, 1024, 0, st>>>(keys, 2, kSortChunk);
    count_launch();
    for (int64_t k = 2 * kSortChunk; k <= P; k <<= 1) {
        for (int64_t j = k >> 1; j >= kSortChunk; j >>= 1) {
            bitonic_global_kernel<<<(unsigned)std::min<int64_t>(cdiv(P / 2, threads), 8192),
                                    threads, 0, st>>>(keys, P, k, j);
            count_launch();
        }
        bitonic_smem_kernel<<<nchunks, 1024, 0, st>>>(keys, k, k);
        count_launch();
    }
    }
pack:
    pack_sorted_kernel<<<(unsigned)std::min<int64_t>(cdiv(Np, threads), 8192), threads, 0, st>>>(
        pos, mass, keys, N, Np, soa, perm);
    count_launch();
    // every unit up to Np: units past N get an empty box (never near)
    slot_boxes_kernel<<<(unsigned)(Np / tile_unit), 256, 0, st>>>(soa, N, Np, tile_unit,
                                                                  tile_boxes);
    count_launch();
    slot_boxes_kernel<<<(unsigned)(Np / block_unit), 256, 0, st>>>(soa, N, Np, block_unit,
                                                                   block_boxes);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace nb
