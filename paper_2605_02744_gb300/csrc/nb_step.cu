// O(N) kernels of the leapfrog step and the energy bookkeeping.
//
// kick_drift_pack: the opening half-kick and the drift of a kick-drift-kick
// step, v += (dt/2) a; x += dt v, in FP64, followed by the split FP32 SoA
// pack (hi/lo) of the new positions for the next force evaluation.  The closing half-kick is
// fused into the force kernel's epilogue.  This replaces the host-side FP64
// predict/correct around the device evaluation of Sec. 2.1 / Sec. 3.1.
//
// energy: K = 1/2 sum m |v|^2 and W = 1/2 sum m phi in FP64 with a fixed
// reduction tree (per-block tree in shared memory, then one block folds the
// block partials in index order), so the result is bitwise reproducible.
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {

__global__ void kick_drift_pack_kernel(double *__restrict__ pos, double *__restrict__ vel,
                                       const double *__restrict__ acc,
                                       const double *__restrict__ mass, int64_t N, int64_t Np,
                                       double dt, float *__restrict__ soa) {
    const double half = 0.5 * dt;
    const int64_t n_iter = soa ? Np : N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_iter;
         i += (int64_t)gridDim.x * blockDim.x) {
        float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
        float m = 0.f;
        if (i < N) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double v = vel[3 * i + c] + half * acc[3 * i + c];
                const double x = pos[3 * i + c] + dt * v;
                vel[3 * i + c] = v;
                pos[3 * i + c] = x;
                hi[c] = __double2float_rn(x);
                lo[c] = __double2float_rn(x - (double)hi[c]);
            }
            m = __double2float_rn(mass[i]);
        }
        if (soa) store_packed(soa, Np, i, hi, lo, m);
    }
}

int launch_kick_drift_pack(double *pos, double *vel, const double *acc, const double *mass,
                           int64_t N, int64_t Np, double dt, float *soa, cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>(cdiv(Np, threads), 8192);
    kick_drift_pack_kernel<<<(unsigned)blocks, threads, 0, st>>>(pos, vel, acc, mass, N, Np, dt,
                                                                 soa);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

__global__ void kick_drift_kernel(double *__restrict__ pos, double *__restrict__ vel,
                                  const double *__restrict__ acc, int64_t n, double kick,
                                  double drift) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double v = vel[t] + kick * acc[t];
        vel[t] = v;
        if (drift != 0.0) pos[t] = pos[t] + drift * v;
    }
}

int launch_kick_drift(double *pos, double *vel, const double *acc, int64_t n, double kick,
                      double drift, cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>(cdiv(3 * n, threads), 8192);
    kick_drift_kernel<<<(unsigned)blocks, threads, 0, st>>>(pos, vel, acc, n, kick, drift);
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

constexpr int kEnergyThreads = 256;
constexpr int kEnergyMaxBlocks = 1024;

__global__ void energy_partial_kernel(const double *__restrict__ vel,
                                      const double *__restrict__ mass,
                                      const double *__restrict__ pot, int64_t N,
                                      double *__restrict__ partial) {
    __shared__ double sk[kEnergyThreads], sw[kEnergyThreads];
    double k = 0.0, w = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kEnergyThreads + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * kEnergyThreads) {
        const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        k += 0.5 * mass[i] * (vx * vx + vy * vy + vz * vz);
        w += 0.5 * mass[i] * pot[i];
    }
    sk[threadIdx.x] = k;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int h = kEnergyThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sk[threadIdx.x] += sk[threadIdx.x + h];
            sw[threadIdx.x] += sw[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sk[0];
        partial[2 * blockIdx.x + 1] = sw[0];
    }
}

__global__ void energy_final_kernel(const double *__restrict__ partial, int nblocks,
                                    double *__restrict__ out3, uint32_t *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double K = 0.0, W = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            K += partial[2 * b];
            W += partial[2 * b + 1];
        }
        out3[0] = K;
        out3[1] = W;
        out3[2] = K + W;
        if (!(isfinite(K) && isfinite(W))) dev::set_status(status, kStatusNonFinite);
    }
}

int launch_energy(const double *vel, const double *mass, const double *pot, int64_t N,
                  double *out3, char *ws, const WsLayout &L, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>(cdiv(N, kEnergyThreads), kEnergyMaxBlocks);
    double *partial = reinterpret_cast<double *>(ws + L.scratch);
    energy_partial_kernel<<<blocks, kEnergyThreads, 0, st>>>(vel, mass, pot, N, partial);
    count_launch();
    NB_CUDA(cudaGetLastError());
    energy_final_kernel<<<1, 32, 0, st>>>(partial, blocks, out3,
                                          reinterpret_cast<uint32_t *>(ws + L.status));
    count_launch();
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace nb
