// nb_forces_noalloc: the force + potential evaluation of nb_forces for
// callers that may not allocate device memory and so cannot supply a
// workspace.  Its scratch (packed positions, arrival counters, stream-K
// partial records, status word) lives in one file-scope device array of
// fixed size, which every GPU that loads this library holds until the
// process exits.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "nb_internal.h"

namespace nb {

// Largest N this entry point serves, the fixed launch shape it uses, and
// the resulting scratch size (about 6.2 MB).
constexpr int64_t kNoAllocMaxN = 32768;
constexpr int kNoAllocThreads = 128, kNoAllocIpt = 2, kNoAllocTileJ = 128, kNoAllocStages = 3;
constexpr int kNoAllocCtasPerSm = 2;
constexpr int64_t kNoAllocMaxGrid = 320;  // >= 2 CTAs x 152 SMs
constexpr int64_t kNoAllocBlockI = kNoAllocThreads * kNoAllocIpt;
constexpr size_t kNaStatus = 0;
constexpr size_t kNaCounters = 256;
constexpr size_t kNaPack = kNaCounters + 4096;
constexpr size_t kNaRecords = kNaPack + (size_t)kPackArrays * 4 * kNoAllocMaxN;
constexpr size_t kNaBytes = kNaRecords + 2 * (size_t)kNoAllocMaxGrid * kNoAllocBlockI * 32;
static_assert(kNaPack % 256 == 0 && kNaRecords % 256 == 0, "regions must stay 256-B aligned");
static_assert(kNoAllocMaxN / 64 + 1 <= 4096 / 4, "counter region too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch, looked up once per device.
static std::mutex g_na_mu;
static void *g_na_ptr[64];

static int scratch_address(void **out) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NB_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return NB_OK;
}

// Status word of the array on the current device (nb_poll_status(NULL, ...)).
int noalloc_status_word(uint32_t **out) {
    void *base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != NB_OK) return rc;
    *out = reinterpret_cast<uint32_t *>(static_cast<char *>(base) + kNaStatus);
    return NB_OK;
}

}  // namespace nb

using namespace nb;

extern "C" int nb_forces_noalloc(const double *pos, const double *mass, int64_t N, double eps,
                                 double *acc, double *pot, const nb_opts *o) {
    clear_error();
    if (!o) return fail(NB_ERR_INVALID, "opts is NULL");
    if (N > kNoAllocMaxN)
        return fail(NB_ERR_INVALID,
                    "nb_forces_noalloc serves N <= %lld (got %lld); use nb_forces with a "
                    "workspace for larger systems",
                    (long long)kNoAllocMaxN, (long long)N);
    if (N < 1) return fail(NB_ERR_INVALID, "N must be >= 1 (got %lld)", (long long)N);
    if (!pos || !mass || !acc) return fail(NB_ERR_INVALID, "pos, mass and acc must be non-NULL");
    if (((uintptr_t)pos | (uintptr_t)mass | (uintptr_t)acc | (uintptr_t)pot) & 7)
        return fail(NB_ERR_INVALID, "arrays must be 8-byte aligned");
    if (!(eps >= 0.0) || !isfinite(eps)) return fail(NB_ERR_INVALID, "eps must be finite and >= 0");
    if (eps > 0.0 && (float)eps * (float)eps < 1.2e-38f)
        return fail(NB_ERR_INVALID, "eps^2 underflows FP32; use eps = 0 or eps >= 1.1e-19");
    if (!isfinite(o->G)) return fail(NB_ERR_INVALID, "G must be finite");
    if (o->precision < NB_PREC_FP32 || o->precision > NB_PREC_FP64)
        return fail(NB_ERR_INVALID, "unknown precision %d", o->precision);
    if (o->positions < NB_POS_DEFAULT || o->positions > NB_POS_ADAPTIVE)
        return fail(NB_ERR_INVALID, "unknown positions mode %d", o->positions);
    if (o->pairs < NB_PAIRS_DEFAULT || o->pairs > NB_PAIRS_SYMMETRIC)
        return fail(NB_ERR_INVALID, "unknown pairs mode %d", o->pairs);
    // the fixed array holds the direct kernel's scratch only: no Hilbert
    // sort buffers, no symmetric-pair sums, one compiled launch shape
    if (o->positions == NB_POS_ADAPTIVE)
        return fail(NB_ERR_UNSUPPORTED, "nb_forces_noalloc has no adaptive (sorted) positions");
    if (o->pairs == NB_PAIRS_SYMMETRIC)
        return fail(NB_ERR_UNSUPPORTED, "nb_forces_noalloc evaluates every ordered pair only");
    if (o->tune)
        return fail(NB_ERR_UNSUPPORTED, "nb_forces_noalloc runs one fixed launch shape");
    if ((int64_t)kNoAllocCtasPerSm * device_sm_count() > kNoAllocMaxGrid)
        return fail(NB_ERR_UNSUPPORTED, "device has more SMs than the fixed scratch serves");

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != NB_OK) return rc;
    char *ws = static_cast<char *>(base);
    cudaStream_t st = (cudaStream_t)o->stream;
    // The array keeps the previous call's contents: the status word and the
    // arrival counters must start at zero (a status the caller has not polled
    // is lost here).
    NB_CUDA(cudaMemsetAsync(ws, 0, kNaPack, st));

    ForceJob j;
    memset(&j, 0, sizeof j);
    j.L.status = kNaStatus;
    j.L.counters = kNaCounters;
    j.L.packA = kNaPack;
    j.L.records = kNaRecords;
    j.L.Np = kNoAllocMaxN;
    j.L.total = kNaBytes;
    j.shape = Shape{kNoAllocThreads, kNoAllocIpt, kNoAllocTileJ, kNoAllocStages,
                    kNoAllocCtasPerSm};
    j.pos = pos;
    j.mass = mass;
    j.N = N;
    j.i0 = 0;
    j.ni = N;
    j.eps = eps;
    j.G = o->G;
    j.acc = acc;
    j.pot = pot;
    j.precision = o->precision;
    j.split = positions_split(o);
    j.timeout = o->timeout_cycles > 0 ? (long long)o->timeout_cycles : kDefaultTimeoutCycles;
    j.unissued = o->test_unissued_stage > 0 ? (int64_t)o->test_unissued_stage - 1 : -1;
    j.stream = st;
    j.ws = ws;
    return launch_force(j);
}
