// Host side of the C ABI (include/nbody.h): argument checks, workspace
// layout, launch-shape choice, the leapfrog driver and CUDA-graph replay.
#include <cuda_runtime.h>

#include <cmath>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "nb_fixed.cuh"
#include "nb_fpconv.cuh"
#include "nb_internal.h"

namespace nb {

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = '\0'; }

int cuda_check(cudaError_t e, const char *what) {
    return fail(NB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// Kernel timer: a ring of at most kTimerPairs event pairs on the device that
// was current when timing was switched on.  A launch that finds every pair
// holding an unread measurement first folds the oldest one into g_tm_ms (an
// event synchronisation on the host), so a long step loop reuses the same
// few events instead of creating one pair per launch.
constexpr size_t kTimerPairs = 64;
static std::mutex g_tm_mu;
static bool g_tm_on = false, g_tm_open = false;
static int g_tm_err = 0;
static int g_tm_dev = -1;
static double g_tm_ms = 0.0;        // folded measurements
static int64_t g_tm_count = 0;      // launches recorded since timing was switched on
static size_t g_tm_head = 0, g_tm_live = 0;  // ring: oldest unread pair, unread pairs
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_tm_ev;

static bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// Folds the oldest unread pair into g_tm_ms (caller holds g_tm_mu).
static int timer_fold_oldest() {
    auto &e = g_tm_ev[g_tm_head];
    float ms = 0.f;
    cudaError_t r = cudaEventSynchronize(e.second);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e.first, e.second);
    if (r != cudaSuccess) return 1;
    g_tm_ms += ms;
    g_tm_head = (g_tm_head + 1) % kTimerPairs;
    --g_tm_live;
    return 0;
}

void kernel_timer_begin(cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_tm_mu);
    if (!g_tm_on || g_tm_open || g_tm_err || capturing(st)) return;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || (g_tm_dev >= 0 && dev != g_tm_dev)) {
        g_tm_err = 1;  // events belong to one device
        return;
    }
    g_tm_dev = dev;
    if (g_tm_live == kTimerPairs && timer_fold_oldest()) {
        g_tm_err = 1;
        return;
    }
    const size_t slot = (g_tm_head + g_tm_live) % kTimerPairs;
    while (g_tm_ev.size() <= slot) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            g_tm_err = 1;
            return;
        }
        g_tm_ev.push_back({a, b});
    }
    if (cudaEventRecord(g_tm_ev[slot].first, st) != cudaSuccess) {
        g_tm_err = 1;
        return;
    }
    g_tm_open = true;
}

void kernel_timer_end(cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_tm_mu);
    if (!g_tm_open) return;
    g_tm_open = false;
    const size_t slot = (g_tm_head + g_tm_live) % kTimerPairs;
    if (cudaEventRecord(g_tm_ev[slot].second, st) != cudaSuccess) {
        g_tm_err = 1;
        return;
    }
    ++g_tm_live;
    ++g_tm_count;
}

// ----------------------------------------------------------------- device
int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();  // no device here: size for a full GB300
        return 152;
    }
    return n;
}

int smem_optin(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<std::tuple<const void *, int, size_t>> done;
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(kernel, dev, bytes);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) return NB_OK;
    NB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.insert(key);
    return NB_OK;
}

// ------------------------------------------------------------ shapes
bool force_shape_compiled(const Shape &s);
bool vjp_shape_compiled(const Shape &s);

bool shape_compiled(const Shape &s, int kind) {
    return kind == kKindForce ? force_shape_compiled(s) : vjp_shape_compiled(s);
}

// Built-in shapes, from autotuner sweeps on GB300 (Kahan / F64ACC, default
// positions): 512 threads x 2 i/thread with 1024-particle tiles from
// N = 2^18 (the adaptive path; 2^20: 449 ms vs 538 ms for 256 x 4 x 256,
// because two i per thread leave room for 16 resident warps per SM);
// 256 x 2 x 512 from 2^15; 256 x 2 x 256 from 2^12; 128 x 1 x 64 below.
Shape default_shape(int64_t N, int precision, int kind) {
    (void)precision;
    if (kind == kKindForce) {
        if (N >= (1 << 18)) return Shape{512, 2, 1024, 2, 1};
        if (N >= (1 << 15)) return Shape{256, 2, 512, 2, 2};
        if (N >= (1 << 12)) return Shape{256, 2, 256, 3, 2};
        return Shape{128, 1, 64, 2, 4};
    }
    // VJP: (128, 2, 128, 3) fastest at 16384 and 65536 in a GB300 sweep
    if (N >= (1 << 12)) return Shape{128, 2, 128, 3, 4};
    return Shape{128, 1, 64, 2, 4};
}

bool resolve_shape(const nb_opts *opts, int64_t N, int kind, Shape *out) {
    Shape s = default_shape(N, opts ? opts->precision : NB_PREC_F64ACC, kind);
    if (opts && opts->tune) {
        const nb_tune *t = opts->tune;
        if (t->threads) s.threads = t->threads;
        if (t->i_per_thread) s.ipt = t->i_per_thread;
        if (t->tile_j) s.tile_j = t->tile_j;
        if (t->stages) s.stages = t->stages;
        if (t->ctas_per_sm) s.ctas_per_sm = t->ctas_per_sm;
    }
    if (s.ctas_per_sm < 1 || s.ctas_per_sm > 4) return false;
    *out = s;
    return shape_compiled(s, kind);
}

// ---------------------------------------------------------- workspace
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int64_t kPadParticles = 2048;  // >= every i-block and j-tile size
constexpr int64_t kForceRecordBytes = 32;
constexpr int64_t kVjpRecordBytes = 128;
constexpr size_t kScratchBase = 64 * 1024;

WsLayout ws_layout(int64_t N, int32_t B, const nb_opts *opts) {
    WsLayout L{};
    if (N < 1) N = 1;
    if (B < 1) B = 1;
    Shape sf, sv;
    if (!resolve_shape(opts, N, kKindForce, &sf)) sf = default_shape(N, 0, kKindForce);
    if (!resolve_shape(opts, N, kKindVjp, &sv)) sv = default_shape(N, 0, kKindVjp);
    L.Np = round_up(N, kPadParticles);
    const int64_t sms = device_sm_count();
    L.max_grid = 4 * sms;
    L.max_blocks = cdiv(N, 64) + 1;
    L.record_bytes_per_i = std::max(kForceRecordBytes * sf.block_i(),
                                    kVjpRecordBytes * sv.block_i());
    size_t off = 0;
    L.status = off;
    off = align256(off + 256);
    L.counters = off;
    off = align256(off + sizeof(uint32_t) * (size_t)L.max_blocks);
    L.packA = off;
    off = align256(off + 4 * kPackArrays * (size_t)L.Np);
    L.packB = off;
    off = align256(off + 16 * (size_t)L.Np);
    L.cot64 = off;
    off = align256(off + 32 * (size_t)L.Np);
    L.sortbuf = off;
    off = align256(off + sortbuf_bytes(L.Np));
    L.records = off;
    off = align256(off + 2 * (size_t)L.max_grid * (size_t)L.record_bytes_per_i);
    L.scratch = off;
    off = align256(off + kScratchBase + batched_scratch_bytes(B));
    if (sym_wanted(opts, N, B)) {
        const SymSizes z = sym_sizes(L.Np);
        L.sym_fx = off;
        L.sym_fx_bytes = z.fx_bytes;
        off = align256(off + z.fx_bytes);
        L.sym_cost = off;
        off = align256(off + z.cost_bytes);
    }
    if (bsym_wanted(opts, N, B)) {
        L.bsym = off;
        L.bsym_bytes = bsym_layout(N, B, bsym_item_blocks(opts)).bytes;
        off = align256(off + L.bsym_bytes);
    }
    L.total = off;
    return L;
}

int bsym_item_blocks(const nb_opts *o) {
    const int g = (o && o->tune) ? o->tune->item_blocks : 0;
    return g == 0 ? 8 : ((g == 2 || g == 4 || g == 8) ? g : 0);
}

bool bsym_wanted(const nb_opts *o, int64_t N, int32_t B) {
    (void)N;
    return o && B > 1 && o->precision != NB_PREC_FP64 && o->pairs != NB_PAIRS_DIRECT;
}

bool sym_wanted(const nb_opts *o, int64_t N, int32_t B) {
    if (!o || B != 1) return false;
    if (o->pairs == NB_PAIRS_SYMMETRIC) return true;
    return o->pairs == NB_PAIRS_DEFAULT && N >= kSymMinN && N <= kSymMaxN;
}

int check_ws(const void *ws, size_t ws_bytes, const WsLayout &L) {
    if (!ws) return fail(NB_ERR_INVALID, "workspace pointer is NULL");
    if (((uintptr_t)ws & 255) != 0) return fail(NB_ERR_INVALID, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(NB_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes,
                    L.total);
    return NB_OK;
}

bool positions_split(const nb_opts *o) {
    if (o->positions == NB_POS_SPLIT || o->positions == NB_POS_ADAPTIVE) return true;
    if (o->positions == NB_POS_SINGLE) return false;
    return o->precision != NB_PREC_FP32;
}

// Default thresholds of the adaptive path: a single evaluation pays a full
// Hilbert sort (symmetric Kahan evaluation, split / adaptive: 0.55 / 0.62 ms
// at 32768, 1.83 / 1.66 at 65536, 6.90 / 5.68 at 131072), a step loop sorts
// once per kResortEvery steps.
constexpr int64_t kAdaptiveMinN = 1 << 16;
constexpr int64_t kAdaptiveMinNStepping = 1 << 15;

bool positions_adaptive(const nb_opts *o, int64_t N, bool stepping) {
    if (o->precision == NB_PREC_FP64) return false;
    if (o->positions == NB_POS_ADAPTIVE) return true;
    if (o->positions != NB_POS_DEFAULT) return false;
    return o->precision != NB_PREC_FP32 &&
           N >= (stepping ? kAdaptiveMinNStepping : kAdaptiveMinN);
}

// ------------------------------------------------------------ checks
static int check_ptr(const void *p, const char *name, bool nullable = false) {
    if (!p) return nullable ? NB_OK : fail(NB_ERR_INVALID, "%s is NULL", name);
    if (((uintptr_t)p & 7) != 0) return fail(NB_ERR_INVALID, "%s is not 8-byte aligned", name);
    return NB_OK;
}

static int check_common(const nb_opts *o, int64_t N, double eps) {
    if (!o) return fail(NB_ERR_INVALID, "opts is NULL");
    if (N < 1) return fail(NB_ERR_INVALID, "N must be >= 1 (got %lld)", (long long)N);
    if (N > (int64_t)1 << 30) return fail(NB_ERR_INVALID, "N above 2^30 is not supported");
    if (!(eps >= 0.0) || !isfinite(eps)) return fail(NB_ERR_INVALID, "eps must be finite and >= 0");
    if (eps > 0.0 && (float)eps * (float)eps < 1.2e-38f)
        return fail(NB_ERR_INVALID, "eps^2 underflows FP32; use eps = 0 or eps >= 1.1e-19");
    if (!isfinite(o->G)) return fail(NB_ERR_INVALID, "G must be finite");
    if (o->precision < NB_PREC_FP32 || o->precision > NB_PREC_FP64)
        return fail(NB_ERR_INVALID, "unknown precision %d", o->precision);
    if (o->timeout_cycles < 0) return fail(NB_ERR_INVALID, "timeout_cycles must be >= 0");
    if (o->test_unissued_stage < 0) return fail(NB_ERR_INVALID, "test_unissued_stage must be >= 0");
    if (o->positions < NB_POS_DEFAULT || o->positions > NB_POS_ADAPTIVE)
        return fail(NB_ERR_INVALID, "unknown positions mode %d", o->positions);
    if (o->pairs < NB_PAIRS_DEFAULT || o->pairs > NB_PAIRS_SYMMETRIC)
        return fail(NB_ERR_INVALID, "unknown pairs mode %d", o->pairs);
    if (!(o->near_gamma >= 0.f) || !isfinite(o->near_gamma))
        return fail(NB_ERR_INVALID, "near_gamma must be finite and >= 0");
    return NB_OK;
}

static long long timeout_of(const nb_opts *o) {
    return o->timeout_cycles > 0 ? (long long)o->timeout_cycles : kDefaultTimeoutCycles;
}

static int64_t unissued_of(const nb_opts *o) {
    return o->test_unissued_stage > 0 ? (int64_t)o->test_unissued_stage - 1 : -1;
}

#define NB_TRY(expr)              \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != NB_OK) return rc_; \
    } while (0)

static int make_force_job(ForceJob *j, const double *pos, const double *mass, int64_t N,
                          double eps, double *acc, double *pot, void *ws, size_t ws_bytes,
                          const nb_opts *o) {
    NB_TRY(check_common(o, N, eps));
    NB_TRY(check_ptr(pos, "pos"));
    NB_TRY(check_ptr(mass, "mass"));
    NB_TRY(check_ptr(acc, "acc"));
    NB_TRY(check_ptr(pot, "pot", true));
    j->L = ws_layout(N, 1, o);
    NB_TRY(check_ws(ws, ws_bytes, j->L));
    if (o->precision != NB_PREC_FP64 && !resolve_shape(o, N, kKindForce, &j->shape))
        return fail(NB_ERR_UNSUPPORTED, "requested force kernel shape is not compiled");
    j->pos = pos;
    j->mass = mass;
    j->N = N;
    j->i0 = 0;
    j->ni = N;
    j->eps = eps;
    j->G = o->G;
    j->acc = acc;
    j->pot = pot;
    j->vel = nullptr;
    j->kick = 0.0;
    j->precision = o->precision;
    j->split = positions_split(o);
    j->adaptive = positions_adaptive(o, N);
    j->reuse_order = false;
    j->gamma = o->near_gamma > 0.f ? o->near_gamma : kNearFarGamma;
    j->packed_ready = false;
    // the default takes the symmetric path only where it applies (eps > 0);
    // an explicit NB_PAIRS_SYMMETRIC with eps = 0 is refused by the launcher
    j->sym = sym_wanted(o, N, 1) && (eps > 0.0 || o->pairs == NB_PAIRS_SYMMETRIC);
    j->timeout = timeout_of(o);
    j->unissued = unissued_of(o);
    j->stream = (cudaStream_t)o->stream;
    j->ws = (char *)ws;
    return NB_OK;
}

// ------------------------------------------------------- graph cache
struct GraphKey {
    nb_state s;
    double dt;
    int64_t nsteps;
    nb_opts o;
    nb_tune t;
    int device;
};
struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;
constexpr size_t kMaxGraphs = 16;

static bool same_key(const GraphKey &a, const GraphKey &b) {
    return memcmp(&a, &b, sizeof(GraphKey)) == 0;
}

}  // namespace nb

using namespace nb;

// =================================================================== ABI
extern "C" {

void nb_opts_default(nb_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = NB_PREC_F64ACC;
    o->G = 1.0;
}

const char *nb_version(void) {
    return "nbody-gb300 1.1 (sm_103a; FP32 pairs, direct or symmetric (each unordered pair "
           "once), with FP32/Kahan/FP64 accumulation; FP64 pairs)";
}

const char *nb_last_error(void) { return g_err; }

int nb_check_fp_conversions(int64_t n, uint64_t seed, int64_t *mismatches) {
    clear_error();
    if (!mismatches || n < 0) return fail(NB_ERR_INVALID, "need mismatches != NULL and n >= 0");
    // splitmix64 (Steele, Lea and Flood, 2014) for the random bit patterns
    uint64_t z = seed;
    auto next = [&z]() {
        uint64_t x = (z += 0x9e3779b97f4a7c15ull);
        x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
        x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
        return x ^ (x >> 31);
    };
    int64_t bad = 0;
    auto check_f = [&](uint32_t b) {
        const float f = fpconv::from_bits_f(b);
        const double want = (double)f, got = fpconv::f2d(f);
        const bool same = fpconv::bits_d(got) == fpconv::bits_d(want) || (want != want && got != got);
        if (!same) ++bad;
    };
    auto check_d = [&](uint64_t b) {
        const double d = fpconv::from_bits_d(b);
        if (fpconv::finite_d(d) != (bool)std::isfinite(d)) ++bad;
        const float want = (float)d, got = fpconv::d2f(d);
        if (!(fpconv::bits_f(got) == fpconv::bits_f(want) || (want != want && got != got))) ++bad;
    };
    // every exponent with edge significands, then random patterns
    for (uint32_t e = 0; e < 256; ++e)
        for (uint32_t m : {0u, 1u, 2u, 0x400000u, 0x3fffffu, 0x7fffffu, 0x123456u})
            for (uint32_t sg : {0u, 1u}) check_f((sg << 31) | (e << 23) | m);
    // every double exponent with significands at and around the float
    // rounding boundaries (ties at 2^28 below the kept bits, just below,
    // odd and even kept parts, all ones)
    for (uint64_t e = 0; e < 2048; ++e)
        for (uint64_t m : {0ull, 1ull, 0x10000000ull, 0x0fffffffull, 0x30000000ull, 0x20000000ull,
                           0xffffff0000000ull, 0xfffffe0000000ull | 0x10000000ull,
                           0xfffffffffffffull})
            for (uint64_t sg : {0ull, 1ull}) check_d((sg << 63) | (e << 52) | m);
    for (int64_t k = 0; k < n; ++k) {
        const uint64_t r = next();
        check_f((uint32_t)r);
        check_f((uint32_t)(r >> 32));
        check_f((uint32_t)(r >> 16) & 0x807fffffu);  // subnormals and zeros
        check_d(r);
        // doubles around the float range with tie and near-tie significands
        const uint64_t e = 1023 - 160 + (r >> 56) % 300;
        const uint64_t t = (r >> 3) & 3;
        const uint64_t m = (r & 0xfffffe0000000ull) |
                           (t == 0 ? 0x10000000ull : t == 1 ? 0x0fffffffull : (r & 0x1fffffffull));
        check_d((r & 0x8000000000000000ull) | (e << 52) | m);
    }
    // the fixed-point split of FP64 partials: hi 2^40 + lo (two's
    // complement) is v 2^F rounded half away from zero, or nothing past 2^100
    auto check_split = [&](double v, int F) {
        unsigned long long hi, lo;
        const bool ok = fx::split_f64(v, F, hi, lo);
        const double X = std::ldexp(v, F);  // exact: a power-of-two scaling
        if (!std::isfinite(v) || !(std::fabs(X) < 0x1p100)) {
            if (ok && std::isfinite(v) && std::fabs(X) < 0x1p100) ++bad;
            if (!std::isfinite(v) && ok) ++bad;
            return;
        }
        if (!ok) { ++bad; return; }
        const double ax = std::fabs(X);
        unsigned __int128 ref;
        if (ax >= 0x1p52)
            ref = (unsigned __int128)ax;            // already an integer
        else
            ref = (unsigned __int128)std::floor(ax + 0.5);  // exact below 2^52
        const __int128 got = (__int128)(long long)hi * ((__int128)1 << fx::kLoBits) + (__int128)lo;
        const __int128 want = std::signbit(v) ? -(__int128)ref : (__int128)ref;
        if (got != want) ++bad;
    };
    for (int F : {-900, -60, -1, 0, 1, 40, 60, 99, 120, 900})
        for (double v : {0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 1.5, 2.5, -2.5, 0x1p-1074, 1e300, -1e-300,
                         0x1p99, 0x1.fffffffffffffp99, 0x1p100, 3.0 * 0x1p-60, 0x1p-61})
            check_split(v, F);
    for (int64_t k = 0; k < n; ++k) {
        const uint64_t r = next();
        const int F = (int)(next() % 301) - 150;
        // magnitudes around the grid and the bound of that F
        const uint64_t e = (uint64_t)(1023 - F - 60 + (int)((r >> 56) % 170));
        check_split(fpconv::from_bits_d((r & 0x800fffffffffffffull) | ((e & 0x7ff) << 52)), F);
    }
    *mismatches = bad;
    return NB_OK;
}

unsigned long long nb_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int nb_kernel_timing(int32_t enable) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_tm_mu);
    if (enable) {
        // events of an earlier device are released; this device's are reused
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
        if (dev != g_tm_dev && g_tm_dev >= 0) {
            for (auto &e : g_tm_ev) {
                cudaEventDestroy(e.first);
                cudaEventDestroy(e.second);
            }
            g_tm_ev.clear();
        }
        g_tm_dev = dev;
        g_tm_ms = 0.0;
        g_tm_count = 0;
        g_tm_head = g_tm_live = 0;
        g_tm_err = 0;
        g_tm_open = false;
    }
    g_tm_on = enable != 0;
    return NB_OK;
}

int nb_kernel_time(double *total_ms, int64_t *launches) {
    clear_error();
    if (!total_ms || !launches) return fail(NB_ERR_INVALID, "total_ms and launches are required");
    std::lock_guard<std::mutex> lk(g_tm_mu);
    *total_ms = 0.0;
    *launches = 0;
    if (g_tm_err) return fail(NB_ERR_CUDA, "a timing event could not be created, recorded or read");
    while (g_tm_live > 0) {
        if (timer_fold_oldest()) {
            g_tm_err = 1;
            return fail(NB_ERR_CUDA, "kernel timing events could not be read");
        }
    }
    *total_ms = g_tm_ms;
    *launches = g_tm_count;
    return NB_OK;
}

int nb_tune_valid(const nb_tune *t) {
    if (!t) return 0;
    nb_opts o;
    nb_opts_default(&o);
    o.tune = t;
    if (bsym_item_blocks(&o) == 0) return 0;
    Shape s;
    return resolve_shape(&o, 1 << 20, kKindForce, &s) ? 1 : 0;
}

size_t nb_workspace_bytes(int64_t N_total, int32_t B, const nb_opts *opts) {
    if (N_total < 1 || B < 1) return 0;
    return ws_layout(N_total, B, opts).total;
}

int nb_forces(const double *pos, const double *mass, int64_t N, double eps, double *acc,
              double *pot, void *ws, size_t ws_bytes, const nb_opts *opts) {
    clear_error();
    ForceJob j;
    NB_TRY(make_force_job(&j, pos, mass, N, eps, acc, pot, ws, ws_bytes, opts));
    return launch_force(j);
}

int nb_forces_range(const double *pos, const double *mass, int64_t N, int64_t i0, int64_t i1,
                    double eps, double *acc, double *pot, void *ws, size_t ws_bytes,
                    const nb_opts *opts) {
    clear_error();
    if (i0 < 0 || i1 <= i0 || i1 > N)
        return fail(NB_ERR_INVALID, "need 0 <= i0 < i1 <= N (got i0 = %lld, i1 = %lld, N = %lld)",
                    (long long)i0, (long long)i1, (long long)N);
    ForceJob j;
    NB_TRY(make_force_job(&j, pos, mass, N, eps, acc, pot, ws, ws_bytes, opts));
    j.i0 = i0;
    j.ni = i1 - i0;
    // rows of the whole system in particle order: the direct kernel, no
    // Hilbert sort (ADAPTIVE is taken as SPLIT)
    j.sym = false;
    j.adaptive = false;
    return launch_force(j);
}

int nb_kick_drift(double *pos, double *vel, const double *acc, int64_t n, double kick,
                  double drift, const nb_opts *o) {
    clear_error();
    if (!o) return fail(NB_ERR_INVALID, "opts is NULL");
    if (n < 1) return fail(NB_ERR_INVALID, "n must be >= 1");
    if (!isfinite(kick) || !isfinite(drift))
        return fail(NB_ERR_INVALID, "kick and drift must be finite");
    NB_TRY(check_ptr(pos, "pos"));
    NB_TRY(check_ptr(vel, "vel"));
    NB_TRY(check_ptr(acc, "acc"));
    return launch_kick_drift(pos, vel, acc, n, kick, drift, (cudaStream_t)o->stream);
}

int nb_forces_batched(const double *pos, const double *mass, const int64_t *offsets, int32_t B,
                      int64_t N, const double *eps, double *acc, double *pot, void *ws,
                      size_t ws_bytes, const nb_opts *o) {
    clear_error();
    if (!o) return fail(NB_ERR_INVALID, "opts is NULL");
    if (B < 1) return fail(NB_ERR_INVALID, "B must be >= 1");
    if (N < B) return fail(NB_ERR_INVALID, "N must be >= B (every cluster holds a particle)");
    if (N > (int64_t)1 << 30) return fail(NB_ERR_INVALID, "N above 2^30 is not supported");
    NB_TRY(check_ptr(pos, "pos"));
    NB_TRY(check_ptr(mass, "mass"));
    NB_TRY(check_ptr(offsets, "offsets"));
    NB_TRY(check_ptr(eps, "eps"));
    NB_TRY(check_ptr(acc, "acc"));
    NB_TRY(check_ptr(pot, "pot", true));
    if (!isfinite(o->G)) return fail(NB_ERR_INVALID, "G must be finite");
    if (o->precision < NB_PREC_FP32 || o->precision > NB_PREC_FP64)
        return fail(NB_ERR_INVALID, "unknown precision %d", o->precision);
    BatchedJob j{};
    j.L = ws_layout(N, B, o);
    NB_TRY(check_ws(ws, ws_bytes, j.L));
    j.mass = mass;
    j.offsets = offsets;
    j.B = B;
    j.eps = eps;
    j.G = o->G;
    j.pos = const_cast<double *>(pos);
    j.vel = nullptr;
    j.acc = acc;
    j.pot = pot;
    j.N = N;
    j.dt = 0.0;
    j.nsteps = 0;
    j.acc_valid = false;
    j.precision = o->precision;
    j.cluster = o->tune ? o->tune->cluster_ctas : 0;
    j.threads = o->tune ? o->tune->threads : 0;
    j.item_blocks = o->tune ? o->tune->item_blocks : 0;
    j.positions = o->positions;
    j.gamma = o->near_gamma;
    j.sym = bsym_wanted(o, N, B);
    j.timeout = timeout_of(o);
    j.unissued = unissued_of(o);
    j.stream = (cudaStream_t)o->stream;
    j.ws = (char *)ws;
    return launch_batched(j);
}

static int step_batched_direct(nb_state *s, double dt, int64_t nsteps, const nb_opts *o) {
    BatchedJob j{};
    j.L = ws_layout(s->N, s->B, o);
    NB_TRY(check_ws(s->ws, s->ws_bytes, j.L));
    j.mass = s->mass;
    j.offsets = s->offsets;
    j.B = s->B;
    j.eps = s->eps_b;
    j.G = o->G;
    j.pos = s->pos;
    j.vel = s->vel;
    j.acc = s->acc;
    j.pot = s->pot;
    j.N = s->N;
    j.dt = dt;
    j.nsteps = nsteps;
    j.acc_valid = s->acc_valid != 0;
    j.precision = o->precision;
    j.cluster = o->tune ? o->tune->cluster_ctas : 0;
    j.threads = o->tune ? o->tune->threads : 0;
    j.item_blocks = o->tune ? o->tune->item_blocks : 0;
    j.positions = o->positions;
    j.gamma = o->near_gamma;
    j.sym = bsym_wanted(o, s->N, s->B);
    j.timeout = timeout_of(o);
    j.unissued = unissued_of(o);
    j.stream = (cudaStream_t)o->stream;
    j.ws = (char *)s->ws;
    return launch_batched(j);
}

static int step_single_direct(nb_state *s, double dt, int64_t nsteps, const nb_opts *o) {
    ForceJob j;
    NB_TRY(make_force_job(&j, s->pos, s->mass, s->N, s->eps, s->acc, s->pot, s->ws, s->ws_bytes, o));
    j.adaptive = positions_adaptive(o, s->N, nsteps > 0);
    int64_t sorted_at = -1;  // step index of the last full Hilbert sort
    // the potential is evaluated only where the caller can see it: a
    // forces-only call (nsteps = 0) or the last step of the loop
    double *pot = s->pot;
    if (!s->acc_valid) {
        ForceJob f = j;
        f.pot = nsteps == 0 ? pot : nullptr;
        NB_TRY(launch_force(f));
        sorted_at = 0;
    }
    float *soa = reinterpret_cast<float *>(j.ws + j.L.packA);
    for (int64_t n = 0; n < nsteps; ++n) {
        // the adaptive path packs in Hilbert order inside launch_force
        NB_TRY(launch_kick_drift_pack(s->pos, s->vel, s->acc, s->mass, s->N, j.L.Np, dt,
                                      j.adaptive ? nullptr : soa, j.stream));
        ForceJob k = j;
        k.packed_ready = !j.adaptive;
        k.reuse_order = j.adaptive && sorted_at >= 0 && n + 1 - sorted_at < kResortEvery;
        if (j.adaptive && !k.reuse_order) sorted_at = n + 1;
        k.vel = s->vel;
        k.kick = 0.5 * dt;
        k.pot = n == nsteps - 1 ? pot : nullptr;
        NB_TRY(launch_force(k));
    }
    return NB_OK;
}

int nb_step(nb_state *s, double dt, int64_t nsteps, const nb_opts *o) {
    clear_error();
    if (!s) return fail(NB_ERR_INVALID, "state is NULL");
    if (!o) return fail(NB_ERR_INVALID, "opts is NULL");
    if (!isfinite(dt)) return fail(NB_ERR_INVALID, "dt must be finite");
    if (nsteps < 0) return fail(NB_ERR_INVALID, "nsteps must be >= 0");
    NB_TRY(check_ptr(s->pos, "state.pos"));
    NB_TRY(check_ptr(s->vel, "state.vel"));
    NB_TRY(check_ptr(s->mass, "state.mass"));
    NB_TRY(check_ptr(s->acc, "state.acc"));
    NB_TRY(check_ptr(s->pot, "state.pot", true));
    const bool batched = s->B > 1 || s->offsets;
    if (batched) {
        if (s->B < 1) return fail(NB_ERR_INVALID, "B must be >= 1");
        NB_TRY(check_ptr(s->offsets, "state.offsets"));
        NB_TRY(check_ptr(s->eps_b, "state.eps_b"));
        if (s->N < s->B) return fail(NB_ERR_INVALID, "N must be >= B");
        if (!isfinite(o->G)) return fail(NB_ERR_INVALID, "G must be finite");
        if (o->precision < NB_PREC_FP32 || o->precision > NB_PREC_FP64)
            return fail(NB_ERR_INVALID, "unknown precision %d", o->precision);
    } else {
        NB_TRY(check_common(o, s->N, s->eps));
    }
    auto run = [&]() {
        return batched ? step_batched_direct(s, dt, nsteps, o) : step_single_direct(s, dt, nsteps, o);
    };
    const bool graph = o->use_graph && o->stream != nullptr && nsteps > 0;
    if (!graph) {
        NB_TRY(run());
    } else {
        GraphKey key;
        memset(&key, 0, sizeof key);
        key.s.N = s->N;
        key.s.B = s->B;
        key.s.offsets = s->offsets;
        key.s.pos = s->pos;
        key.s.vel = s->vel;
        key.s.mass = s->mass;
        key.s.acc = s->acc;
        key.s.pot = s->pot;
        key.s.eps_b = s->eps_b;
        key.s.eps = s->eps;
        key.s.acc_valid = s->acc_valid;
        key.s.ws = s->ws;
        key.s.ws_bytes = s->ws_bytes;
        key.dt = dt;
        key.nsteps = nsteps;
        key.o.precision = o->precision;
        key.o.G = o->G;
        key.o.stream = o->stream;
        key.o.use_graph = o->use_graph;
        key.o.timeout_cycles = o->timeout_cycles;
        key.o.test_unissued_stage = o->test_unissued_stage;
        key.o.positions = o->positions;
        key.o.near_gamma = o->near_gamma;
        key.o.pairs = o->pairs;
        if (o->tune) {
            key.t.threads = o->tune->threads;
            key.t.i_per_thread = o->tune->i_per_thread;
            key.t.tile_j = o->tune->tile_j;
            key.t.stages = o->tune->stages;
            key.t.ctas_per_sm = o->tune->ctas_per_sm;
            key.t.cluster_ctas = o->tune->cluster_ctas;
            key.t.item_blocks = o->tune->item_blocks;
        }
        cudaGetDevice(&key.device);
        cudaGraphExec_t exec = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_graph_mu);
            for (auto &e : g_graphs)
                if (same_key(e.key, key)) exec = e.exec;
        }
        cudaStream_t st = (cudaStream_t)o->stream;
        if (!exec) {
            // The first call of a new configuration captures the loop (state
            // pointers, sizes and dt are baked into the graph).
            NB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int rc = run();
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (rc != NB_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return cuda_check(ce, "cudaStreamEndCapture");
            const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) return cuda_check(ie, "cudaGraphInstantiate");
            std::lock_guard<std::mutex> lk(g_graph_mu);
            if (g_graphs.size() >= kMaxGraphs) {
                cudaGraphExecDestroy(g_graphs.front().exec);
                g_graphs.erase(g_graphs.begin());
            }
            // the captured graph includes the priming force only if acc was invalid
            g_graphs.push_back(GraphEntry{key, exec});
        }
        NB_CUDA(cudaGraphLaunch(exec, st));
    }
    s->acc_valid = 1;
    s->step += nsteps;
    return NB_OK;
}

int nb_energy(const nb_state *s, double *out3, const nb_opts *o) {
    clear_error();
    if (!s || !o) return fail(NB_ERR_INVALID, "state or opts is NULL");
    if (s->N < 1) return fail(NB_ERR_INVALID, "N must be >= 1");
    NB_TRY(check_ptr(s->vel, "state.vel"));
    NB_TRY(check_ptr(s->mass, "state.mass"));
    NB_TRY(check_ptr(s->pot, "state.pot"));
    NB_TRY(check_ptr(out3, "out3"));
    WsLayout L = ws_layout(s->N, s->B < 1 ? 1 : s->B, o);
    NB_TRY(check_ws(s->ws, s->ws_bytes, L));
    return launch_energy(s->vel, s->mass, s->pot, s->N, out3, (char *)s->ws, L,
                         (cudaStream_t)o->stream);
}

static int make_vjp_job(VjpJob *j, const double *pos, const double *mass, int64_t N, double eps,
                        double *pos_bar, double *mass_bar, void *ws, size_t ws_bytes,
                        const nb_opts *o) {
    memset(j, 0, sizeof *j);
    NB_TRY(check_common(o, N, eps));
    NB_TRY(check_ptr(pos, "pos"));
    NB_TRY(check_ptr(mass, "mass"));
    NB_TRY(check_ptr(pos_bar, "pos_bar"));
    NB_TRY(check_ptr(mass_bar, "mass_bar"));
    j->L = ws_layout(N, 1, o);
    NB_TRY(check_ws(ws, ws_bytes, j->L));
    if (o->precision != NB_PREC_FP64 && !resolve_shape(o, N, kKindVjp, &j->shape))
        return fail(NB_ERR_UNSUPPORTED, "requested VJP kernel shape is not compiled");
    j->pos = pos;
    j->mass = mass;
    j->N = N;
    j->eps = eps;
    j->G = o->G;
    j->pos_bar = pos_bar;
    j->mass_bar = mass_bar;
    j->i0 = 0;
    j->ni = N;
    j->kick_coef = 1.0;
    j->precision = o->precision;
    // gradients are gated at 1e-4 (median) / 1e-3 (max): single-float
    // displacements unless the caller asks for the split form
    j->split = o->positions == NB_POS_SPLIT;
    j->timeout = timeout_of(o);
    j->unissued = unissued_of(o);
    j->stream = (cudaStream_t)o->stream;
    j->ws = (char *)ws;
    return NB_OK;
}

int nb_forces_vjp(const double *pos, const double *mass, int64_t N, double eps,
                  const double *acc_bar, const double *pot_bar, double *pos_bar, double *mass_bar,
                  void *ws, size_t ws_bytes, const nb_opts *o) {
    clear_error();
    VjpJob j;
    NB_TRY(make_vjp_job(&j, pos, mass, N, eps, pos_bar, mass_bar, ws, ws_bytes, o));
    NB_TRY(check_ptr(acc_bar, "acc_bar"));
    NB_TRY(check_ptr(pot_bar, "pot_bar", true));
    j.acc_bar = acc_bar;
    j.pot_bar = pot_bar;
    j.step_form = false;
    j.accumulate = false;
    return launch_vjp(j);
}

int nb_forces_vjp_range(const double *pos, const double *mass, int64_t N, int64_t i0, int64_t i1,
                        double eps, double coef, const double *acc_bar, const double *pot_bar,
                        double *pos_bar, double *mass_bar, void *ws, size_t ws_bytes,
                        const nb_opts *o) {
    clear_error();
    if (i0 < 0 || i1 <= i0 || i1 > N)
        return fail(NB_ERR_INVALID, "need 0 <= i0 < i1 <= N (got i0 = %lld, i1 = %lld, N = %lld)",
                    (long long)i0, (long long)i1, (long long)N);
    if (!isfinite(coef)) return fail(NB_ERR_INVALID, "coef must be finite");
    VjpJob j;
    NB_TRY(make_vjp_job(&j, pos, mass, N, eps, pos_bar, mass_bar, ws, ws_bytes, o));
    NB_TRY(check_ptr(acc_bar, "acc_bar"));
    NB_TRY(check_ptr(pot_bar, "pot_bar", true));
    j.acc_bar = acc_bar;
    j.pot_bar = pot_bar;
    j.kick_coef = coef;
    j.i0 = i0;
    j.ni = i1 - i0;
    j.step_form = false;
    j.accumulate = true;
    return launch_vjp(j);
}

int nb_step_vjp(const double *pos_k, const double *mass, int64_t N, double eps, double drift_dt,
                double kick_coef, double *pos_bar, double *vel_bar, double *mass_bar, void *ws,
                size_t ws_bytes, const nb_opts *o) {
    clear_error();
    VjpJob j;
    NB_TRY(make_vjp_job(&j, pos_k, mass, N, eps, pos_bar, mass_bar, ws, ws_bytes, o));
    NB_TRY(check_ptr(vel_bar, "vel_bar"));
    if (!isfinite(drift_dt) || !isfinite(kick_coef))
        return fail(NB_ERR_INVALID, "drift_dt and kick_coef must be finite");
    j.step_form = true;
    j.drift_dt = drift_dt;
    j.kick_coef = kick_coef;
    j.vel_bar = vel_bar;
    j.accumulate = true;
    return launch_vjp(j);
}

int nb_step_vjp_reverse(double *pos, double *vhalf, double *acc, const double *mass, int64_t N,
                        double eps, double rewind_kick, double rewind_drift, double drift_dt,
                        double kick_coef, double *pos_bar, double *vel_bar, double *mass_bar,
                        void *ws, size_t ws_bytes, const nb_opts *o) {
    clear_error();
    VjpJob j;
    NB_TRY(make_vjp_job(&j, pos, mass, N, eps, pos_bar, mass_bar, ws, ws_bytes, o));
    NB_TRY(check_ptr(vel_bar, "vel_bar"));
    NB_TRY(check_ptr(vhalf, "vhalf"));
    NB_TRY(check_ptr(acc, "acc"));
    if (!isfinite(drift_dt) || !isfinite(kick_coef) || !isfinite(rewind_kick) ||
        !isfinite(rewind_drift))
        return fail(NB_ERR_INVALID, "step coefficients must be finite");
    j.step_form = true;
    j.drift_dt = drift_dt;
    j.kick_coef = kick_coef;
    j.vel_bar = vel_bar;
    j.accumulate = true;
    j.acc_out = acc;
    j.vhalf = vhalf;
    j.pos_rw = pos;
    j.rewind_kick = rewind_kick;
    j.rewind_drift = rewind_drift;
    return launch_vjp(j);
}

static int make_jerk_job(JerkJob *j, double *pos, double *vel, const double *mass, int64_t N,
                         double eps, double *acc, double *jerk, double *pot, void *ws,
                         size_t ws_bytes, const nb_opts *o) {
    memset(j, 0, sizeof *j);
    NB_TRY(check_common(o, N, eps));
    NB_TRY(check_ptr(pos, "pos"));
    NB_TRY(check_ptr(vel, "vel"));
    NB_TRY(check_ptr(mass, "mass"));
    NB_TRY(check_ptr(acc, "acc"));
    NB_TRY(check_ptr(jerk, "jerk"));
    NB_TRY(check_ptr(pot, "pot", true));
    j->L = ws_layout(N, 1, o);
    NB_TRY(check_ws(ws, ws_bytes, j->L));
    j->pos = pos;
    j->vel = vel;
    j->mass = mass;
    j->N = N;
    j->eps = eps;
    j->G = o->G;
    j->acc = acc;
    j->jerk = jerk;
    j->pot = pot;
    j->precision = o->precision;
    j->timeout = timeout_of(o);
    j->unissued = unissued_of(o);
    j->stream = (cudaStream_t)o->stream;
    j->ws = (char *)ws;
    return NB_OK;
}

int nb_forces_jerk(const double *pos, const double *vel, const double *mass, int64_t N,
                   double eps, double *acc, double *jerk, double *pot, void *ws, size_t ws_bytes,
                   const nb_opts *o) {
    clear_error();
    JerkJob j;
    NB_TRY(make_jerk_job(&j, const_cast<double *>(pos), const_cast<double *>(vel), mass, N, eps,
                         acc, jerk, pot, ws, ws_bytes, o));
    j.nsteps = 0;
    return launch_jerk(j);
}

int nb_hermite4(double *pos, double *vel, const double *mass, int64_t N, double eps, double *acc,
                double *jerk, int32_t acc_valid, double dt, int64_t nsteps, void *ws,
                size_t ws_bytes, const nb_opts *o) {
    clear_error();
    if (!isfinite(dt)) return fail(NB_ERR_INVALID, "dt must be finite");
    if (nsteps < 0) return fail(NB_ERR_INVALID, "nsteps must be >= 0");
    JerkJob j;
    NB_TRY(make_jerk_job(&j, pos, vel, mass, N, eps, acc, jerk, nullptr, ws, ws_bytes, o));
    if (!acc_valid) {
        JerkJob e = j;
        e.nsteps = 0;
        NB_TRY(launch_jerk(e));
    }
    if (nsteps == 0) return NB_OK;
    j.h = dt;
    j.nsteps = nsteps;
    return launch_jerk(j);
}

int nb_poll_status(void *ws, size_t ws_bytes, void *stream) {
    clear_error();
    if (!ws) {
        // the status word of nb_forces_noalloc's fixed array on this device
        uint32_t *word_dev = nullptr;
        NB_TRY(noalloc_status_word(&word_dev));
        ws = word_dev;
    } else if (ws_bytes < 256) {
        return fail(NB_ERR_INVALID, "workspace too small");
    }
    NB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t word = 0;
    NB_CUDA(cudaMemcpy(&word, ws, sizeof word, cudaMemcpyDeviceToHost));
    if (word) NB_CUDA(cudaMemset(ws, 0, sizeof word));
    if (word & kStatusTimeout) return fail(NB_ERR_TIMEOUT, "a device wait ran out of time");
    if (word & kStatusInvalid) return fail(NB_ERR_INVALID, "the device rejected an argument");
    if (word & kStatusNonFinite) return fail(NB_ERR_NONFINITE, "a non-finite value was produced");
    return NB_OK;
}

}  // extern "C"
