// Internal declarations shared by the library's translation units.
// Not part of the ABI: the public surface is include/nbody.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbody.h"

namespace nb {

// ---------------------------------------------------------------- errors
// Records a message for nb_last_error() and returns `code`.
int fail(int code, const char *fmt, ...);
void clear_error();
int cuda_check(cudaError_t e, const char *what);
#define NB_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return nb::cuda_check(e_, #call); \
    } while (0)

// Device status word bits (latched with atomicOr, read by nb_poll_status).
constexpr uint32_t kStatusTimeout = 1u << NB_ERR_TIMEOUT;
constexpr uint32_t kStatusNonFinite = 1u << NB_ERR_NONFINITE;
constexpr uint32_t kStatusInvalid = 1u << NB_ERR_INVALID;

constexpr long long kDefaultTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------------------- launch shapes
// Shape of the FP32-pair stream-K force kernels (nb_tune resolved).
struct Shape {
    int threads;      // NT
    int ipt;          // i-particles per thread (IR)
    int tile_j;       // TJ
    int stages;       // ST
    int ctas_per_sm;  // persistent CTAs per SM
    int block_i() const { return threads * ipt; }
};

// Shape used for N particles when the caller gives no (or a partial) tune.
Shape default_shape(int64_t N, int precision, int kind);
// Resolves opts->tune against the defaults; returns false if not compiled.
bool resolve_shape(const nb_opts *opts, int64_t N, int kind, Shape *out);
bool shape_compiled(const Shape &s, int kind);
enum Kind { kKindForce = 0, kKindVjp = 1 };

int device_sm_count();
// Raises `kernel`'s dynamic shared-memory limit to `bytes` on the current
// device, once per kernel, device and size (thread-safe); a failure is
// returned as NB_ERR_CUDA.
int smem_optin(const void *kernel, size_t bytes);
// Counts kernels this library enqueued (nb_launch_count); a CUDA-graph
// replay launches the captured kernels without passing through here.
void count_launch(int n = 1);
// Opt-in CUDA-event timing of the symmetric FP32 pair kernel
// (nb_kernel_timing): events recorded on `st` just before and after its
// launch; no-ops when timing is off or `st` is being captured.
void kernel_timer_begin(cudaStream_t st);
void kernel_timer_end(cudaStream_t st);
// Resident CTAs per SM of `kernel` (>= 1), and the persistent grid size:
// min(requested CTAs per SM, occupancy) x SMs, capped at `total` items.
int occupancy(const void *kernel, int threads, size_t smem);
int persistent_grid(int cps, int occ, int64_t total);

// --------------------------------------------------------- workspace
// Byte offsets inside the caller's workspace.  Everything is 256-B aligned.
struct WsLayout {
    size_t status;    // uint32 status word (+ padding to 256 B)
    size_t counters;  // uint32 arrival counters, one per i-block
    size_t packA;     // float SoA [7][Np]: x.hi y.hi z.hi m x.lo y.lo z.lo
    size_t packB;     // float SoA [4][Np]: VJP cotangents (cx, cy, cz, pbar/3)
    size_t cot64;     // double SoA [4][Np]: the same cotangents in FP64
    size_t sortbuf;   // Hilbert keys, permutation, tile/block boxes (adaptive path)
    size_t records;   // stream-K partial records
    size_t scratch;   // O(N) reduction scratch (energy partials, batched queue)
    size_t sym_fx;    // symmetric-pair path: fixed-point totals, 64 B per slot
    size_t sym_cost;  // symmetric-pair path: exponent, item costs, their prefix, CTA ranges
    size_t bsym, bsym_bytes;  // batched symmetric-pair path (0 bytes: not provisioned)
    size_t sym_fx_bytes;      // 0 when the symmetric path is not provisioned
    size_t total;
    int64_t Np;       // padded particle count of the pack arrays
    int64_t max_blocks;
    int64_t max_grid;
    int64_t record_bytes_per_i;
};

WsLayout ws_layout(int64_t N, int32_t B, const nb_opts *opts);
int check_ws(const void *ws, size_t ws_bytes, const WsLayout &L);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Stream-K split: CTA c of C owns linear work items [lo(c), lo(c+1)) of T.
__host__ __device__ inline int64_t sk_lo(int64_t T, int64_t C, int64_t c) { return T * c / C; }
// The CTA whose range holds item t (0 <= t < T).
__host__ __device__ inline int64_t sk_owner(int64_t T, int64_t C, int64_t t) {
    return ((t + 1) * C - 1) / T;
}

// ----------------------------------------------------- kernel launchers
struct ForceJob {
    const double *pos;
    const double *mass;
    int64_t N;
    int64_t i0, ni;     // rows: particles i0 .. i0 + ni - 1 (all N: 0, N); acc/pot
                        // hold ni rows.  A strict sub-range takes the direct kernel.
    double eps;
    double G;
    double *acc;
    double *pot;
    // optional fused closing half-kick: vel += kick * acc
    double *vel;
    double kick;
    int precision;
    bool split;         // hi/lo displacement (nb_positions resolved)
    bool adaptive;      // Hilbert-sorted pack, hi/lo only for near tile pairs
    bool reuse_order;   // adaptive: keep the previous call's Hilbert order
    float gamma;        // near/far threshold of the adaptive path
    bool packed_ready;  // packA already holds float positions of `pos`
    bool sym;           // symmetric-pair evaluation (nb_pairs resolved)
    long long timeout;
    int64_t unissued;  // test hook (nb_opts.test_unissued_stage - 1; -1: off)
    cudaStream_t stream;
    char *ws;
    WsLayout L;
    Shape shape;
};

// Resolves nb_opts::positions for a precision: true = split hi/lo.
bool positions_split(const nb_opts *opts);
// true when the split displacement is applied only to near tile pairs of a
// Hilbert-sorted pack (explicit NB_POS_ADAPTIVE, or the default for the
// KAHAN and F64ACC policies from N >= 2^16 for one evaluation and from
// N >= 2^15 for a step loop; 1/64 is the default near_gamma).
bool positions_adaptive(const nb_opts *opts, int64_t N, bool stepping = false);
// Steps of one nb_step call between full re-sorts of the adaptive path.
constexpr int64_t kResortEvery = 16;

// Well-separated threshold of the adaptive path: a (warp, 64-particle
// sub-tile) pair takes the single-float displacement when the gap between
// their boxes is at least gamma times the largest coordinate magnitude in
// either box (per-pair relative displacement error <= ~sqrt(3) u / gamma,
// u = 2^-24).  On the 2^20 Plummer and 65536 / 262144 log-normal workloads
// the maximum relative acceleration error stayed at 1.2-2.9e-6 for every
// gamma from 1/16 to 1/512; 1/64 is the smallest power of two whose
// per-pair bound (6.6e-6) stays below the 1e-5 gate, so that a particle
// whose acceleration one pair at the threshold dominates still meets it.
constexpr float kNearFarGamma = 0.015625f;

// Sub-buffers of WsLayout::sortbuf.
int64_t sort_keys_len(int64_t N);
inline unsigned long long *sort_keys(char *sb) { return reinterpret_cast<unsigned long long *>(sb); }
inline int *sort_perm(char *sb, const WsLayout &L) {
    return reinterpret_cast<int *>(sb + 8 * sort_keys_len(L.Np));
}
inline float *sort_tile_boxes(char *sb, const WsLayout &L) {
    return reinterpret_cast<float *>(sb + 8 * sort_keys_len(L.Np) + 4 * L.Np);
}
inline float *sort_block_boxes(char *sb, const WsLayout &L) {
    return sort_tile_boxes(sb, L) + 8 * (L.Np / 32 + 1);
}
inline long long *sort_box6(char *sb, const WsLayout &L) {
    return reinterpret_cast<long long *>(sort_block_boxes(sb, L) + 8 * (L.Np / 32 + 1));
}
inline size_t sortbuf_bytes(int64_t Np) {
    return 8 * (size_t)sort_keys_len(Np) + 4 * (size_t)Np + 32 * (size_t)(Np / 32 + 1) +
           32 * (size_t)(Np / 32 + 1) + 64;
}
// reuse_order: the keys already hold a Hilbert order of these N particles
// (an earlier call of the same step loop); only the pack and the boxes are
// redone from the current positions.
int launch_sorted_pack(const double *pos, const double *mass, int64_t N, int64_t Np, float *soa,
                       int *perm, unsigned long long *keys, long long *box6, float *tile_boxes,
                       int tile_unit, float *block_boxes, int block_unit, bool reuse_order,
                       cudaStream_t st);

// Number of float arrays of Np entries in a packed position buffer.
constexpr int kPackArrays = 7;

// Writes particle i of the packed SoA: x.hi y.hi z.hi m x.lo y.lo z.lo.
__host__ __device__ inline void store_packed(float *soa, int64_t Np, int64_t i, const float hi[3],
                                             const float lo[3], float m) {
    soa[i] = hi[0];
    soa[Np + i] = hi[1];
    soa[2 * Np + i] = hi[2];
    soa[3 * Np + i] = m;
    soa[4 * Np + i] = lo[0];
    soa[5 * Np + i] = lo[1];
    soa[6 * Np + i] = lo[2];
}

int launch_pack(const double *pos, const double *mass, int64_t N, int64_t Np, float *soa,
                cudaStream_t st);
int launch_force(const ForceJob &job);

// ------------------------------------------------- symmetric-pair path
// Row blocks of 2048 slots; items are the block pairs (I, J >= I).
constexpr int64_t kSymBlock = 2048;
// Default size range of the symmetric-pair path (its scratch is O(N): 64 B
// per particle of fixed-point totals, 268 MB at N = 2^22, plus 12 B per
// block pair of cost estimates, 25 MB at 2^22, 400 MB at 2^24).  Below the
// lower end the direct kernel is faster (Kahan evaluation, direct /
// symmetric: 0.185 / 0.232 ms at 16384, 0.386 / 0.365 at 24576, 0.673 /
// 0.552 at 32768).
constexpr int64_t kSymMinN = 24576;
constexpr int64_t kSymMaxN = 1 << 24;
struct SymSizes {
    int64_t nb, T, U, ctas;  // row blocks, items, stream-K units, CTAs
    size_t fx_bytes, cost_bytes;
};
SymSizes sym_sizes(int64_t Np);
// Pointers into the symmetric path's workspace regions.
struct SymLayout {
    int *fx_exp;                   // fixed-point exponent of the call
    unsigned long long *mmax_bits; // max |m| while it is reduced (zero between calls)
    unsigned *arrivals;            // blocks done with the reduction (zero between calls)
    uint32_t *cost;                // per item
    unsigned long long *prefix;    // [T + 1]
    int64_t *lo;                   // [ctas + 1] stream-K range starts
    unsigned long long *acc_fx;    // [4][2][Np]
};
SymLayout sym_layout(char *ws, const WsLayout &L);
// Whether the symmetric-pair path is provisioned / taken for N particles in
// B clusters under opts (nb_pairs; FP32-pair policies, single systems).
bool sym_wanted(const nb_opts *opts, int64_t N, int32_t B);
int launch_force_sym(const ForceJob &job, bool adaptive);

struct VjpJob {
    const double *pos;
    const double *mass;
    int64_t N;
    double eps;
    double G;
    // cotangent inputs (nb_forces_vjp form) ...
    const double *acc_bar;
    const double *pot_bar;
    // ... or the step-adjoint form: c = kick_coef * (vel_bar += drift_dt * pos_bar)
    bool step_form;
    double drift_dt;
    double kick_coef;
    double *vel_bar;
    // outputs: rows [i0, i0 + ni) of the N particles (pos_bar [ni][3],
    // mass_bar [ni]); the step forms take all of them
    double *pos_bar;
    double *mass_bar;
    int64_t i0, ni;
    bool accumulate;  // add into pos_bar/mass_bar instead of overwriting
    // optional fused force + reverse drift (nb_step_vjp_reverse)
    double *acc_out;
    double *vhalf;
    double *pos_rw;
    double rewind_kick;
    double rewind_drift;
    int precision;
    bool split;  // hi/lo displacement (the VJP's default is single floats)
    long long timeout;
    int64_t unissued;  // test hook (nb_opts.test_unissued_stage - 1; -1: off)
    cudaStream_t stream;
    char *ws;
    WsLayout L;
    Shape shape;
};
int launch_vjp(const VjpJob &job);

int launch_kick_drift_pack(double *pos, double *vel, const double *acc, const double *mass,
                           int64_t N, int64_t Np, double dt, float *soa, cudaStream_t st);
// v += kick a; x += drift v for n particles (FP64).
int launch_kick_drift(double *pos, double *vel, const double *acc, int64_t n, double kick,
                      double drift, cudaStream_t st);
int launch_energy(const double *vel, const double *mass, const double *pot, int64_t N,
                  double *out3, char *ws, const WsLayout &L, cudaStream_t st);

struct JerkJob {
    double *pos;
    double *vel;
    const double *mass;
    int64_t N;
    double eps;
    double G;
    double *acc;
    double *jerk;
    double *pot;
    double h;
    int64_t nsteps;  // 0 = evaluate a, jerk, phi at the current state
    int precision;
    long long timeout;
    int64_t unissued;  // test hook (nb_opts.test_unissued_stage - 1; -1: off)
    cudaStream_t stream;
    char *ws;
    WsLayout L;
};
int launch_jerk(const JerkJob &job);

struct BatchedJob {
    const double *mass;
    const int64_t *offsets;
    int32_t B;
    const double *eps;
    double G;
    double *pos;
    double *vel;
    double *acc;
    double *pot;
    int64_t N;
    double dt;
    int64_t nsteps;   // 0 = forces only
    bool acc_valid;
    int precision;
    int cluster;      // CTAs per thread-block cluster (0 = default)
    int threads;      // threads per CTA (0 = default)
    int item_blocks;  // symmetric path: j-blocks per work item (0 = default)
    int positions;    // nb_positions: SPLIT = hi/lo everywhere, else adaptive
    float gamma;      // near/far threshold (0 = default)
    bool sym;         // symmetric pairs (nb_pairs resolved)
    long long timeout;
    int64_t unissued;  // test hook (nb_opts.test_unissued_stage - 1; -1: off)
    cudaStream_t stream;
    char *ws;
    WsLayout L;
};
int launch_batched(const BatchedJob &job);
size_t batched_scratch_bytes(int32_t B);

// Batched symmetric-pair path (nb_bsym.cu): the workspace region's layout for
// N particles in B systems cut into items of up to g j-blocks (bounds from
// N, B and g only); g = bsym_item_blocks(opts) is 2, 4 or 8, 0 if the tune
// asks for another width.
struct BsymLayout {
    int64_t Ns, blocks, items, pairs;
    size_t o_sbase, o_ibase, o_pbase, o_rstart, o_bsys, o_bmeta, o_items, o_order, o_misc, o_soa, o_perm,
        o_box32, o_P, o_rec, o_st0, o_st1, o_pots, bytes;
};
BsymLayout bsym_layout(int64_t N, int32_t B, int g);
int bsym_item_blocks(const nb_opts *opts);
bool bsym_wanted(const nb_opts *opts, int64_t N, int32_t B);
int launch_batched_sym(const BatchedJob &job);

// Device address of nb_forces_noalloc's status word on the current device.
int noalloc_status_word(uint32_t **out);

}  // namespace nb
