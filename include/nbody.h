/*
 * nbody.h -- C ABI of the GB300 (sm_103a) direct-summation N-body library.
 *
 * The library evaluates the all-pairs softened Newtonian acceleration and
 * potential (Eq. 1 of Sec. 2.1, divided by m_i; softening "included in the
 * distance computation" as in App. A, taken here as r^2 + eps^2), advances
 * particles with kick-drift-kick leapfrog, and differentiates both.
 *
 *   a_i   =  G sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2}
 *   phi_i = -G sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^{1/2}
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory:   every array argument is a DEVICE pointer owned by the caller,
 *           8-byte aligned (256-byte for the workspace), C-contiguous.  The
 *           library never allocates or frees device memory; scratch space is
 *           the caller's workspace `ws` of `ws_bytes` bytes, sized with
 *           nb_workspace_bytes() and ZERO-FILLED once before its first use
 *           (the kernels leave their arrival counters at zero on exit, so
 *           later calls need no clearing unless a call reported
 *           NB_ERR_TIMEOUT).  One workspace serves one stream at a time.
 * Layout:   positions, velocities, accelerations and their cotangents are
 *           double [N][3] row-major; masses, potentials and their cotangents
 *           double [N].  Batched sets concatenate clusters and describe them
 *           with CSR offsets int64 [B+1] (offsets[0] = 0, offsets[B] = N).
 * Streams:  all work is enqueued asynchronously on opts->stream (a
 *           cudaStream_t; NULL = the legacy default stream).  Calls return
 *           after enqueueing.
 * Errors:   a call returns NB_OK or an NB_ERR_* code.  Argument errors are
 *           detected on the host before anything is enqueued.  Errors found
 *           on the device (a bounded wait that ran out, a non-finite result)
 *           are latched in a status word inside `ws`; nb_poll_status() reads
 *           and clears it.  nb_last_error() gives a message for the last
 *           failing call on the calling host thread.
 * Precision: inputs and outputs are always double.  opts->precision picks
 *           the arithmetic of the pair loop: FP32 pairs with FP32, Kahan-
 *           compensated FP32 or FP64 per-particle accumulation, or FP64
 *           pairs.  The paper's device arithmetic is FP32 with the host in
 *           FP64 (Sec. 3.1); the O(N) state updates here are FP64 on the GPU.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define NB_OK              0
#define NB_ERR_INVALID     1  /* bad argument (size, pointer, alignment, value) */
#define NB_ERR_CUDA        2  /* a CUDA runtime call failed                     */
#define NB_ERR_WORKSPACE   3  /* ws_bytes smaller than nb_workspace_bytes()     */
#define NB_ERR_UNSUPPORTED 4  /* valid request this build cannot serve          */
#define NB_ERR_TIMEOUT     5  /* a device wait exceeded opts->timeout_cycles    */
#define NB_ERR_NONFINITE   6  /* a non-finite value was produced                */

/* ---- pair-loop precision policies ------------------------------------ */
typedef enum {
    NB_PREC_FP32 = 0,   /* FP32 pairs, FP32 running sums                      */
    NB_PREC_KAHAN = 1,  /* FP32 pairs, per-tile FP32 sums Kahan-added         */
    NB_PREC_F64ACC = 2, /* FP32 pairs, per-tile FP32 sums added in FP64       */
    NB_PREC_FP64 = 3    /* FP64 pairs and sums                                */
} nb_precision;

/* How the FP32-pair kernels form the displacement x_j - x_i.  SPLIT keeps
 * each coordinate as an unevaluated sum hi + lo of two floats (hi = x
 * rounded to FP32, lo = the rounding remainder) and forms
 * (x_j.hi - x_i.hi) + (x_j.lo - x_i.lo), so close pairs far from the
 * origin keep ~1e-7 relative accuracy (6 more FP32 operations per pair).
 * SINGLE rounds positions to FP32 once, as the paper's device kernel does
 * (Sec. 3.1); its displacement error is ~6e-8 |x| / |x_j - x_i|, which
 * reaches ~1e-4 relative acceleration error for close pairs at N = 2^20. */
typedef enum {
    NB_POS_DEFAULT = 0, /* KAHAN/F64ACC: SPLIT below N = 65536 (32768 in
                           an nb_step loop), ADAPTIVE from there; FP32:
                           SINGLE                                          */
    NB_POS_SPLIT = 1,
    NB_POS_SINGLE = 2,
    NB_POS_ADAPTIVE = 3 /* particles sorted along a Hilbert curve each call;
                           SPLIT for tile pairs whose bounding boxes are
                           closer than near_gamma (default 1/64; 1/256 on
                           the batched symmetric path) times their largest
                           coordinate, SINGLE for the rest                 */
} nb_positions;

/* How the pairs of one system (nb_forces, nb_step with B = 1) are evaluated
 * by the FP32-pair policies.  DIRECT evaluates every ordered pair (i, j)
 * once for particle i.  SYMMETRIC evaluates every unordered pair once and
 * applies it to both particles: the pair term of Eq. 1 changes sign under
 * i <-> j apart from the masses, so d, r^2 and r^-3 serve a_i and a_j
 * (about 9 FP32 operations per directed interaction instead of 13).  It
 * needs eps > 0.  The partial sums that several CTAs produce for one
 * particle are combined in two-word fixed point with integer atomic adds
 * (exact, so the result does not depend on their order), which takes 64 B
 * per particle of workspace plus 12 B per pair of 2048-particle blocks
 * (about 69 MB at N = 2^20), included by nb_workspace_bytes when the path is
 * in use.  The fixed-point grid is 2^-100 of the a-priori bound
 * N max|m| max(0.385 / eps^2, 1 / eps) on every acceleration component and
 * potential; it is finer than FP64 rounding unless that bound exceeds the
 * smallest |a_i| by more than ~10^14.  DEFAULT takes SYMMETRIC for
 * 24576 <= N <= 2^24 and eps > 0 (FP32 and FP64 pairs), DIRECT otherwise.
 * For batches (B > 1, nb_forces_batched and
 * nb_step with offsets) DEFAULT and SYMMETRIC take the symmetric batched
 * path (warp-granular work items; workspace about 250 B per particle plus
 * 2 KiB per pair of 128-particle blocks of a cluster, provisioned for 64
 * such pairs per block: 1.4 GB for the 512 clusters of 64 to 8192) and
 * DIRECT the persistent direct-pair kernel
 * (nb_tune's cluster_ctas / threads).  Results of both are deterministic;
 * they differ from each other by summation order only. */
typedef enum {
    NB_PAIRS_DEFAULT = 0,
    NB_PAIRS_DIRECT = 1,
    NB_PAIRS_SYMMETRIC = 2
} nb_pairs;

/* Launch shape of the FP32-pair kernels.  Zero fields take the built-in
 * defaults for the problem size; nb_tune_valid() reports whether a shape
 * is one this build was compiled for. */
typedef struct nb_tune {
    int32_t threads;      /* threads per CTA: 128..1024 (batched: 256/512) */
    int32_t i_per_thread; /* i-particles held in registers per thread: 1,2,4,8 */
    int32_t tile_j;       /* j-particles per shared-memory stage: 64..512   */
    int32_t stages;       /* depth of the bulk-copy ring: 2..4               */
    int32_t ctas_per_sm;  /* persistent CTAs per SM: 1..4                    */
    int32_t cluster_ctas; /* batched kernel: CTAs per thread-block cluster, 2/4/8 */
    int32_t item_blocks;  /* batched symmetric path: 128-particle j-blocks per
                             work item, 2/4/8 (0 = 8).  Smaller items balance
                             the queue's tail but write more 4 KiB FP64
                             records: the workspace provisions 6, 10 or 18
                             items per 128 particles for 8, 4 or 2; other
                             values are refused (NB_ERR_INVALID) */
} nb_tune;

typedef struct nb_opts {
    int32_t precision;      /* nb_precision                                   */
    double G;               /* gravitational constant (units: G = 1 usual)    */
    void *stream;           /* cudaStream_t or NULL                            */
    int32_t use_graph;      /* nb_step: replay the step loop as a CUDA graph  */
    const nb_tune *tune;    /* NULL = defaults                                 */
    int64_t timeout_cycles; /* bound on every device wait, in SM clock cycles;
                               0 = default (about 2 s)                         */
    int32_t positions;      /* nb_positions (ignored by NB_PREC_FP64)          */
    float near_gamma;       /* NB_POS_ADAPTIVE: a tile pair is well separated
                               when its box gap >= near_gamma x the largest
                               coordinate magnitude; 0 = default (1/64;
                               1/256 on the batched symmetric path)       */
    int32_t pairs;          /* nb_pairs                                       */
    int32_t test_unissued_stage; /* test hook, 0 = off.  k > 0: the direct-pair
                               kernels that stage j-tiles through a ring of
                               bulk copies (nb_forces / nb_forces_range /
                               nb_forces_noalloc on the direct path,
                               nb_forces_vjp and the step adjoints,
                               nb_forces_jerk / nb_hermite4) never issue the
                               copies of their k-th stage in each CTA, so the
                               bounded wait on it runs out after
                               timeout_cycles and NB_ERR_TIMEOUT is latched:
                               how a test exercises the device-side timeout
                               path without a fault.  Results are then
                               undefined and the workspace needs re-zeroing. */
} nb_opts;

/* Fills *opts with precision F64ACC, G = 1, default stream, no graph,
 * default tune, timeout and position handling. */
void nb_opts_default(nb_opts *opts);

/* Library version string and the list of compiled kernel shapes. */
const char *nb_version(void);

/* Message for the last failing call on this host thread ("" if none). */
const char *nb_last_error(void);

/*
 * Self-check of the integer-pipe float <-> double conversions and
 * finiteness test that FP64-bound kernels use, and of the fixed-point split
 * of FP64 partials: on the host, the same source's results for every float
 * exponent with edge significands, every double exponent with significands
 * at the rounding boundaries, 3 n seeded random float patterns and 2 n
 * double patterns (splitmix64 from `seed`), and edge and n random
 * (value, exponent) pairs for the split, are compared with the C
 * conversions (round to nearest even), isfinite and v 2^F rounded half away
 * from zero;
 * *mismatches receives the count (0 when they agree).  No device work.
 * NB_ERR_INVALID for a NULL pointer or n < 0.
 */
int nb_check_fp_conversions(int64_t n, uint64_t seed, int64_t *mismatches);

/* Number of kernels this library has enqueued in this process (all host
 * threads).  Kernels replayed from a captured CUDA graph are not counted. */
unsigned long long nb_launch_count(void);

/*
 * Opt-in timing of the dominant kernel, the symmetric FP32-pair kernel of
 * nb_forces / nb_step (not its fold or the O(N) kernels): while enabled, a
 * pair of CUDA events is recorded on the launch stream just before and after
 * each of its launches (none inside a stream capture).  The events come from
 * a ring of 64 pairs on the device that is current at nb_kernel_timing(1);
 * when all 64 hold unread times, the next launch first waits on the host for
 * the oldest and adds it to the running total.  Launches on another device
 * mark the record as failed.  enable = 1 clears the record and starts
 * timing, 0 stops it.  Process-wide; meant for one host thread.  Always
 * returns NB_OK.
 */
int nb_kernel_timing(int32_t enable);

/*
 * Waits for the launches timed since nb_kernel_timing(1) and returns their
 * summed duration in ms and their number.  NB_ERR_INVALID for NULL
 * pointers; NB_ERR_CUDA if an event could not be created, recorded or read
 * (the outputs are then 0).
 */
int nb_kernel_time(double *total_ms, int64_t *launches);

/* 1 if `tune` names a kernel shape compiled into this build (and an
 * item_blocks of 0, 2, 4 or 8), else 0. */
int nb_tune_valid(const nb_tune *tune);

/*
 * Workspace bytes needed for problems of up to N_total particles in B
 * clusters (B = 1 for a single system) under `opts` (precision and tune
 * change the size).  Never fails; returns 0 for N_total < 1 or B < 1.
 */
size_t nb_workspace_bytes(int64_t N_total, int32_t B, const nb_opts *opts);

/*
 * Accelerations and potentials of one system (Eq. 1, Sec. 2.1; the pair
 * kernel of App. A, Algorithm 3, without its jerk terms).
 *   pos  [N][3], mass [N]         inputs
 *   eps  >= 0                     Plummer softening length; eps == 0 selects
 *                                 the guarded kernel that skips coincident
 *                                 pairs (meant for tests and exact orbits)
 *   acc  [N][3]                   output, overwritten
 *   pot  [N] or NULL              output, overwritten when non-NULL
 * Returns NB_ERR_INVALID for N < 1, NULL or misaligned arrays, eps < 0 or
 * non-finite, or opts->G non-finite; NB_ERR_WORKSPACE if ws is too small.
 */
int nb_forces(const double *pos, const double *mass, int64_t N, double eps, double *acc,
              double *pot, void *ws, size_t ws_bytes, const nb_opts *opts);

/*
 * Accelerations and potentials of the particles i0 .. i1-1 of a system of N
 * (Eq. 1 for those rows only, each against all N).  This is one rank's
 * share when the particles of one system are split over several GPUs in
 * contiguous ranges -- the data decomposition of Sec. 3.2 (approach 1):
 * every rank holds all N positions (gathered each step) and evaluates its
 * own rows; no other exchange is needed for the forces.
 *   pos [N][3], mass [N]          all particles (inputs)
 *   0 <= i0 < i1 <= N             the rows
 *   acc [i1-i0][3]                output rows, overwritten
 *   pot [i1-i0] or NULL           output rows, overwritten when non-NULL
 * Every ordered pair of the rows is evaluated (the direct kernel, whatever
 * opts->pairs says); positions ADAPTIVE is taken as SPLIT.  The workspace
 * is sized for the whole system: nb_workspace_bytes(N, 1, opts).
 * Returns NB_ERR_INVALID for a bad range and as nb_forces otherwise.
 */
int nb_forces_range(const double *pos, const double *mass, int64_t N, int64_t i0, int64_t i1,
                    double eps, double *acc, double *pot, void *ws, size_t ws_bytes,
                    const nb_opts *opts);

/*
 * The kick and drift of kick-drift-kick leapfrog for n particles, in FP64:
 *   vel += kick * acc;   pos += drift * vel   (the updated vel)
 * pos, vel, acc device [n][3].  A KDK step of size h whose force evaluation
 * the caller drives itself (nb_forces_range on several GPUs) is
 * nb_kick_drift(h/2, h), the evaluation at the new positions, then
 * nb_kick_drift(h/2, 0).  With drift == 0, pos is neither read nor written
 * (it may alias vel: a plain v += kick a).  NB_ERR_INVALID for n < 1, NULL
 * or misaligned arrays, non-finite kick or drift.
 */
int nb_kick_drift(double *pos, double *vel, const double *acc, int64_t n, double kick,
                  double drift, const nb_opts *opts);

/*
 * nb_forces for callers that cannot allocate device memory and therefore
 * cannot hand the library a workspace: for instance a plug-in whose host
 * application owns every device allocation through its own pool, or a
 * latency-critical loop that must never reach cudaMalloc (it can block and
 * synchronise the device).  The paper has no counterpart; this is a
 * convenience of this library.
 *
 * Same arguments and results as nb_forces without (ws, ws_bytes), on the
 * direct kernel (every ordered pair) with one fixed launch shape: the
 * scratch is a fixed device array inside the library (about 6.2 MB, held on
 * every GPU that loads the library until the process exits), so N is limited
 * to 32768; larger N returns NB_ERR_INVALID.  Options it does not serve are
 * refused with NB_ERR_UNSUPPORTED: opts->pairs = NB_PAIRS_SYMMETRIC,
 * opts->positions = NB_POS_ADAPTIVE and a non-NULL opts->tune (DEFAULT pairs
 * mean DIRECT here; DEFAULT positions mean SPLIT for KAHAN and F64ACC and
 * SINGLE for FP32, as in nb_forces).  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress), so make the first call
 * on each device before capturing any CUDA stream.  Every call shares the
 * one array: calls that may overlap on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.  Each
 * call clears the array's counters and status word itself.  Device-side
 * errors (a non-finite result, a wait that ran out) are latched in the
 * array's status word: nb_poll_status(NULL, 0, stream) reads and clears it
 * for the current device, and must be called before the next call, which
 * clears it.
 */
int nb_forces_noalloc(const double *pos, const double *mass, int64_t N, double eps, double *acc,
                      double *pot, const nb_opts *opts);

/*
 * Accelerations and potentials of B independent clusters in one launch; the
 * particles of cluster c are offsets[c] .. offsets[c+1]-1 and interact only
 * with each other.  offsets (int64 [B+1], offsets[0] = 0, offsets[B] = N) and
 * eps (double [B]) are device arrays; each cluster must hold between 1 and
 * 8192 particles and every eps[c] must be > 0.  These device-side
 * conditions are checked on the device: a violating cluster is skipped and
 * NB_ERR_INVALID is latched for nb_poll_status.  N is the total particle
 * count (the workspace is sized with nb_workspace_bytes(N, B, opts)).  FP32
 * pairs only (precision FP32, KAHAN or F64ACC).  The work division over
 * clusters follows the SPMD split of Sec. 3.1 (independent work per core):
 * warp-granular work items of every cluster on the symmetric path
 * (default), one cluster per thread-block cluster on the direct path
 * (opts->pairs = NB_PAIRS_DIRECT).  Host-side errors: NB_ERR_INVALID for
 * B < 1, N < B, N > 2^30, NULL arrays, a non-finite G, an unknown
 * precision, or (symmetric path) a tune item_blocks other than 0, 2, 4, 8;
 * NB_ERR_UNSUPPORTED for FP64 pairs; NB_ERR_WORKSPACE if ws is too small.
 */
int nb_forces_batched(const double *pos, const double *mass, const int64_t *offsets, int32_t B,
                      int64_t N, const double *eps, double *acc, double *pot, void *ws,
                      size_t ws_bytes, const nb_opts *opts);

/*
 * State advanced by nb_step.  Single system: B = 1, offsets = NULL, eps used.
 * Batched: B > 1 (or offsets != NULL), offsets/eps_b device arrays as in
 * nb_forces_batched, eps ignored.  pos/vel/acc/pot device [N][3]/[N]
 * (pot may be NULL).  acc_valid = 1 means acc already holds a(pos) (first-
 * same-as-last reuse); nb_step sets it to 1 and adds nsteps to `step`.
 */
typedef struct nb_state {
    int64_t N;
    int32_t B;
    const int64_t *offsets;
    double *pos;
    double *vel;
    const double *mass;
    double *acc;
    double *pot;
    const double *eps_b;
    double eps;
    int64_t step;
    int32_t acc_valid;
    void *ws;
    size_t ws_bytes;
} nb_state;

/*
 * nsteps kick-drift-kick leapfrog steps of size dt:
 *   v += (dt/2) a(x);  x += dt v;  v += (dt/2) a(x)
 * The paper advances with a predict-evaluate-correct Hermite scheme (Sec. 2.1)
 * around the same all-pairs evaluation; this library uses leapfrog.  On
 * return acc holds a(x) and pot (if not NULL) phi(x) at the final
 * positions; the potential of intermediate steps is not observable and is
 * not summed (nsteps = 0 evaluates a and phi at the current positions).
 * The batched form runs all clusters' steps in a few launches per step
 * (symmetric path) or one persistent launch (direct path).  dt must be
 * finite, nsteps >= 0.
 */
int nb_step(nb_state *s, double dt, int64_t nsteps, const nb_opts *opts);

/*
 * Energy bookkeeping of the state: out3 (device double[3]) receives
 * K = 1/2 sum m |v|^2, W = 1/2 sum m phi, E = K + W, summed in a fixed order
 * (bitwise reproducible).  Needs s->pot valid (call after nb_forces or
 * nb_step with a non-NULL pot).  For batched states the sums run over all
 * clusters together.
 */
int nb_energy(const nb_state *s, double *out3, const nb_opts *opts);

/*
 * Vector-Jacobian product of (a, phi) with respect to (x, m) at (pos, mass):
 *   pos_bar_k  = sum_i (d a_i/d x_k)^T acc_bar_i + sum_i (d phi_i/d x_k) pot_bar_i
 *   mass_bar_k = sum_i (d a_i/d m_k) . acc_bar_i + sum_i (d phi_i/d m_k) pot_bar_i
 * i.e. pos_bar_k = G sum_{j!=k} K(d)(m_k abar_j - m_j abar_k)
 *                  - G sum_{j!=k} s^-3 (m_k pbar_j + m_j pbar_k) d,
 *      mass_bar_k = -G sum_{j!=k} (s^-3 abar_j . d + s^-1 pbar_j),
 * with d = x_j - x_k, s^2 = |d|^2 + eps^2, K(d) = s^-3 I - 3 s^-5 d d^T.
 * acc_bar [N][3] in; pot_bar [N] in or NULL (zero); pos_bar [N][3] and
 * mass_bar [N] out, overwritten.  Derived from Eq. 1; the paper itself does
 * not differentiate its simulation.  The VJP kernels form displacements
 * from single FP32 positions unless opts->positions is NB_POS_SPLIT
 * (gradients tolerate the ~1e-5 displacement error; the adjoint tests gate
 * FP32-pair gradients at 1e-4 median / 1e-3 max against FP64).
 */
int nb_forces_vjp(const double *pos, const double *mass, int64_t N, double eps,
                  const double *acc_bar, const double *pot_bar, double *pos_bar,
                  double *mass_bar, void *ws, size_t ws_bytes, const nb_opts *opts);

/*
 * nb_forces_vjp for the rows i0 .. i1-1, scaled and accumulated:
 *   pos_bar[r]  += coef * pos_bar_(i0+r),  mass_bar[r] += coef * mass_bar_(i0+r)
 * (the sums above, each against all N).  One rank's share of a step
 * adjoint when the particles of one system are split over several GPUs in
 * contiguous ranges (Sec. 3.2, approach 1): the cotangents of all N
 * (gathered each step) come in, the rank's rows go out.
 *   pos [N][3], mass [N]            all particles (inputs)
 *   0 <= i0 < i1 <= N               the rows
 *   coef                            finite scale of the cotangents
 *   acc_bar [N][3], pot_bar [N] or NULL   all particles' cotangents
 *   pos_bar [i1-i0][3], mass_bar [i1-i0]  rows, accumulated into
 * The workspace is sized for the whole system: nb_workspace_bytes(N, 1,
 * opts).  Returns NB_ERR_INVALID for a bad range or non-finite coef and as
 * nb_forces_vjp otherwise.
 */
int nb_forces_vjp_range(const double *pos, const double *mass, int64_t N, int64_t i0, int64_t i1,
                        double eps, double coef, const double *acc_bar, const double *pot_bar,
                        double *pos_bar, double *mass_bar, void *ws, size_t ws_bytes,
                        const nb_opts *opts);

/*
 * One merged reverse step of the discrete KDK adjoint at positions pos_k:
 *   vel_bar  += drift_dt * pos_bar          (adjoint of the drift x += dt v)
 *   c         = kick_coef * vel_bar          (cotangent of the kicks at x_k)
 *   pos_bar  += J_x(pos_k)^T c,  mass_bar += J_m(pos_k)^T c
 * where J is the Jacobian of a(x, m).  The reverse sweep of K steps of size
 * h from the final cotangents is: one call at x_K with (drift_dt, kick_coef)
 * = (0, h/2); calls at x_{K-1} .. x_1 with (h, h); one call at x_0 with
 * (h, h/2).  The two half-kick cotangents meeting at each interior x_k are
 * thereby applied in one VJP.  pos_bar, vel_bar, mass_bar are read and
 * updated in place.
 */
int nb_step_vjp(const double *pos_k, const double *mass, int64_t N, double eps, double drift_dt,
                double kick_coef, double *pos_bar, double *vel_bar, double *mass_bar, void *ws,
                size_t ws_bytes, const nb_opts *opts);

/*
 * Reverse-time reconstruction fused with the adjoint: one call replaces a
 * recomputed forward step plus nb_step_vjp when the trajectory is rebuilt
 * backwards instead of stored.  With the positions x_k in pos:
 *   acc      = a(x_k)                       (written)
 *   vel_bar, pos_bar, mass_bar              updated exactly as
 *                                           nb_step_vjp(x_k, drift_dt, kick_coef)
 *   vhalf   -= rewind_kick * acc;  pos -= rewind_drift * vhalf
 * With vhalf = v_{k+1/2} and rewind_kick = rewind_drift = h this leaves
 * v_{k-1/2} and x_{k-1}; with vhalf = v_k and rewind_kick = h/2 it starts
 * the rewind from a stored full-step state; zeros leave the state alone.
 * The leapfrog map is time-reversible, so this recovers the forward
 * trajectory up to rounding; callers re-anchor at stored checkpoints.
 * pos, vhalf, acc: device [N][3]; the pair loop reads a packed copy of pos
 * taken before any update.
 */
int nb_step_vjp_reverse(double *pos, double *vhalf, double *acc, const double *mass, int64_t N,
                        double eps, double rewind_kick, double rewind_drift, double drift_dt,
                        double kick_coef, double *pos_bar, double *vel_bar, double *mass_bar,
                        void *ws, size_t ws_bytes, const nb_opts *opts);

/*
 * Acceleration, jerk and potential at (pos, vel): the quantities of the
 * paper's pair kernel (App. A, Algorithm 3; jerk = time derivative of the
 * acceleration along the motion),
 *   jerk_i = G sum_{j != i} m_j [ (v_j - v_i) / s^3 - 3 ((x_j - x_i).(v_j - v_i)) (x_j - x_i) / s^5 ]
 * with s^2 = |x_j - x_i|^2 + eps^2.  pos, vel, acc, jerk [N][3]; mass, pot
 * [N] (pot nullable).  FP32 pairs from split hi/lo positions and FP32
 * velocities; precision FP32, KAHAN or F64ACC (FP64 returns
 * NB_ERR_UNSUPPORTED).
 */
int nb_forces_jerk(const double *pos, const double *vel, const double *mass, int64_t N,
                   double eps, double *acc, double *jerk, double *pot, void *ws, size_t ws_bytes,
                   const nb_opts *opts);

/*
 * nsteps of the fourth-order Hermite predictor-corrector around the
 * acceleration + jerk evaluation (the predict / evaluate / correct cycle of
 * Sec. 2.1, at fourth order; the paper's own integrator is sixth order):
 *   xp = x + v h + a h^2/2 + j h^3/6,  vp = v + a h + j h^2/2
 *   a1, j1 = evaluation at (xp, vp)
 *   v <- v + (a + a1) h/2 + (j - j1) h^2/12,  x <- x + (v_old + v) h/2 + (a - a1) h^2/12
 * acc/jerk must hold a(x), j(x) when acc_valid != 0 (else they are computed
 * first) and hold the last evaluation on return.  Other arguments as
 * nb_forces_jerk.
 */
int nb_hermite4(double *pos, double *vel, const double *mass, int64_t N, double eps, double *acc,
                double *jerk, int32_t acc_valid, double dt, int64_t nsteps, void *ws,
                size_t ws_bytes, const nb_opts *opts);

/*
 * Synchronises `stream`, reads the device status word latched in ws (a
 * bitwise OR of 1 << NB_ERR_TIMEOUT, 1 << NB_ERR_INVALID and
 * 1 << NB_ERR_NONFINITE), clears it, and returns the matching NB_ERR_* code
 * (timeout first, then invalid, then non-finite) or NB_OK.  ws = NULL reads
 * the status word of nb_forces_noalloc's fixed array on the current device
 * (ws_bytes is then ignored).  NB_ERR_INVALID (as a host error) for a
 * non-NULL ws of fewer than 256 bytes.
 */
int nb_poll_status(void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
