/*
 * ising_ds.h - C ABI of the GB300 pruning + domain-selection Ising solver.
 *
 * The solver follows Li, Dong and Pan, "Fast Numerical Solver of Ising
 * Optimization Problems via Pruning and Domain Selection":
 *   - the problem (Sec. II, Eq. primal): minimise E(s) over s in {-1,+1}^n,
 *   - pruning (Sec. III-A, Algorithm 1): fix determined and semi-determined
 *     spins and fold them into a smaller problem plus a constant,
 *   - domain selection (Sec. III-B, Eq. loss function): relax each spin to
 *     sin(theta_i), run Adam on many restarts at once, round, keep the best,
 *   - reconstruction: recover the pruned spins from the record of pruning.
 *
 * Conventions shared by every call
 * --------------------------------
 * An instance holds stored couplings J (symmetric, zero diagonal), an
 * optional field h, a scale j_scale and a convention:
 *   ISING_CONV_PHYSICS:  E(s) = -1/2 * j_scale * s^T J s - h^T s
 *                        (max-cut with weights W is J = -W, j_scale = 1/2),
 *   ISING_CONV_PAPER:    E(s) = j_scale * s^T J s + h^T s   (Sec. II form).
 * Both reduce to E(s) = cQ s^T J s + cH h^T s, (cQ, cH) = (-j_scale/2, -1)
 * or (j_scale, +1).
 *
 * Dense J is n*n row-major. CSR J stores both (i,j) and (j,i), columns
 * strictly increasing inside a row, no diagonal entry; indptr has n+1
 * entries. Spin vectors are int8 +1/-1. Restart-major arrays of B vectors of
 * length n are [B][n] with the spin index contiguous.
 *
 * Memory: every pointer of an instance and every output pointer is host or
 * device memory as the call's `mem` argument (or the instance's `mem` field)
 * says; the library copies what it needs and never keeps a caller pointer
 * past the call. Objects returned through `**out` are owned by the library
 * and released by the matching *_destroy / *_free call.
 *
 * Errors: every call returns an ising_status. On error nothing is written to
 * the outputs, and ising_last_error(ctx) describes the failure. A CUDA error
 * is reported as ISING_ECUDA. No exception and no abort crosses the ABI.
 * A context is not thread-safe: serialise calls on one context.
 */
#ifndef ISING_DS_H
#define ISING_DS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ising_status {
  ISING_OK = 0,
  ISING_EINVAL = 1,   /* bad argument: shape, dtype, asymmetric J, diagonal */
  ISING_ENOMEM = 2,   /* device or host allocation failed */
  ISING_ECUDA = 3,    /* a CUDA call failed */
  ISING_ETIMEOUT = 4, /* a bounded device wait gave up */
  ISING_EBUSY = 5,    /* server: request does not fit the memory budget now */
  ISING_ENOTSUP = 6   /* combination of options the library does not support */
} ising_status;

enum { ISING_LAYOUT_DENSE = 0, ISING_LAYOUT_CSR = 1 };
enum { ISING_F64 = 0, ISING_F32 = 1, ISING_I8 = 2, ISING_I32 = 3 };
enum { ISING_CONV_PHYSICS = 0, ISING_CONV_PAPER = 1 };
enum { ISING_MEM_HOST = 0, ISING_MEM_DEVICE = 1 };

/* Coupling product precision of the domain-selection step (Sec. III-B).
 *  AUTO        dense -> TC, CSR -> sparse FP32/int kernel.
 *  FP32_PLAIN  dense J in FP32 on the CUDA cores (SIMT FMA), the plain form.
 *  TC          dense J on the tensor cores (tcgen05, FP32 accumulate), exact
 *              to FP32 level: integer |J| <= 256 as one BF16 plane, integer
 *              |J| <= 2048 as one FP16 plane, integer |J| <= 65504 as two
 *              FP16 planes hi + lo (all exact), other J as two FP16 planes of
 *              J_ij / 2^e_i with a power-of-two scale per row (about 22
 *              significant bits: |J - hi - lo| <= 2^-22 |J| + 2^-25 2^e_i).
 *  BF16        dense J rounded once to BF16 (lossy for non-integer J).
 *  FP8         dense J as E4M3 with one FP32 scale per row; spins E4M3
 *              (exact for integer |J| <= 16, lossy otherwise).
 * Every candidate is rounded to +-1 and its energy re-evaluated exactly
 * (integer J) or in FP64 (other J) by the final energy pass. */
enum {
  ISING_PREC_AUTO = 0,
  ISING_PREC_FP32_PLAIN = 1,
  ISING_PREC_TC = 2,
  ISING_PREC_BF16 = 3,
  ISING_PREC_FP8 = 4
};

/* Execution path actually used, reported in ising_ds_stats.path. */
enum { ISING_PATH_PLAIN = 0, ISING_PATH_TC = 1, ISING_PATH_SPARSE = 2 };

typedef struct ising_ctx ising_ctx;
typedef struct ising_ds ising_ds;
typedef struct ising_prune_result ising_prune_result;

/* An Ising instance (Sec. II). Borrowed for the duration of a call. */
typedef struct ising_instance {
  int64_t n;              /* number of spins, >= 1 */
  int32_t layout;         /* ISING_LAYOUT_* */
  int32_t j_dtype;        /* ISING_F64/F32/I8/I32 */
  const void* J;          /* dense: n*n; CSR: nnz values */
  const int64_t* indptr;  /* CSR: n+1 row offsets, else NULL */
  const int32_t* indices; /* CSR: nnz column indices, else NULL */
  int64_t nnz;            /* CSR: number of stored entries */
  int32_t h_dtype;        /* ISING_F64/F32/I32 (ignored when h is NULL) */
  int32_t reserved0;
  const void* h;          /* n fields, or NULL for h = 0 */
  double j_scale;         /* effective coupling = j_scale * stored J */
  int32_t convention;     /* ISING_CONV_* */
  int32_t mem;            /* ISING_MEM_* for J, indptr, indices, h */
} ising_instance;

/* Domain-selection parameters (Sec. III-B, Sec. IV-B). */
typedef struct ising_ds_params {
  int64_t restarts; /* B >= 1 independent runs ("sweeps") */
  int64_t steps;    /* T >= 0 Adam steps; energies at steps 1..T+1 */
  double lr;        /* Adam learning rate (the paper uses 6.0) */
  double mu;        /* penalty weight of Eq. (lagrange function), >= 0 */
  double beta1;     /* Adam first-moment decay, in [0,1) (0.9) */
  double beta2;     /* Adam second-moment decay, in [0,1) (0.999) */
  double eps;       /* Adam epsilon, > 0 (1e-8) */
  uint64_t seed;    /* theta_init = asin(x0), x0 from SplitMix64(seed) */
  int32_t precision;/* ISING_PREC_* */
  int32_t flags;    /* ISING_DS_PROFILE or 0 */
} ising_ds_params;

/* params.flags: time every step-kernel launch with CUDA events on the
 * context's stream and report the sum in ising_ds_stats.kernel_ms (for the
 * resident tensor-core form, one launch runs many steps: kernel_ms / kernel_launches
 * is then the time per step). */
#define ISING_DS_PROFILE 1
/* params.flags: keep the tensor-core path's state in device memory between
 * steps (one launch per step) even when a resident form would fit. The
 * resident forms keep theta, m and v in tensor memory across a whole run in
 * one launch: for n <= 128 the small form (every CTA holds all of J and the
 * spins of its block of restarts in shared memory, no grid-wide barrier), for
 * larger n the grid-wide form, used when every 128 x BN tile gets its own SM
 * (one cooperative launch). */
#define ISING_DS_STREAMING 2
/* params.flags: skip the launch-shape autotuner and use the default shape.
 * The autotuner times the first steps of a run once per problem shape with
 * each candidate shape and keeps the fastest: on the sparse path one or two
 * slices of 128 restarts per warp, on the tensor cores' streaming form the
 * restart-tile width (64, 128, 224 or 256 restarts per tile); results do not
 * depend on the shape. Choices are cached per process and, when the
 * environment variable ISING_TUNE_CACHE names a file, across processes. */
#define ISING_DS_NO_AUTOTUNE 4
/* params.flags: the convergence rule of Sec. IV-B, read on the energy of the
 * rounded spins: restart b stops at the first step t >= 5 where
 * max - min of E_{t-4..t}(b) <= 0.005 |E_t(b) - E_1(b)| (at convergence
 * sin(theta) -> s and the paper's loss equals E - mu d). A stopped restart's
 * best and last energy are those of steps 1..t; the streaming tensor-core,
 * sparse and plain step kernels skip every tile or slice whose restarts have
 * all stopped (early retirement, see ising_ds_work); the run ends once every
 * restart has stopped (checked every 48 steps, so up to 47 more steps may run,
 * which change nothing) and ising_ds_stats.steps_done tells how far it went;
 * the final evaluation (step T+1) applies to restarts still running after T.
 * Per-restart stopping steps: ising_ds_convergence. */
#define ISING_DS_CONVERGE 8
/* params.flags: the relaxed coupling product G = J sin(theta) in the update
 * (the loss field F = cQ G + cH h - mu s and the gradient cos(theta) F keep
 * their form; s and the energies stay those of the rounded spins), instead
 * of the paper's G = J s of the local optimum s (Sec. III-B). Dense paths
 * evaluate the energies with a second product on s each step; the tensor
 * cores take x in BF16 (so G is within 2^-8 sum_j |J_ij| of the exact
 * product; E4M3 operands and the resident form are not used), the CUDA-core
 * and sparse paths in FP32. */
#define ISING_DS_RELAXED 16

typedef struct ising_ds_stats {
  int64_t best_restart;     /* restart holding the overall best */
  int64_t best_step;        /* step (1..T+1) at which it was reached */
  double last_best_energy;  /* lowest energy of the final spins (step T+1) */
  int64_t last_best_restart;
  int64_t steps_done;
  int32_t path;             /* ISING_PATH_* */
  int32_t precision;        /* ISING_PREC_* actually used */
  double device_ms;         /* device time of the steps (CUDA events) */
  double kernel_ms;         /* step kernels only (with ISING_DS_PROFILE) */
  int64_t kernel_launches;  /* step-kernel launches timed in kernel_ms */
  int32_t resident;         /* tensor-core path kept the state in tensor memory: 1 in the
                               grid-wide form, 2 in the small form (n <= 128, each CTA holds
                               all of J and its restarts' spins on chip); 0 otherwise */
  int32_t operand_planes;   /* tensor-core path: operand planes of J per product (1 or 2;
                               the tensor cores execute that many products), else 1 */
  int32_t tile_restarts;    /* tensor-core streaming form: restarts per tile, else 0 */
  int32_t tile_pair;        /* tensor-core streaming form: 0 one CTA per tile, 1 CTA pairs
                               sharing spin tiles by multicast, 2 one MMA per CTA pair
                               (see ising_ds_set_tiles); else 0 */
} ising_ds_stats;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`, issuing work on `stream`
 * (a cudaStream_t, NULL = the legacy default stream). */
int ising_create(ising_ctx** out, int device, void* stream);
/* Destroy a context. Every session and pruning result created on it must be
 * destroyed first (they refer to the context). */
int ising_destroy(ising_ctx* ctx);
/* Message of the last failed call on this context ("" if none). The string
 * lives until the next call on the context. */
const char* ising_last_error(const ising_ctx* ctx);
int ising_set_stream(ising_ctx* ctx, void* stream);
/* Wait for all work the context issued. */
int ising_synchronize(ising_ctx* ctx);
/* ABI version: major * 10000 + minor * 100 + patch. */
int ising_version(void);
/* Diagnostic of the failure handling (the paper has no counterpart): runs
 * on the context's stream a kernel with two waits that nothing completes,
 * each bounded by `limit_cycles` SM clock cycles in the same way as the
 * tensor-core kernels' waits: an mbarrier that receives no arrival and a poll
 * of a device flag that nothing sets. Both give up; `gave_up` (nullable)
 * receives the bitmask of the waits that did (1 mbarrier, 2 flag) and the
 * call returns ISING_ETIMEOUT, after which the context stays usable.
 * limit_cycles must lie in [1, 2^34]. */
int ising_selftest_waits(ising_ctx* ctx, int64_t limit_cycles, int32_t* gave_up);

/* ------------------------------------------------------------------ energy */

/* E(s) (Sec. II) of `count` spin vectors spins[count][n] (int8, memory
 * `mem`). Writes E_out[count] (float64) and, if Q_out / H_out are not NULL
 * and the instance is integer, the exact parts Q = s^T J s and H = h^T s
 * (int64, E = cQ Q + cH H). Integer couplings accumulate in integers and
 * are exact; other couplings accumulate in FP64. Outputs are in memory
 * `mem`. */
int ising_energy(ising_ctx* ctx, const ising_instance* inst, const int8_t* spins,
                 int64_t count, double* E_out, int64_t* Q_out, int64_t* H_out, int mem);

/* E(s) of `count` spin vectors like ising_energy, but allocating nothing, for
 * callers that cannot allocate device memory (they own fixed buffers, or
 * they run where cudaMalloc is not allowed). The paper has no counterpart:
 * this is a deployment convenience.
 *   - Every pointer (the instance's, spins[count][n] int8, E_out[count]
 *     float64) must be device memory; inst->mem must be ISING_MEM_DEVICE.
 *     No context is needed and the instance is not validated (J must be
 *     symmetric with zero diagonal, CSR columns sorted).
 *   - Work is queued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) and is not waited for; E_out is ready when the stream is.
 *   - count must lie in [0, 65535] (one grid row per vector); larger
 *     counts return ISING_EINVAL.
 *   - Partial sums live in one 2 MiB static device array per device (held
 *     until the process exits); a call needs count * ceil(n / 64) * 16
 *     bytes of it and larger calls return ISING_EINVAL. Every call reuses the
 *     same array: calls whose work overlaps on the GPU (two streams, or two
 *     threads) race and give wrong results. Nothing in it has to start at
 *     zero (each call writes every slot it reads).
 *   - The first call made with a device current looks up the array's device
 *     address and keeps it for the process; make that first call before any
 *     stream capture. A device reset by the caller invalidates the kept
 *     address.
 * Integer J and h (I8/I32) accumulate exactly in int64; others in FP64.
 * Errors return a status; ising_energy_noalloc_error() describes the last
 * one on the calling thread. */
int ising_energy_noalloc(const ising_instance* inst, const int8_t* spins, int64_t count,
                         double* E_out, void* stream);
const char* ising_energy_noalloc_error(void);

/* ------------------------------------------------------------------ batching */

/* Several domain-selection sessions of different sizes advanced together:
 * each step of every member runs as one persistent tensor-core launch over
 * the concatenated tiles of all members, which also tracks every member's
 * previous step (a tracking launch over all their restarts follows each
 * step instead when a member uses ISING_DS_CONVERGE, and one follows the
 * last step of each ising_pack_run) (the restarts, or "sweeps", of Sec. IV-C
 * batched across instances); from the pack's second ising_pack_run on, the step loop is
 * replayed from a CUDA graph captured then. Each member keeps its own step
 * counter on the device and computes exactly what it computes alone (the
 * same products in the same order): a member's state, bests and result are
 * identical to running it by itself.
 * Members: sessions of the tensor-core path in the streaming form (created
 * with ISING_DS_STREAMING, without ISING_DS_RELAXED), all with the same
 * operand type (E4M3 or 16-bit), energy mode (integer or FP32 partials) and
 * number of J planes (one, or two FP16 planes hi + lo);
 * every member is switched to one restart-tile width chosen for the pack
 * (the least waves of tiles over the SMs times the width, padding of the
 * members' restarts included; the results do not depend on it). Sessions may belong to different contexts
 * of the same device. Otherwise ISING_ENOTSUP / ISING_EINVAL. The pack borrows the
 * sessions: destroy it before any member. Work is queued on `ctx`'s stream,
 * ordered after work already queued on the members' streams and before work
 * queued on them later. */
typedef struct ising_pack ising_pack;
int ising_pack_create(ising_ctx* ctx, ising_ds* const* sessions, int32_t count, ising_pack** out);
/* Advance every member by `steps` steps (each must have that many left);
 * waits for the work and returns ISING_ETIMEOUT if a bounded device wait
 * gave up. */
int ising_pack_run(ising_pack* pack, int64_t steps);
int ising_pack_destroy(ising_pack* pack);

/* ------------------------------------------------------------------ pruning */

/* Algorithm 1 (Sec. III-A) on `inst`, rounds run until nothing changes:
 * determined spins (strict rule, Eq. determined spin), then isolated spins
 * with zero field if flags & 1 (ISING_PRUNE_ZERO_RULE, an extension), then
 * semi-determined spins (Eq. semi determined spin) on what is left; fields
 * fold in FP64 in row order, so decisions are reproducible bit for bit.
 * The result (reduced instance, constant, record) lives on the device and
 * is released by ising_prune_free. */
#define ISING_PRUNE_ZERO_RULE 1
int ising_prune(ising_ctx* ctx, const ising_instance* inst, int flags,
                ising_prune_result** out);
/* Sizes and scalars of a pruning result; any pointer may be NULL.
 * constant: E(s) = E_reduced(s_G) + constant for the reconstructed s.
 * eta: pruning rate 1 - n_reduced / n (Eq. pruning rate). */
int ising_prune_info(const ising_prune_result* res, int64_t* n_reduced,
                     int64_t* nnz_reduced, double* constant, double* eta,
                     int32_t* rounds);
/* The reduced instance: device pointers owned by `res` (valid until
 * ising_prune_free), same layout, j_dtype, j_scale and convention as the
 * input, h as float64. */
int ising_prune_reduced(const ising_prune_result* res, ising_instance* out);
/* Copies the reduced instance into caller buffers in memory `mem` (any may
 * be NULL): J (dense n_reduced^2 or nnz_reduced values, input j_dtype),
 * indptr (CSR, n_reduced + 1, int64), indices (CSR, nnz_reduced, int32),
 * h (n_reduced, float64, in the input's convention). */
int ising_prune_reduced_copy(const ising_prune_result* res, void* J, int64_t* indptr,
                             int32_t* indices, double* h, int mem);
/* The record of pruning, per original spin (arrays of n, memory `mem`, any
 * may be NULL): kind 0 kept / 1 determined / 2 isolated-zero / 3 semi,
 * round (0 if kept), value (+-1 for kinds 1 and 2), parent (kind 3),
 * sign (kind 3: s = sign * s_parent), g_index (position in the reduced
 * problem or -1). */
int ising_prune_record(const ising_prune_result* res, int8_t* kind, int32_t* round,
                       int8_t* value, int32_t* parent, int8_t* sign,
                       int64_t* g_index, int mem);
int ising_prune_free(ising_prune_result* res);
/* Full spins (n) from the reduced problem's spins (n_reduced), both int8 in
 * memory `mem`: kept spins copied, fixed spins set, semi-determined spins
 * follow their parent chain. */
int ising_reconstruct(ising_ctx* ctx, const ising_prune_result* res,
                      const int8_t* reduced_spins, int8_t* full_spins, int mem);

/* ------------------------------------------------------- domain selection */

/* One-shot domain selection (Sec. III-B) on `inst`: B restarts x T steps,
 * then the energy of the last rounded spins. Writes the best spins (n,
 * int8) and energy over all steps and restarts (lowest energy, then lowest
 * restart, then earliest step), in memory `mem`; stats may be NULL. */
int ising_select_domain(ising_ctx* ctx, const ising_instance* inst,
                        const ising_ds_params* p, int8_t* best_spins,
                        double* best_energy, ising_ds_stats* stats, int mem);

/* Full solve: pruning, domain selection on the reduced instance,
 * reconstruction and the energy of the reconstructed spins on the full
 * instance. prune_flags as ising_prune; best_spins has n entries. */
int ising_solve(ising_ctx* ctx, const ising_instance* inst, const ising_ds_params* p,
                int prune_flags, int8_t* best_spins, double* best_energy,
                ising_ds_stats* stats, int mem);

/* Session form of domain selection: create (uploads and converts J,
 * initialises theta, m = v = 0, step 0), advance, inspect, destroy. */
int ising_ds_create(ising_ctx* ctx, const ising_instance* inst,
                    const ising_ds_params* p, ising_ds** out);
/* Advance `steps` steps (stops at T). */
int ising_ds_run(ising_ds* ds, int64_t steps);
/* Evaluate the final spins (step T+1) and fill the result; idempotent. */
int ising_ds_finish(ising_ds* ds);
/* Current state, restart-major [B][n]: theta, m, v (float32), the spins
 * s_{t+1} = sgn+(sin theta) the next step will use (int8), and t. Any pointer
 * may be NULL. Memory `mem`. */
int ising_ds_export_state(ising_ds* ds, float* theta, float* m, float* v,
                          int8_t* spins, int64_t* t, int mem);
/* Replace the state (theta, m, v restart-major, step counter t); the spins
 * are re-derived from theta. Resets nothing else. */
int ising_ds_import_state(ising_ds* ds, const float* theta, const float* m,
                          const float* v, int64_t t, int mem);
/* The coupling product G = J s (Sec. III-B, the term inside the loss field)
 * of the spins the next step will use, computed by the session's own step
 * kernel and precision (tensor cores, CUDA cores or sparse); restart-major
 * [B][n] float32 in memory `mem`. Does not advance the session. */
int ising_ds_coupling(ising_ds* ds, float* G_out, int mem);
/* Role timeline of the most recent step launch of a session created with
 * ISING_DS_PROFILE (tensor-core path): 8 globaltimer stamps (ns) per CTA -
 * start, first / last TMA issue, first MMA issue, last MMA commit, first
 * accumulator seen by the epilogue, epilogue done, end. Copies
 * min(cap, 8 * CTAs) values to host `out`; *count receives 8 * CTAs (0 when
 * the path keeps no timeline). */
int ising_ds_trace(ising_ds* ds, uint64_t* out, int64_t cap, int64_t* count);
/* Energies E(s_t) of the spins consumed by the most recent step, [B]. */
int ising_ds_last_energies(ising_ds* ds, double* E, int mem);
/* Per-restart best so far: energy [B], step [B], spins [B][n] (any NULL). */
/* Restart-steps the session's update launches computed so far: every tile
 * or slice of restarts counts its restarts once per step (the resident
 * tensor-core forms count B per step). Without ISING_DS_CONVERGE this is
 * B x steps; with it, tiles and slices whose restarts have all stopped are
 * skipped (early retirement: their results are final, their state is left
 * where it stopped), so it falls below B x steps. The resident tensor-core
 * forms keep every restart running. Synchronises the session's stream. */
int ising_ds_work(ising_ds* ds, int64_t* restart_steps);
/* Launch shape of the tensor-core streaming form set by hand: 64, 128, 224
 * or 256 restarts per tile; pair = 1 runs the tiles over clusters of two
 * CTAs that share each spin tile (each loads half and multicasts it to
 * both; widths 224 and 256, more than 128 spins); pair = 2 as well, but
 * each CTA keeps its half and the pair's MMAs run as one (M 256 over the
 * two CTAs, cta_group::2). The autotuner leaves the
 * session alone afterwards. Results do not depend on the shape. ISING_ENOTSUP
 * on other forms, ISING_EINVAL for a shape the session cannot take. No
 * counterpart in the paper: a tuning control. */
int ising_ds_set_tiles(ising_ds* ds, int32_t restarts_per_tile, int32_t pair);
/* With ISING_DS_CONVERGE: the step at which each restart stopped (0 while it
 * runs), [B] int64 in memory `mem`. Without the flag all zeros. */
int ising_ds_convergence(ising_ds* ds, int64_t* step, int mem);
int ising_ds_restart_best(ising_ds* ds, double* E, int64_t* step, int8_t* spins,
                          int mem);
/* Overall best (after ising_ds_finish, or the best so far). */
int ising_ds_result(ising_ds* ds, int8_t* best_spins, double* best_energy,
                    ising_ds_stats* stats, int mem);
int ising_ds_destroy(ising_ds* ds);

/* ------------------------------------------------------------------ serving */

/* A request server: callers submit instances as they arrive; a worker thread
 * admits queued requests while their estimated device footprint fits the
 * memory budget and a slot is free, advances every admitted request by
 * `chunk_steps` steps per round on its own stream (the kernels of different
 * requests overlap on the device, and requests that arrive meanwhile join at
 * the next round), and posts each result when its steps are done; each
 * request's set-up (upload, pruning, session) and finishing run on helper
 * threads, so they do not hold up the other requests' chunks. A request
 * is solved exactly as ising_solve would solve it alone (pruning, domain
 * selection with the state kept in device memory between steps, best of
 * restarts, reconstruction, energy), so its result does not depend on what
 * else is being served. Requests run the tensor-core path in its streaming
 * form (no grid barrier shared with other requests' kernels), except
 * instances of at most 128 spins without ISING_DS_CONVERGE or
 * ISING_DS_RELAXED, whose small resident form has none either and runs a
 * whole chunk of steps in one launch. The paper has no counterpart.
 * The requests' streams reach the device through the context's hardware
 * work queues (8 unless the environment variable CUDA_DEVICE_MAX_CONNECTIONS,
 * read when the process creates its CUDA context, says more): with more
 * requests active than queues, streams share queues and their kernels
 * overlap less. */
typedef struct ising_server ising_server;

typedef struct ising_server_cfg {
  uint64_t budget_bytes; /* device memory the admitted requests may use */
  int32_t max_active;    /* requests on the GPU at once (streams), >= 1 */
  int32_t chunk_steps;   /* steps per request per scheduling round, >= 1 */
  int32_t flags;         /* 0 or ISING_SERVER_PACK */
  int32_t helper_threads;/* threads for requests' set-up and finishing, 0..16 (0: 2) */
} ising_server_cfg;

/* cfg.flags: the dense tensor-core requests ready in a scheduling round are
 * grouped by kind (operand type, energy mode) and each group advances its
 * chunk as one pack (see ising_pack_create) on one of four server streams
 * that the packs take in turn (the chunks of different groups overlap);
 * results are those of the requests alone. */
#define ISING_SERVER_PACK 1

typedef struct ising_result {
  int32_t status;        /* ISING_OK, or the error the request failed with */
  int32_t done;          /* 1 once the result is final */
  int64_t n;
  double best_energy;    /* energy of the returned spins on the full instance */
  int64_t best_restart;
  int64_t best_step;
  int64_t footprint;     /* estimated device bytes while admitted */
  double t_submit_ms;    /* host clock, ms since the server was created */
  double t_admit_ms;
  double t_done_ms;
  int64_t steps_done;    /* domain-selection steps the request ran */
  int32_t reached;       /* submitted with a target: 1 if best_energy <= target */
  int32_t cancelled;     /* 1 if ising_server_cancel ended it early */
} ising_result;

/* Creates the server on the context's device; the context must outlive it. */
int ising_server_create(ising_ctx* ctx, const ising_server_cfg* cfg, ising_server** out);
/* Copies the instance (host or device memory) and queues it with its
 * parameters and prune flags; *req_id identifies it. ISING_EBUSY when its
 * estimated footprint exceeds the whole budget (it could never be admitted). */
int ising_server_submit(ising_server* srv, const ising_instance* inst, const ising_ds_params* p,
                        int prune_flags, uint64_t* req_id);
/* Like ising_server_submit, for a time-to-target query: after every chunk
 * of steps the server evaluates the energy of the request's best spins so
 * far on the full instance (the best restart by tracked energy, the
 * near-best re-evaluated exactly as in ising_ds_result, reconstructed, then
 * ising_energy) and finishes the request as soon as it is <= target_energy,
 * without running its remaining steps (ising_result.steps_done tells how
 * many ran, .reached whether the target was met, by a check or by the
 * final result). Otherwise the request runs all its steps. The check synchronises the request's stream once per
 * chunk. */
int ising_server_submit_target(ising_server* srv, const ising_instance* inst,
                               const ising_ds_params* p, int prune_flags, double target_energy,
                               uint64_t* req_id);
/* Non-blocking: fills *res (res->done tells whether it is final) and, once
 * done, copies the n best spins to host `spins` if not NULL. ISING_EINVAL for
 * an unknown id. */
int ising_server_poll(ising_server* srv, uint64_t req_id, ising_result* res, int8_t* spins);
/* Blocks until the request is done or `timeout_s` passes (ISING_ETIMEOUT). */
int ising_server_wait(ising_server* srv, uint64_t req_id, double timeout_s, ising_result* res,
                      int8_t* spins);
/* Ends a request early: an admitted one finishes at the end of its current
 * chunk with the best of the steps run so far (its result as usual, with
 * cancelled = 1); a queued one is dropped and done at once, without spins
 * (best_energy NaN, steps_done 0). No effect on a finished request. */
int ising_server_cancel(ising_server* srv, uint64_t req_id);
/* The message of a finished request's failure (empty when it succeeded or
 * is not done), truncated to len - 1 bytes and NUL-terminated. */
int ising_server_error(ising_server* srv, uint64_t req_id, char* buf, int64_t len);
/* Drops a finished request's stored result. */
int ising_server_release(ising_server* srv, uint64_t req_id);
/* Where the server threads' host time went since the server was created
 * (ms of the host clock, summed over the worker and the helper threads; the
 * device work of the chunks overlaps it and is not included). */
typedef struct ising_server_stats {
  int64_t completed;     /* requests finished */
  int64_t rounds;        /* scheduling rounds that found work */
  int64_t chunks;        /* chunks queued for single requests */
  int64_t pack_chunks;   /* chunks queued as packs (one per pack) */
  int64_t packs_created; /* packs built (a new group of ready requests) */
  int64_t target_checks; /* time-to-target evaluations */
  double setup_ms;       /* admitted requests' set-up: upload, pruning, session */
  double setup_upload_ms;  /* of which the instance's upload */
  double setup_prune_ms;   /* of which pruning */
  double setup_session_ms; /* of which the session's creation */
  double advance_ms;     /* queueing chunks, single and packed (pack creation included) */
  double pack_create_ms; /* of which building packs */
  double check_ms;       /* convergence-count reads and target evaluations */
  double finish_ms;      /* finishing requests: final pass, result, reconstruction, energy */
  double release_ms;     /* freeing finished requests' device memory and session */
  double idle_ms;        /* waiting with no request ready */
  double elapsed_ms;     /* since the server was created */
} ising_server_stats;
int ising_server_stats_get(ising_server* srv, ising_server_stats* out);
/* Finishes the queued and active requests, stops the worker, frees all. */
int ising_server_destroy(ising_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* ISING_DS_H */
