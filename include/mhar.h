/*
 * mhar.h -- C ABI of the GB300 Matrix Hit-and-Run library (libmhar.so).
 *
 * Matrix Hit-and-Run (MHAR; Vazquez Corte & Montiel, arXiv 2104.07097,
 * Algorithm 2) moves z walkers together inside the polytope
 *     Delta = { x in R^n : A x <= b,  A_E x = b_E }       (Section 2.1, Eqs. TS1-TS3)
 * Each iteration draws Gaussian directions H (n x z; Section 4.3), projects
 * them onto the null space of A_E (D = P H with P = I - A_E^T (A_E A_E^T)^{-1} A_E,
 * Section 3.2), finds every walker's chord (lambda_min, lambda_max) from the
 * ratios (b - A X) / (A D) (Section 4.4), draws theta uniformly on it and
 * moves x^k += theta^k d^k (Section 4.5).  Every `thin` iterations the z
 * points are emitted (the thinning factor phi of Algorithm 2).
 *
 * Everything below runs as hand-written CUDA kernels for sm_103a on the
 * current CUDA device.  There is no CPU fallback: without a usable device
 * every entry point returns MHAR_E_CUDA.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major FP64 host arrays unless stated otherwise; the
 *     library copies what it needs, the caller keeps ownership.
 *   - Return value 0 (MHAR_OK) or a negative MHAR_E_* code.  After an error
 *     the context stays usable; mhar_last_error() describes the failure.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef MHAR_H
#define MHAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define MHAR_OK                 0
#define MHAR_E_ARG             -1  /* bad pointer, size or option            */
#define MHAR_E_X0_INFEASIBLE   -2  /* start not strictly inside A x <= b, or
                                      |A_E x0 - b_E| too large               */
#define MHAR_E_UNBOUNDED       -3  /* some walker met a chord open on one side
                                      (the body is unbounded, Section 2.1
                                      assumes bounded bodies)                */
#define MHAR_E_NONFINITE       -4  /* a non-finite slack, ratio or point, or
                                       (tensor-core modes) a point or direction
                                       beyond the FP16 range of its operands  */
#define MHAR_E_CUDA            -5  /* CUDA runtime / driver failure, or no
                                      sm_103 device                          */
#define MHAR_E_RANK            -6  /* A_E rank-deficient or cond > ~1e7      */
#define MHAR_E_UNSUPPORTED     -7  /* size or mode the library does not cover */
#define MHAR_E_TIMEOUT         -8  /* a bounded wait inside a tensor-core
                                      kernel expired (about 2 s): the pipeline
                                      stalled; the iteration's results are not
                                      to be trusted                          */
#define MHAR_E_INFEASIBLE_DRIFT -9 /* MHAR_MIXED_F16X3: a periodic refresh
                                      found the tracked slack further from
                                      b - A x than its error bound allows    */

/* ---- arithmetic modes -------------------------------------------------- */
/* MHAR_FP64: every step in FP64 on CUDA cores; the slack b - A x and A d are
 *   recomputed each iteration exactly as Lemma 4.2 lists them.
 * MHAR_FP32: the same recompute formulation in FP32 on CUDA cores (points are
 *   kept as FP32 pairs, "double-float", so they do not drift).
 * MHAR_MIXED_F16X3: A D on tcgen05 tensor cores.  Each row of A is scaled by
 *   a power of two and split into FP16 high + low parts, each direction into
 *   FP16 high + low parts; three products (hi.hi + hi.lo + lo.hi) accumulate
 *   in FP32 in tensor memory, which carries A d to about 2^-22 relative.  The
 *   slack S = b - A X is stored (FP32), updated as S -= (A D) diag(theta) in
 *   the same kernel, and recomputed from X every refresh_k iterations.
 * MHAR_MIXED_RECOMPUTE: the paper's own formulation (Lemma 4.2) on the tensor
 *   cores: every iteration one fused kernel forms A X and A D from FP16 pairs
 *   (three products each, FP32 accumulation), the slack b - A X, the ratios
 *   and the chord, moves the walkers, and prepares the next iteration's
 *   operands (and, without equalities or preconditioner, its directions).
 *   No slack is stored, so there is nothing to refresh and no drift;
 *   refresh_k is ignored.
 *
 * Feasibility in every mode.  Each chord end (Section 4.4) is computed from
 * a slack lowered by a bound on its rounding error and from an a_i . d
 * pushed away from zero by a bound on its own:
 *     lambda = (s_i - e_s) / (g_i +- e_g),
 *     e_s = K_i ||x / sigma||_2 + 3 u |b_i|,   e_g = K_i ||d / sigma||_2,
 * with sigma the power-of-two column scales of A (largest entry of each
 * column of A sigma in [0.5, 1) up to one common factor), u the unit
 * roundoff, and K_i = gamma_{n+4} ||a_i sigma||_2 on CUDA cores (gamma_k =
 * k u / (1 - k u)), or, on the tensor cores, the exact representation error
 * of row i's FP16 pair, the dropped products and (T + 1) 2^-22 ||a_i sigma||
 * for the FP32 accumulation of a chain of T MMAs (T = 3 n / 16 here, 4 n / 16
 * in MHAR_MIXED_F16X3, where the tracked slack's error since the last refresh
 * is added).  So a point on the computed chord satisfies A x <= b exactly
 * under that error model: the chord can only be shorter than the exact one
 * by those bounds (about (T + 1) 2^-22 relative on the tensor cores).  Every
 * iteration of a run can be checked in FP64 (opts.audit_every). */
#define MHAR_FP64             0
#define MHAR_FP32             1
#define MHAR_MIXED_F16X3      2
#define MHAR_MIXED_RECOMPUTE  3

typedef struct {
  uint64_t seed;          /* Philox4x32-10 key (default 0)                      */
  int32_t  precision;     /* MHAR_FP64 (default) | MHAR_FP32 | MHAR_MIXED_F16X3 |
                             MHAR_MIXED_RECOMPUTE                              */
  int32_t  refresh_k;     /* mixed mode: recompute S = b - A X every refresh_k
                             iterations (default 64; 0 = never)               */
  int32_t  out_on_device; /* 1: `out` of mhar_run is a device pointer          */
  uint32_t walker0;       /* global index of walker 0 (shards of one ensemble
                             use disjoint ranges; results are then identical
                             to the unsharded run)                            */
  void*    stream;        /* cudaStream_t for all work (NULL: legacy stream)   */
  int32_t  graph_chunk;   /* iterations per captured CUDA graph (default 16;
                             0 = launch kernels one by one)                   */
  int32_t  refresh_fp64;  /* mixed mode: 0 (default) recomputes S on the tensor
                             cores from the same FP16-pair operands the walk
                             uses (FP32 accumulation); 1 recomputes it in FP64
                             on CUDA cores (exact, far slower on GB300)       */
  int32_t  smem_operands; /* recompute mode: 0 (default) keeps the walker operands
                             in tensor memory when n <= 128; 1 always streams
                             them through shared memory (the kernel used for
                             larger n)                                        */
  int32_t  emit_walkers;  /* samples written by mhar_run hold walkers 0..W-1
                             only (0 = all z); e.g. a trace of a subset for
                             effective-sample-size estimates                 */
  int32_t  schedule;      /* recompute mode with shared-memory operands (n > 128
                             or smem_operands): 0 (default) picks the faster
                             of 1 = clusters of CTAs along the rows of A and
                             2 = stream-K (every SM takes an equal share of
                             the (walker strip, row tile) work; strips split
                             over SMs combine their partial chords in global
                             memory).  Results do not depend on it.          */
  int32_t  audit_every;   /* > 0: after every audit_every iterations of
                             mhar_run, an FP64 check of A x <= b and A_E x = b_E
                             on walkers 0..audit_walkers-1 folds into the
                             running maxima of mhar_stats (default 0: off)   */
  int32_t  audit_walkers; /* walkers checked by each audit (0: all z)          */
  int32_t  reserved;      /* must be zero                                     */
} mhar_opts;

typedef struct {
  uint64_t step;            /* iterations completed since creation            */
  int64_t  walker_steps;    /* step * z                                        */
  int64_t  stalls;          /* walker-iterations that kept theta = 0 because
                               the clamped chord was empty                     */
  int64_t  unbounded;       /* walker-iterations with a one-sided chord        */
  int32_t  status_bits;     /* OR of MHAR_ST_* seen so far                     */
  int32_t  precision;
  double   refresh_drift;   /* max |S_tracked - S_recomputed| at the last
                               refresh (mixed mode; 0 otherwise)               */
  double   max_violation;   /* max over walkers, rows of a_i x - b_i (FP64),
                               filled by mhar_check                            */
  double   eq_residual;     /* max over walkers of |A_E x - b_E|_inf (FP64),
                               filled by mhar_check                            */
  int64_t  kernel_launches; /* library kernels launched so far (graph replays
                               count every kernel node)                        */
  double   run_max_violation; /* max of a_i x - b_i over every audit since
                               creation (-inf before the first)              */
  double   run_eq_residual; /* max |A_E x - b_E|_inf over every audit          */
  int64_t  audits;          /* audits run since creation                       */
} mhar_stats;

#define MHAR_ST_UNBOUNDED 1
#define MHAR_ST_STALL     2
#define MHAR_ST_NONFINITE 4
#define MHAR_ST_DRIFT     8   /* a refresh found the tracked slack off its bound */

typedef struct mhar_ctx mhar_ctx;

/* Fills *opts with the defaults listed above. */
void mhar_default_opts(mhar_opts* opts);

/* Creates a context holding z walkers, all at x0 (Algorithm 2 initialises
 * every column of X to the same strictly interior point).
 *   A    m x n  (m >= 1, n >= 1)        b   m
 *   AE   mE x n or NULL when mE == 0    bE  mE or NULL
 *        0 <= mE < n, mE <= 25600; A_E of full row rank, condition number below about 1e7
 *        (MHAR_E_RANK otherwise)
 *   x0   n, strictly inside: b - A x0 > 0 and |A_E x0 - b_E|_inf <= 1e-9 (1 + |b_E|_inf)
 *   z    number of walkers; z <= 0 selects the paper's default max(m, n) + 1
 *   opts NULL for defaults
 * Copies all inputs to the device; when mE > 0 forms, in FP64 on the device,
 * the orthonormal rows Q = L^{-1} A_E (L the Cholesky factor of A_E A_E^T,
 * taken twice: CholeskyQR2), so that the projector of Section 3.2 is
 * P = I - Q^T Q; and prepares the per-mode operands.  On success *out is a new
 * context (free with mhar_destroy). */
int mhar_create(const double* A, const double* b, int m, int n,
                const double* AE, const double* bE, int mE,
                const double* x0, int z, const mhar_opts* opts, mhar_ctx** out);

/* Advances every walker `steps` iterations (Algorithm 2's loop) and writes
 * floor(steps / thin) samples to `out`, laid out out[s][k][i] (s-th sample,
 * walker k < W, coordinate i; FP64; W = opts.emit_walkers, or z when 0): the
 * points after iterations thin, 2 thin, ... of this call.  `out` may be NULL when steps < thin.  It is host memory
 * unless opts.out_on_device.  Iteration counters (and thus the random
 * streams) continue across calls.  Returns MHAR_E_UNBOUNDED /
 * MHAR_E_NONFINITE if any walker met that condition during the call (the
 * walkers concerned kept theta = 0; the state is still that of the last
 * iteration). */
int mhar_run(mhar_ctx* ctx, int64_t steps, int64_t thin, double* out);

/* Copies the current points (z x n, FP64, host) and the iteration counter. */
int mhar_get_state(const mhar_ctx* ctx, double* X, uint64_t* step);

/* Replaces the points (z x n host FP64, each strictly feasible) and the
 * iteration counter (checkpoint / resume; per-walker starts).  The stored
 * slack is recomputed. */
int mhar_set_state(mhar_ctx* ctx, const double* X, uint64_t step);

/* Chord and step length of every walker at the last iteration run:
 * lambda_min, lambda_max, theta (each z doubles on the host; any may be NULL). */
int mhar_get_chord(const mhar_ctx* ctx, double* lmin, double* lmax, double* theta);

/* Recomputes feasibility in FP64 from the current points (max_violation,
 * eq_residual) and returns all statistics. */
int mhar_check(mhar_ctx* ctx, mhar_stats* stats);

/* Statistics without the FP64 feasibility pass. */
int mhar_get_stats(const mhar_ctx* ctx, mhar_stats* stats);

/* Turns the per-iteration FP64 audit on or off for later mhar_run calls (the
 * opts.audit_every / opts.audit_walkers of mhar_create): every > 0 checks
 * walkers 0..walkers-1 (0: all) after every `every` iterations and folds the
 * results into mhar_stats.run_max_violation / run_eq_residual; every == 0
 * stops auditing (the running maxima are kept).  MHAR_E_ARG on negative
 * values or walkers > z. */
int mhar_set_audit(mhar_ctx* ctx, int32_t every, int32_t walkers);

/* Device-time profile of the walker step on the context's stream.  Captures
 * `iters` (1..4096) real iterations into a CUDA graph and times one replay
 * with CUDA events; times the direction kernels alone the same way (they are
 * idempotent for a fixed iteration counter); then times one slack refresh
 * (mixed mode).  Writes average device milliseconds:
 *   ms[0] direction draw (+ projection when mE > 0)   (Section 4.3); 0 in
 *         MHAR_MIXED_RECOMPUTE mode without equalities or preconditioner,
 *         where the chord kernel draws the next directions itself
 *   ms[1] the rest of one iteration: the fused tensor-core kernel in the
 *         tensor-core modes, the chord and update kernels otherwise
 *         (Sections 4.4-4.5)
 *   ms[2] one slack refresh (mixed mode; 0 otherwise)
 * The timed iterations are real: the chain and its counters advance. */
int mhar_time_kernels(mhar_ctx* ctx, int iters, double* ms);

/* Chord of every walker without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate --
 * a process that works inside a fixed device-memory budget reserved up front
 * (so a cudaMalloc inside a library would break its accounting or fail), or a
 * latency-critical loop that cannot take the device synchronisation cudaMalloc
 * and cudaFree may bring.  It computes, in FP64, for walker k the chord
 * (lmin[k], lmax[k]) of the line X[k] + lambda D[k] through {A x <= b}: over
 * the rows with a_i . d > 0 the least (b_i - a_i . x) / (a_i . d) is lmax,
 * over the rows with a_i . d < 0 the greatest is lmin; rows with a_i . d == 0
 * give nothing, a slack made negative by rounding counts as 0, and a side
 * without rows stays open (-inf / +inf).  A walker whose slack or a_i . d is
 * not finite gets lmin = lmax = NaN.  Unlike mhar_get_chord it takes no
 * rounding margin: the values are the plain FP64 ratios.
 *   A  m x n, b  m, X  z x n, D  z x n: device pointers, FP64, row-major, no
 *      padding; only read.
 *   lmin, lmax: z doubles each, device pointers, written.
 *   stream: cudaStream_t to enqueue on (NULL: legacy default stream).  The
 *      call returns once the work is enqueued; nothing is copied to the host.
 * Its only working memory is a fixed 1 MiB array compiled into the library,
 * which every GPU that loads the library holds until the process exits; it
 * limits z to 65536 (larger z: MHAR_E_ARG).  The first call on each device
 * looks up that array's device address (with that device current), so make
 * the first call on a device before any stream capture.  All calls share the
 * array and each call clears the part it uses; calls whose work overlaps on
 * the GPU race on it and give wrong results.
 * Returns MHAR_OK, MHAR_E_ARG or MHAR_E_CUDA; mhar_last_error(NULL) then
 * describes the failure (per host thread). */
int mhar_chord_noalloc(const double* A, const double* b, int m, int n,
                       const double* X, const double* D, int z,
                       double* lmin, double* lmax, void* stream);

/* ---- learned direction preconditioner ----------------------------------- */
/* The paper draws isotropic directions (Section 4.3) and assumes the body was
 * brought to near-isotropic position beforehand (Sections 1.2 and 3.1).  With
 * a preconditioner set, walker k's direction at every iteration becomes
 *     d = P (delta .* h + U g),
 * h ~ N(0, I_n) the Section 4.3 draw (Philox stream 0), g ~ N(0, I_r) from
 * Philox stream 2 (quad q of walker k at step t: counter (q, k, t_lo,
 * (t_hi << 8) | 2)), P the projector of Section 3.2 (identity when mE == 0).
 * The law of d does not depend on the walker's position and is centrally
 * symmetric, so the uniform distribution on the body stays the target of
 * the walk; only the speed of mixing changes.
 * In the tensor-core modes the coordinate scales sigma (see "Feasibility in
 * every mode" above) are A's column scales times one power of two, each kept
 * within [6.8 (delta_i + sum_q |U_iq|) / 65504, 2^8 sqrt(delta_i^2 +
 * (U U^T)_ii)] so that the scaled directions fit the FP16 range and stay
 * clear of its subnormals. */

/* Sets the preconditioner (delta != NULL) or removes it (delta == NULL:
 * isotropic directions again).  delta: n values, finite, >= 0; U: n x rank,
 * row-major, NULL when rank == 0; 0 <= rank <= 32.  The library copies both.
 * The walkers keep their points; the next iteration's directions are redrawn
 * with the new law, and the next mhar_run re-captures its graphs.
 * MHAR_E_ARG on a bad rank or pointer, MHAR_E_NONFINITE on a non-finite entry. */
int mhar_set_preconditioner(mhar_ctx* ctx, const double* delta, const double* U, int32_t rank);

/* Current preconditioner: *rank = -1 when none is set (delta and U are then
 * left untouched), else its rank, delta (n values) and U (n x rank,
 * row-major).  Any pointer may be NULL. */
int mhar_get_preconditioner(const mhar_ctx* ctx, double* delta, double* U, int32_t* rank);

/* Learns a preconditioner from the chain itself and freezes it.
 * Runs `warmup` iterations with the directions in force (their points are not
 * emitted), and keeps `snapshots` copies of all z points: after iterations
 * warmup - (snapshots - 1 - s) gap, s = 0..snapshots-1, gap =
 * max(1, floor(warmup / (2 snapshots))).  From those N = z snapshots points:
 *   Sigma = sum (x - mu)(x - mu)^T / (N - 1)                      (FP64)
 *   Y = Sigma Omega, Omega n x rank with column c = Philox stream 3 normals
 *     of walker c at step 0; `power_iters` times Q = orth(Y), Y = Sigma Q;
 *     Q = orth(Y) (Q factor of the thin QR with a positive diagonal in R)
 *   T = Q^T Sigma Q = V Lambda V^T; U = Q V Lambda_+^{1/2} (largest first)
 *   delta_i^2 = max(Sigma_ii - (U U^T)_ii, 1e-2 Sigma_ii, 1e-9 trace(Sigma)/n)
 * then sets (delta, U) as mhar_set_preconditioner does.  All of it runs on
 * the device; scratch memory (about 8 n^2 bytes) is allocated for the call.
 * Requires warmup >= 1, 1 <= snapshots <= warmup, z * snapshots >= 2,
 * 0 <= rank <= min(32, n), 0 <= power_iters <= 64 (else MHAR_E_ARG).  Returns
 * what the warm-up mhar_run returned if that failed, MHAR_E_NONFINITE if the
 * covariance is not finite. */
int mhar_fit_preconditioner(mhar_ctx* ctx, int64_t warmup, int32_t snapshots, int32_t rank,
                            int32_t power_iters);

/* The same fit in two halves, so that the shards of one ensemble on several
 * GPUs (disjoint walker0 ranges; walkers are independent chains, Section 4.1)
 * can pool their warm-up points into one fit: every shard calls
 * mhar_fit_moments with the same `shift`, the caller sums s1, s2 and count
 * over the shards (an all-reduce), and every shard calls
 * mhar_fit_from_moments with the sums, so all of them adopt the same
 * preconditioner -- the one a single context holding all the walkers fits.
 *
 * mhar_fit_moments: runs the warm-up of mhar_fit_preconditioner (same
 * iterations and snapshots) and returns, about `shift` (n, host; NULL =
 * walker 0's point at the first snapshot, which differs between shards),
 *   s1 = sum (x - shift)                 (n, host, caller-allocated)
 *   s2 = sum (x - shift)(x - shift)^T    (n x n row-major, symmetric)
 *   *count = z * snapshots
 * Requires warmup >= 1, 1 <= snapshots <= warmup, z * snapshots >= 2 (else
 * MHAR_E_ARG); MHAR_E_NONFINITE for a non-finite shift.
 * mhar_fit_from_moments: Sigma = (s2 - s1 s1^T / count) / (count - 1), then
 * the rank-`rank` + diagonal fit and its adoption exactly as in
 * mhar_fit_preconditioner.  Requires count >= 2 and the rank / power_iters
 * bounds above (else MHAR_E_ARG); MHAR_E_NONFINITE for non-finite moments. */
int mhar_fit_moments(mhar_ctx* ctx, int64_t warmup, int32_t snapshots, const double* shift,
                     double* s1, double* s2, int64_t* count);
int mhar_fit_from_moments(mhar_ctx* ctx, const double* s1, const double* s2, int64_t count,
                          int32_t rank, int32_t power_iters);

/* ---- batches of polytopes ------------------------------------------------- */
/* Many independent problems advanced together, two kernel launches per
 * iteration for all of them -- the chord kernel and the walker update (the
 * moves and the next operands) -- (the paper runs one polytope at a time; its
 * padding study, Section 6.2, is about filling the GPU with walkers, which a
 * batch does with problems).  Every problem is a full MHAR_MIXED_RECOMPUTE
 * sampler of its own (Algorithm 2, Lemma 4.2 on the tensor cores) with z
 * walkers, no equalities, and Philox key opts.seed + p for problem p, so
 * problem p's walk is the one a single context with that seed would take.
 * Two launch shapes, over the (problem, strip of 128 walkers) units,
 * largest first: each unit on a cluster of C CTAs along its rows (C = 1, 2,
 * 4, 8); or a persistent launch of one CTA per SM in which every CTA pulls
 * whole units from a device queue, with its pipelines carried from unit to
 * unit (shape 0).  mhar_batch_tune picks the shape, for the whole batch or
 * per bucket (below; in per-bucket mode each bucket has its own two
 * launches). */
typedef struct {
  const double* A;   /* m x n, row-major (copied)                 */
  const double* b;   /* m                                         */
  int32_t m, n;
  const double* x0;  /* n, strictly inside A x <= b                */
} mhar_problem;

typedef struct mhar_batch mhar_batch;

/* Creates the batch: `count` problems, z walkers each.  opts as for
 * mhar_create (precision is forced to MHAR_MIXED_RECOMPUTE; stream,
 * out_on_device and emit_walkers apply to every problem).  Errors as
 * mhar_create, for the first problem that fails. */
int mhar_batch_create(const mhar_problem* problems, int32_t count, int32_t z,
                      const mhar_opts* opts, mhar_batch** out);

/* Autotuner (no counterpart in the paper; its padding study, Section 6.2,
 * times throughput against the number of walkers).  Times `iters` (1..1024)
 * real iterations of the whole batch for every single shape -- the
 * persistent launch (0) and cluster sizes C in {1, 2, 4, 8} up to the
 * largest problem's row tiles.  Then, when the batch spans two or more
 * buckets, it tries a shape per bucket by coordinate descent from the best
 * single shape: one bucket at a time, most work first, takes every other
 * shape allowed for its problems, the whole batch timed each time; a change
 * stays only if the batch runs more than 1 % faster.  Per-bucket shapes are
 * kept if they beat the best single shape by more than 1 %.  *cluster (may
 * be NULL) receives the single shape kept (0 for the persistent launch), or
 * -1 for per-bucket shapes (mhar_batch_get_shapes tells them).  Every timed
 * iteration advances every walk (1 + iters per candidate).  Results do not
 * depend on the shapes. */
int mhar_batch_tune(mhar_batch* batch, int32_t iters, int32_t* cluster);

/* Sets one launch shape for the whole batch without timing: 0 the
 * persistent launch, 1, 2, 4 or 8 clusters of that many CTAs (MHAR_E_ARG
 * otherwise, or when C exceeds every problem's row tiles).  Results do not
 * depend on it. */
int mhar_batch_set_shape(mhar_batch* batch, int32_t shape);

/* Buckets: the problems of a batch fall into buckets by the 64-column K
 * chunks of their operands (n rounded up to a multiple of 64): bucket 0 one
 * chunk (n <= 64), 1 two, 2 three or four, 3 five to eight, 4 more.  In
 * per-bucket mode every non-empty bucket's units are launched with the
 * bucket's own shape, each bucket on a stream of its own forked from and
 * joined back into the batch's stream, so that the buckets run side by side;
 * the step counters advance after all of them (one launch per bucket and
 * iteration).  mhar_batch_set_bucket_shape switches to per-bucket mode (on
 * the first switch every bucket takes the batch's current shape, clamped to
 * its problems' row tiles) and sets bucket `bucket`'s shape; MHAR_E_ARG for
 * an empty bucket or a shape mhar_batch_set_shape would reject for that
 * bucket's problems.  mhar_batch_set_shape returns to one shape. */
int mhar_batch_set_bucket_shape(mhar_batch* batch, int32_t bucket, int32_t shape);

/* Current shapes: *per_bucket (may be NULL) is 1 in per-bucket mode, else 0;
 * shape[5] (may be NULL) receives every bucket's shape (-1 for an empty
 * bucket; with one shape for the batch, that shape); bucket_of (may be NULL,
 * one entry per problem) the bucket of every problem. */
int mhar_batch_get_shapes(const mhar_batch* batch, int32_t* per_bucket, int32_t* shape,
                          int32_t* bucket_of);

/* Advances every problem `steps` iterations; out[p] receives problem p's
 * floor(steps / thin) samples, laid out as for mhar_run (out[p] may be NULL
 * to skip a problem).  Returns the first problem's failure code (unbounded,
 * non-finite) after the whole call. */
int mhar_batch_run(mhar_batch* batch, int64_t steps, int64_t thin, double* const* out);

/* Problem p's points (z x n, host FP64) and iteration counter. */
int mhar_batch_get_state(const mhar_batch* batch, int32_t problem, double* X, uint64_t* step);

/* mhar_check for problem p (kernel_launches adds the batch's own launches). */
int mhar_batch_check(mhar_batch* batch, int32_t problem, mhar_stats* stats);

/* mhar_set_audit for every problem of the batch (audits run after every
 * `every` iterations of mhar_batch_run). */
int mhar_batch_set_audit(mhar_batch* batch, int32_t every, int32_t walkers);

/* Description of the batch's last error (never NULL). */
const char* mhar_batch_last_error(const mhar_batch* batch);

/* Frees the batch and every problem's device memory; NULL is ignored. */
void mhar_batch_destroy(mhar_batch* batch);

/* Name of the kernel that runs the chord of one iteration on this context
 * (e.g. "recompute_ts_kernel"); never NULL. */
const char* mhar_kernel_name(const mhar_ctx* ctx);

/* Human-readable description of the last error on ctx (never NULL); with
 * ctx == NULL, on this host thread, the last failed mhar_create /
 * mhar_batch_create, or the last mhar_chord_noalloc failure (cleared when a
 * later mhar_chord_noalloc call succeeds). */
const char* mhar_last_error(const mhar_ctx* ctx);

/* Name of a return code. */
const char* mhar_strerror(int code);

/* The return code mhar_run gives for a device status word: status_bits, the
 * OR of MHAR_ST_* seen, and wait_expired, nonzero when a bounded wait in a
 * tensor-core kernel ran out (the kernel stops waiting there and raises the
 * flag; that call's results are not to be trusted).  Precedence: timeout,
 * non-finite, drift, unbounded; stalls alone are not an error. */
int mhar_status_code(int32_t status_bits, int32_t wait_expired);

/* Frees the context and its device memory; NULL is ignored. */
void mhar_destroy(mhar_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
