/*
 * mhar_oracle.h -- plain single-threaded FP64 CPU oracle for Matrix Hit-and-Run.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against
 * the paper.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  The product path never links, loads or calls it,
 * and it shares no code, header, table or constant with the CUDA sources.
 *
 * What it follows (Vazquez Corte & Montiel, "Novel Matrix Hit and Run for
 * Sampling Polytopes and Its GPU Implementation", arXiv 2104.07097):
 *   - Algorithm 2 (MHAR pseudocode), Section 4: z walks advanced together.
 *   - Section 3.2, the projection matrix P = I - A_E^T (A_E A_E^T)^{-1} A_E.
 *   - Section 4.3 "Generating D": i.i.d. N(0,1) direction entries by Box-Muller,
 *     D = H when m_E = 0, D = P H otherwise.
 *   - Section 4.4 "Finding the line sets": lambda_i = (b_i - a_i x)/(a_i d),
 *     lambda_min = max over a_i d < 0, lambda_max = min over a_i d > 0.
 *   - Section 4.5 "Choosing samples" (Lemma 4.3): theta uniform on the open
 *     chord, x <- x + theta d.
 * Random numbers: the paper does not name a generator.  Both sides implement
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) from its published
 * definition, with the counter layout documented below.
 *
 * Parity pins live in tests/ (known-answer Philox vectors, closed forms on the
 * interval and the square, projector identities, cube / simplex / polygon
 * distributions, Friedman-Rafsky).
 */
#ifndef MHAR_ORACLE_H
#define MHAR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Random-stream ids, carried in the top byte of counter word 3. */
#define ORC_STREAM_DIRECTION 0u
#define ORC_STREAM_CHORD     1u
#define ORC_STREAM_LOWRANK   2u   /* the r low-rank normals of a preconditioned direction */
#define ORC_STREAM_FIT       3u   /* the starting block of the preconditioner fit        */

/* Status bits returned by orc_chord / orc_mhar_run (OR-ed over walkers). */
#define ORC_UNBOUNDED 1   /* no row with a.d > 0 or no row with a.d < 0      */
#define ORC_STALL     2   /* lambda_min > lambda_max after clamping the slack */
#define ORC_NONFINITE 4   /* a non-finite slack, a.d or theta                 */

/* Philox4x32-10 block function: out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* h[0..n): the N(0,1) entries of walker `walker`'s direction at step `step`.
 * Counter for quad q: (q, walker, step_lo32, (step_hi24 << 8) | STREAM_DIRECTION);
 * key = (seed_lo32, seed_hi32).  Each 32-bit word w maps to u = (w + 1/2) 2^-32;
 * Box-Muller on (u0,u1) gives h[4q], h[4q+1]; on (u2,u3) gives h[4q+2], h[4q+3]. */
void orc_direction_normals(uint64_t seed, uint64_t step, uint32_t walker, int n, double* h);

/* `count` N(0,1) values of stream `stream` for (step, walker): quads q with
 * counter (q, walker, step_lo32, (step_hi24 << 8) | stream), Box-Muller as
 * above.  Stream 0 is orc_direction_normals. */
void orc_stream_normals(uint64_t seed, uint64_t step, uint32_t walker, uint32_t stream, int count,
                        double* out);

/* u in (0,1) for the point drawn on walker `walker`'s chord at step `step`:
 * counter (0, walker, step_lo32, (step_hi24 << 8) | STREAM_CHORD), word 0. */
double orc_chord_uniform(uint64_t seed, uint64_t step, uint32_t walker);

/* Dense projector P (n x n, row-major) onto the null space of A_E (mE x n).
 * Returns 0, or -1 if A_E A_E^T is not positive definite. */
int orc_projector(const double* AE, int mE, int n, double* P);

/* Chord of the line x + lambda d through {A x <= b}: writes lambda_min and
 * lambda_max (+-infinity when a side is open).  Slack is b - A x, computed
 * fresh and clamped at 0.  Returns status bits. */
int orc_chord(const double* A, const double* b, int m, int n,
              const double* x, const double* d, double* lmin, double* lmax);

/* Runs Algorithm 2 for `steps` iterations starting at global step `step0`.
 *   X      z x n, row k = walker k (in: start points, out: final points);
 *   walker0  global index of row 0 (walkers are independent, so a shard of
 *            walkers reproduces the same rows of an unsharded run);
 *   P      n x n projector or NULL when mE == 0;
 *   out    floor(steps/thin) x z x n samples, X after steps thin, 2 thin, ...
 *          (may be NULL);
 *   t_tr, lmin_tr, lmax_tr   steps x z traces (each may be NULL).
 * Returns the OR of status bits over all walkers and steps. */
int orc_mhar_run(const double* A, const double* b, int m, int n,
                 const double* P, double* X, int z, uint32_t walker0,
                 uint64_t seed, uint64_t step0, int64_t steps, int64_t thin,
                 double* out, double* t_tr, double* lmin_tr, double* lmax_tr);

/* Same with a direction preconditioner: each direction is
 *   d = P (delta .* h + U g),   h ~ N(0, I_n) (stream 0),  g ~ N(0, I_r) (stream 2),
 * delta (n), U (n x r row-major), 1 <= r <= 32 or r == 0 with U NULL (diagonal only).
 * The law of d is centrally symmetric, so the chain still targets the
 * uniform distribution on the body. */
int orc_mhar_run_pre(const double* A, const double* b, int m, int n,
                     const double* P, double* X, int z, uint32_t walker0,
                     uint64_t seed, uint64_t step0, int64_t steps, int64_t thin,
                     const double* delta, const double* U, int r,
                     double* out, double* t_tr, double* lmin_tr, double* lmax_tr);

#ifdef __cplusplus
}
#endif
#endif
