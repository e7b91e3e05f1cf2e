/*
 * mhar_oracle.c -- plain single-threaded FP64 CPU oracle for Matrix Hit-and-Run.
 *
 * TEST INFRASTRUCTURE ONLY (see mhar_oracle.h).  Every function is written for
 * a reader checking it against the paper by eye: plain loops, FP64, no
 * blocking, no fusion, no reordering beyond what the text states.
 */
#include "mhar_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Section 5): ten rounds of            */
/*   (L0,R0,L1,R1) -> (hi(M0 R0) ^ L0... ) with Weyl-sequence key bumps.       */
/* Round constants as published: multipliers M0, M1 and key bumps W0, W1.     */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    if (r < 9) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void make_counter(uint32_t q, uint32_t walker, uint64_t step, uint32_t stream,
                         uint32_t ctr[4]) {
  ctr[0] = q;
  ctr[1] = walker;
  ctr[2] = (uint32_t)(step & 0xffffffffu);
  ctr[3] = ((uint32_t)((step >> 32) & 0xffffffu) << 8) | (stream & 0xffu);
}

/* A 32-bit word as a uniform in the open interval (0,1): (w + 1/2) 2^-32.
 * Exact in FP64. */
static double word_to_open_uniform(uint32_t w) {
  return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* Box-Muller (Box & Muller 1958): for u_a, u_b uniform on (0,1),
 * sqrt(-2 ln u_a) cos(2 pi u_b) and sqrt(-2 ln u_a) sin(2 pi u_b) are
 * independent N(0,1).  Section 4.3 of the paper. */
static void box_muller(double ua, double ub, double* z0, double* z1) {
  const double two_pi = 6.283185307179586476925286766559;
  double r = sqrt(-2.0 * log(ua));
  double th = two_pi * ub;
  *z0 = r * cos(th);
  *z1 = r * sin(th);
}

void orc_stream_normals(uint64_t seed, uint64_t step, uint32_t walker, uint32_t stream, int n,
                        double* h) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  int quads = (n + 3) / 4;
  for (int q = 0; q < quads; ++q) {
    uint32_t ctr[4], w[4];
    make_counter((uint32_t)q, walker, step, stream, ctr);
    orc_philox4x32_10(ctr, key, w);
    double z[4];
    box_muller(word_to_open_uniform(w[0]), word_to_open_uniform(w[1]), &z[0], &z[1]);
    box_muller(word_to_open_uniform(w[2]), word_to_open_uniform(w[3]), &z[2], &z[3]);
    for (int e = 0; e < 4; ++e) {
      int i = 4 * q + e;
      if (i < n) h[i] = z[e];
    }
  }
}

void orc_direction_normals(uint64_t seed, uint64_t step, uint32_t walker, int n, double* h) {
  orc_stream_normals(seed, step, walker, ORC_STREAM_DIRECTION, n, h);
}

double orc_chord_uniform(uint64_t seed, uint64_t step, uint32_t walker) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t ctr[4], w[4];
  make_counter(0u, walker, step, ORC_STREAM_CHORD, ctr);
  orc_philox4x32_10(ctr, key, w);
  return word_to_open_uniform(w[0]);
}

/* ------------------------------------------------------------------------- */
/* Projection matrix, Section 3.2: P = I - A_E^T (A_E A_E^T)^{-1} A_E.        */
/* The inverse is applied through a Cholesky factorisation of the Gram        */
/* matrix G = A_E A_E^T (symmetric positive definite when A_E has full row    */
/* rank, which the paper's "no redundant constraints" assumption gives).      */
/* ------------------------------------------------------------------------- */
int orc_projector(const double* AE, int mE, int n, double* P) {
  double* G = (double*)calloc((size_t)mE * mE, sizeof(double));
  double* W = (double*)calloc((size_t)mE * n, sizeof(double));
  if (!G || !W) { free(G); free(W); return -1; }
  /* G = A_E A_E^T */
  for (int r = 0; r < mE; ++r)
    for (int c = 0; c < mE; ++c) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += AE[(size_t)r * n + k] * AE[(size_t)c * n + k];
      G[(size_t)r * mE + c] = s;
    }
  /* Cholesky G = L L^T, L stored in the lower triangle of G. */
  for (int j = 0; j < mE; ++j) {
    double d = G[(size_t)j * mE + j];
    for (int k = 0; k < j; ++k) d -= G[(size_t)j * mE + k] * G[(size_t)j * mE + k];
    if (!(d > 0.0)) { free(G); free(W); return -1; }
    double ljj = sqrt(d);
    G[(size_t)j * mE + j] = ljj;
    for (int i = j + 1; i < mE; ++i) {
      double s = G[(size_t)i * mE + j];
      for (int k = 0; k < j; ++k) s -= G[(size_t)i * mE + k] * G[(size_t)j * mE + k];
      G[(size_t)i * mE + j] = s / ljj;
    }
  }
  /* W = G^{-1} A_E, column by column of A_E: solve L y = a, then L^T w = y. */
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < mE; ++i) {
      double s = AE[(size_t)i * n + c];
      for (int k = 0; k < i; ++k) s -= G[(size_t)i * mE + k] * W[(size_t)k * n + c];
      W[(size_t)i * n + c] = s / G[(size_t)i * mE + i];
    }
    for (int i = mE - 1; i >= 0; --i) {
      double s = W[(size_t)i * n + c];
      for (int k = i + 1; k < mE; ++k) s -= G[(size_t)k * mE + i] * W[(size_t)k * n + c];
      W[(size_t)i * n + c] = s / G[(size_t)i * mE + i];
    }
  }
  /* P = I - A_E^T W */
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = 0; k < mE; ++k) s += AE[(size_t)k * n + r] * W[(size_t)k * n + c];
      P[(size_t)r * n + c] = (r == c ? 1.0 : 0.0) - s;
    }
  free(G);
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Line set, Section 4.4.  For each inequality row i:                          */
/*   s_i = b_i - a_i x   (the slack, computed fresh as in Lemma 4.2 step 2),   */
/*   g_i = a_i d,                                                              */
/*   lambda_i = s_i / g_i;                                                     */
/*   lambda_max = min{lambda_i : g_i > 0},  lambda_min = max{lambda_i : g_i < 0}.*/
/* Rows with g_i == 0 belong to neither set (the paper's strict signs).        */
/* A slack that rounding made negative is clamped to 0 before the ratio.       */
/* ------------------------------------------------------------------------- */
int orc_chord(const double* A, const double* b, int m, int n,
              const double* x, const double* d, double* lmin, double* lmax) {
  double lo = -INFINITY, hi = INFINITY;
  int status = 0;
  for (int i = 0; i < m; ++i) {
    const double* a = A + (size_t)i * n;
    double ax = 0.0, ad = 0.0;
    for (int k = 0; k < n; ++k) { ax += a[k] * x[k]; ad += a[k] * d[k]; }
    double s = b[i] - ax;
    if (!isfinite(s) || !isfinite(ad)) { status |= ORC_NONFINITE; continue; }
    if (s < 0.0) s = 0.0;
    if (ad > 0.0) {
      double lam = s / ad;
      if (lam < hi) hi = lam;
    } else if (ad < 0.0) {
      double lam = s / ad;
      if (lam > lo) lo = lam;
    }
  }
  if (isinf(lo) || isinf(hi)) status |= ORC_UNBOUNDED;
  *lmin = lo;
  *lmax = hi;
  return status;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2.  Per iteration j: generate H; D = H (m_E = 0) or D = P H;      */
/* find every walk's chord; draw theta^k uniformly on it; x^k += theta^k d^k;  */
/* every `thin` iterations append all z columns to the sample set.             */
/* Walks are independent (Section 4.1), so the loop over k is just the         */
/* columns of the padded matrices taken one at a time.                         */
/* ------------------------------------------------------------------------- */
int orc_mhar_run_pre(const double* A, const double* b, int m, int n,
                     const double* P, double* X, int z, uint32_t walker0,
                     uint64_t seed, uint64_t step0, int64_t steps, int64_t thin,
                     const double* delta, const double* U, int r,
                     double* out, double* t_tr, double* lmin_tr, double* lmax_tr) {
  double* h = (double*)malloc((size_t)n * sizeof(double));
  double* d = (double*)malloc((size_t)n * sizeof(double));
  double* g = (double*)malloc((size_t)(r > 0 ? r : 1) * sizeof(double));
  if (!h || !d || !g) { free(h); free(d); free(g); return -1; }
  int status = 0;
  int64_t emitted = 0;
  for (int64_t j = 0; j < steps; ++j) {
    uint64_t step = step0 + (uint64_t)j;
    for (int k = 0; k < z; ++k) {
      uint32_t walker = walker0 + (uint32_t)k;
      double* x = X + (size_t)k * n;
      /* Generate h^k (Section 4.3). */
      orc_direction_normals(seed, step, walker, n, h);
      /* Preconditioned draw: h <- delta .* h + U g (centrally symmetric). */
      if (delta) {
        if (r > 0) orc_stream_normals(seed, step, walker, ORC_STREAM_LOWRANK, r, g);
        for (int i = 0; i < n; ++i) {
          double s = delta[i] * h[i];
          for (int c = 0; c < r; ++c) s += U[(size_t)i * r + c] * g[c];
          h[i] = s;
        }
      }
      /* d^k = h^k, or P h^k when there are equalities. */
      if (P) {
        for (int row = 0; row < n; ++row) {
          double s = 0.0;
          for (int c = 0; c < n; ++c) s += P[(size_t)row * n + c] * h[c];
          d[row] = s;
        }
      } else {
        memcpy(d, h, (size_t)n * sizeof(double));
      }
      /* Chord Lambda^k = (lambda_min, lambda_max) (Section 4.4). */
      double lo, hi;
      int st = orc_chord(A, b, m, n, x, d, &lo, &hi);
      double t = 0.0;
      if (st & (ORC_UNBOUNDED | ORC_NONFINITE)) {
        t = 0.0; /* the walk stays; the status reports why */
      } else if (lo > hi) {
        st |= ORC_STALL;
        t = 0.0;
      } else {
        /* theta^k uniform on the chord (Section 4.5). */
        double u = orc_chord_uniform(seed, step, walker);
        t = lo + u * (hi - lo);
      }
      status |= st;
      for (int i = 0; i < n; ++i) x[i] += t * d[i];
      if (t_tr) t_tr[(size_t)j * z + k] = t;
      if (lmin_tr) lmin_tr[(size_t)j * z + k] = lo;
      if (lmax_tr) lmax_tr[(size_t)j * z + k] = hi;
    }
    /* Thinning: emit X after iterations thin, 2 thin, ... */
    if (out && thin > 0 && ((j + 1) % thin) == 0) {
      memcpy(out + (size_t)emitted * z * n, X, (size_t)z * n * sizeof(double));
      ++emitted;
    }
  }
  free(h);
  free(d);
  free(g);
  return status;
}

/* Algorithm 2 with isotropic directions (Section 4.3). */
int orc_mhar_run(const double* A, const double* b, int m, int n,
                 const double* P, double* X, int z, uint32_t walker0,
                 uint64_t seed, uint64_t step0, int64_t steps, int64_t thin,
                 double* out, double* t_tr, double* lmin_tr, double* lmax_tr) {
  return orc_mhar_run_pre(A, b, m, n, P, X, z, walker0, seed, step0, steps, thin, NULL, NULL, 0,
                          out, t_tr, lmin_tr, lmax_tr);
}
