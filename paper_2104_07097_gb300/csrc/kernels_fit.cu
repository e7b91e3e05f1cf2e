// kernels_fit.cu -- learned direction preconditioner: covariance of warm-up
// points and the rank-r plus diagonal fit, in FP64 on CUDA cores.
//
// The paper draws isotropic directions and assumes the body was brought to
// near-isotropic position beforehand (Sections 1.2 and 3.1).  The fit learns
// that position from the chain itself:
//   1. Sigma = sum_k (x_k - mu)(x_k - mu)^T / (N - 1) over the N warm-up
//      points (all walkers at every snapshot), accumulated about a shift c
//      (walker 0's first snapshot) as S1 = sum (x - c), S2 = sum (x - c)(x - c)^T,
//      Sigma = (S2 - S1 S1^T / N) / (N - 1);
//   2. randomized subspace iteration: Y = Sigma Omega (Omega's column c is
//      Philox stream 3 for walker c at step 0), then power_iters times
//      Q = orth(Y), Y = Sigma Q, and finally Q = orth(Y);
//      orth is the Q factor with a positive diagonal in R, computed by
//      classical Gram-Schmidt with one re-orthogonalisation pass;
//   3. Rayleigh-Ritz: T = Q^T Sigma Q, T = V Lambda V^T by cyclic Jacobi
//      rotations (Golub & Van Loan, Matrix Computations, Section 8.5),
//      U = Q V Lambda_+^{1/2}, largest eigenvalue first;
//   4. delta_i^2 = max(Sigma_ii - (U U^T)_ii, 1e-2 Sigma_ii, 1e-9 tr(Sigma) / n).
// The host then sets the coordinate scales of the tensor-core operands from
// the fitted (delta, U), as for a preconditioner given by the caller.
// None of this is on the per-iteration path; it runs once, then the
// preconditioner is frozen.
#include <cmath>

#include "mhar_device.cuh"
#include "mhar_internal.h"

namespace mhar {
namespace {

constexpr int kCovTile = 64;     // Sigma tile edge
constexpr int kCovChunk = 1024;  // walkers per block
constexpr int kCovStage = 16;    // walkers staged in shared memory at once
constexpr int kFitThreads = 1024;
constexpr double kEpsRel = 1e-2;
constexpr double kEpsAbs = 1e-9;

__device__ __forceinline__ double point(int mode, const double* X64, const float* Xhi,
                                        const float* Xlo, size_t idx) {
  return mode == 0 ? X64[idx] : static_cast<double>(Xhi[idx]) + static_cast<double>(Xlo[idx]);
}

__global__ void fit_shift_kernel(int mode, int n, const double* X64, const float* Xhi,
                                 const float* Xlo, double* shift) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    shift[i] = point(mode, X64, Xhi, Xlo, static_cast<size_t>(i));
}

// One (row tile ti, column tile tj >= ti) of S2 and, on diagonal tiles, the
// matching part of S1, over one chunk of walkers.  16 x 16 threads, 4 x 4
// outputs each.
__global__ void __launch_bounds__(256)
cov_accumulate_kernel(int mode, int z, int n, int n_ld, int tiles, const double* X64,
                      const float* Xhi, const float* Xlo, const double* shift, double* s1,
                      double* s2) {
  int t = blockIdx.x, ti = 0;
  while (t >= tiles - ti) {
    t -= tiles - ti;
    ++ti;
  }
  const int tj = ti + t;
  // Centred values (x - shift, formed in FP64) are staged as FP32; the
  // products of one stage of kCovStage walkers are summed in FP32 and each
  // stage's sum is added to an FP64 total, so FP64 work is 1 / kCovStage of
  // the products (FP64 runs at a small fraction of the FP32 rate on GB300).
  __shared__ float xa[kCovStage][kCovTile];
  __shared__ float xb[kCovStage][kCovTile];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;
  double col_sum = 0.0;
  const int kbeg = blockIdx.y * kCovChunk;
  const int kend = min(z, kbeg + kCovChunk);
  for (int kb = kbeg; kb < kend; kb += kCovStage) {
    for (int e = threadIdx.x; e < kCovStage * kCovTile; e += blockDim.x) {
      const int w = e / kCovTile, q = e % kCovTile, k = kb + w;
      const int ia = ti * kCovTile + q, ib = tj * kCovTile + q;
      double va = 0.0, vb = 0.0;
      if (k < kend) {
        const size_t row = static_cast<size_t>(k) * n_ld;
        if (ia < n) va = point(mode, X64, Xhi, Xlo, row + ia) - shift[ia];
        if (ib < n) vb = point(mode, X64, Xhi, Xlo, row + ib) - shift[ib];
      }
      xa[w][q] = static_cast<float>(va);
      xb[w][q] = static_cast<float>(vb);
    }
    __syncthreads();
    float part[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) part[r][q] = 0.0f;
#pragma unroll 4
    for (int w = 0; w < kCovStage; ++w) {
      float a[4], bb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = xa[w][ty * 4 + r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bb[q] = xb[w][tx * 4 + q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) part[r][q] = fmaf(a[r], bb[q], part[r][q]);
      if (ti == tj && threadIdx.x < kCovTile) col_sum += static_cast<double>(xa[w][threadIdx.x]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] += static_cast<double>(part[r][q]);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = ti * kCovTile + ty * 4 + r, jj = tj * kCovTile + tx * 4 + q;
      if (i < n && jj < n) atomicAdd(&s2[static_cast<size_t>(i) * n + jj], acc[r][q]);
    }
  if (ti == tj && threadIdx.x < kCovTile) {
    const int i = ti * kCovTile + threadIdx.x;
    if (i < n) atomicAdd(&s1[i], col_sum);
  }
}

// Sigma (full, symmetric) from S1 and the upper tiles of S2.
__global__ void cov_finalize_kernel(int n, double N, const double* s1, const double* s2,
                                    double* sigma, int* flag) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n) * n) return;
  const int i = static_cast<int>(idx / n), jj = static_cast<int>(idx % n);
  const int lo = min(i, jj), hi = max(i, jj);
  const double v = (s2[static_cast<size_t>(lo) * n + hi] - s1[i] * s1[jj] / N) / (N - 1.0);
  if (!isfinite(v)) atomicOr(flag, 1);
  sigma[idx] = v;
}

// Omega: column c < rank holds stream 3's normals of walker c at step 0.
__global__ void omega_kernel(uint64_t seed, int n, int rank, double* Q) {
  const int quads = (n + 3) >> 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kMaxPcRank * quads) return;
  const int c = idx / quads, q = idx % quads;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (c < rank) {
    const U4 w = philox_block(seed, 0ull, static_cast<uint32_t>(c), static_cast<uint32_t>(q),
                              kStreamFit);
    box_muller_f64(open_unit_f64(w.x), open_unit_f64(w.y), v[0], v[1]);
    box_muller_f64(open_unit_f64(w.z), open_unit_f64(w.w), v[2], v[3]);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (4 * q + e < n) Q[static_cast<size_t>(4 * q + e) * kMaxPcRank + c] = v[e];
}

// Y = Sigma Q (n x n times n x 32): a warp per row, a lane per column.
__global__ void symm_block_kernel(int n, const double* __restrict__ sigma,
                                  const double* __restrict__ Q, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const double* row = sigma + static_cast<size_t>(i) * n;
  double acc = 0.0;
  for (int k = 0; k < n; ++k) acc = fma(row[k], Q[static_cast<size_t>(k) * kMaxPcRank + lane], acc);
  Y[static_cast<size_t>(i) * kMaxPcRank + lane] = acc;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < static_cast<int>(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Q = orth(Y) for the first `rank` columns (zero beyond): classical
// Gram-Schmidt, each column projected out twice, then normalised.  One block.
__global__ void __launch_bounds__(kFitThreads)
orth_kernel(int n, int rank, const double* __restrict__ Y, double* __restrict__ Q) {
  __shared__ double dots[kMaxPcRank];
  __shared__ double red[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < kMaxPcRank; ++c) {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      Q[static_cast<size_t>(i) * kMaxPcRank + c] = c < rank ? Y[static_cast<size_t>(i) * kMaxPcRank + c] : 0.0;
    if (c >= rank) continue;
    for (int pass = 0; pass < 2; ++pass) {
      __syncthreads();
      if (warp < c) {
        double acc = 0.0;
        for (int i = lane; i < n; i += 32)
          acc = fma(Q[static_cast<size_t>(i) * kMaxPcRank + warp],
                    Q[static_cast<size_t>(i) * kMaxPcRank + c], acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) dots[warp] = acc;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = Q[static_cast<size_t>(i) * kMaxPcRank + c];
        for (int p = 0; p < c; ++p) v = fma(-dots[p], Q[static_cast<size_t>(i) * kMaxPcRank + p], v);
        Q[static_cast<size_t>(i) * kMaxPcRank + c] = v;
      }
    }
    __syncthreads();
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = Q[static_cast<size_t>(i) * kMaxPcRank + c];
      part = fma(v, v, part);
    }
    const double nrm2 = block_sum(part, red);
    const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      Q[static_cast<size_t>(i) * kMaxPcRank + c] *= inv;
    __syncthreads();
  }
}

// Rayleigh-Ritz on span(Q) with SQ = Sigma Q, the diagonal floor, and the
// outputs.  One block of 1024 threads; Jacobi on warp 0.
__global__ void __launch_bounds__(kFitThreads)
ritz_kernel(int n, int n_ld, int rank, const double* __restrict__ Q, const double* __restrict__ SQ,
            const double* __restrict__ sigma_mat, double* delta64, double* U64, float* delta32,
            float* U32, float* coord_scale, int* flag) {
  __shared__ double T[kMaxPcRank][kMaxPcRank + 1];
  __shared__ double V[kMaxPcRank][kMaxPcRank + 1];
  __shared__ double lam[kMaxPcRank];
  __shared__ int perm[kMaxPcRank];
  __shared__ double red[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // T = Q^T (Sigma Q), symmetrised.
  {
    const int a = warp, bcol = lane;
    double acc = 0.0;
    if (a < rank && bcol < rank)
      for (int i = 0; i < n; ++i)
        acc = fma(Q[static_cast<size_t>(i) * kMaxPcRank + a], SQ[static_cast<size_t>(i) * kMaxPcRank + bcol], acc);
    T[a][bcol] = acc;
    V[a][bcol] = a == bcol ? 1.0 : 0.0;
  }
  __syncthreads();
  {
    const int a = warp, bcol = lane;
    const double s = 0.5 * (T[a][bcol] + T[bcol][a]);
    __syncthreads();
    T[a][bcol] = s;
  }
  __syncthreads();
  if (warp == 0 && rank > 1) {
    for (int sweep = 0; sweep < 60; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int a = 0; a < rank; ++a) {
        const double v = lane < rank ? T[a][lane] : 0.0;
        tot += v * v;
        if (lane != a) off += v * v;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (!(off > 1e-30 * tot)) break;
      for (int p = 0; p < rank - 1; ++p) {
        for (int q = p + 1; q < rank; ++q) {
          const double apq = T[p][q];
          if (apq == 0.0) continue;
          const double tau = (T[q][q] - T[p][p]) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double cs = 1.0 / sqrt(1.0 + t * t);
          const double sn = t * cs;
          __syncwarp();
          // T <- T J (columns p, q), V <- V J.
          if (lane < rank) {
            const double tp = T[lane][p], tq = T[lane][q];
            T[lane][p] = cs * tp - sn * tq;
            T[lane][q] = sn * tp + cs * tq;
            const double vp = V[lane][p], vq = V[lane][q];
            V[lane][p] = cs * vp - sn * vq;
            V[lane][q] = sn * vp + cs * vq;
          }
          __syncwarp();
          // T <- J^T T (rows p, q).
          if (lane < rank) {
            const double tp = T[p][lane], tq = T[q][lane];
            T[p][lane] = cs * tp - sn * tq;
            T[q][lane] = sn * tp + cs * tq;
          }
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Eigenvalues largest first (selection sort over at most 32 values).
    bool used[kMaxPcRank];
    for (int a = 0; a < kMaxPcRank; ++a) used[a] = false;
    for (int a = 0; a < rank; ++a) {
      int best = -1;
      for (int q = 0; q < rank; ++q)
        if (!used[q] && (best < 0 || T[q][q] > T[best][best])) best = q;
      used[best] = true;
      perm[a] = best;
      lam[a] = fmax(T[best][best], 0.0);
    }
  }
  __syncthreads();
  // Trace of Sigma for the absolute floor.
  double part = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) part += sigma_mat[static_cast<size_t>(i) * n + i];
  const double tr = block_sum(part, red);
  // Rows of U, delta and the coordinate scale: a warp per coordinate.
  for (int i = warp; i < n_ld; i += blockDim.x >> 5) {
    double u = 0.0;
    if (i < n && lane < rank) {
      const int col = perm[lane];
      for (int bcol = 0; bcol < rank; ++bcol)
        u = fma(Q[static_cast<size_t>(i) * kMaxPcRank + bcol], V[bcol][col], u);
      u *= sqrt(lam[lane]);
    }
    double u2 = u * u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u2 += __shfl_xor_sync(0xffffffffu, u2, o);
    double d2 = 0.0, sc = 1.0;
    if (i < n) {
      const double sii = sigma_mat[static_cast<size_t>(i) * n + i];
      d2 = fmax(sii - u2, fmax(kEpsRel * sii, kEpsAbs * tr / n));
      const double var = d2 + u2;
      if (!isfinite(var) || !isfinite(u)) atomicOr(flag, 1);
      if (var > 0.0 && isfinite(var)) {
        int e = 0;
        frexp(sqrt(var), &e);
        sc = ldexp(1.0, e);
      }
    }
    U64[static_cast<size_t>(i) * kMaxPcRank + lane] = u;
    U32[static_cast<size_t>(i) * kMaxPcRank + lane] = static_cast<float>(u);
    if (lane == 0) {
      delta64[i] = sqrt(d2);
      delta32[i] = static_cast<float>(sqrt(d2));
      if (coord_scale) coord_scale[i] = static_cast<float>(sc);
    }
  }
}

inline int blocks_for(long long count, int per_block) {
  return static_cast<int>((count + per_block - 1) / per_block);
}

}  // namespace

cudaError_t launch_fit_shift(mhar_ctx* c, FitScratch* f) {
  const int mode = c->opts.precision == MHAR_FP64 ? 0 : 1;
  fit_shift_kernel<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(mode, c->n, c->d.X64, c->d.Xhi,
                                                                c->d.Xlo, f->shift);
  return cudaGetLastError();
}

cudaError_t launch_fit_accumulate(mhar_ctx* c, FitScratch* f) {
  const int mode = c->opts.precision == MHAR_FP64 ? 0 : 1;
  const int tiles = blocks_for(c->n, kCovTile);
  dim3 grid(tiles * (tiles + 1) / 2, blocks_for(c->z, kCovChunk));
  cov_accumulate_kernel<<<grid, 256, 0, c->stream>>>(mode, c->z, c->n, c->n_ld, tiles, c->d.X64,
                                                     c->d.Xhi, c->d.Xlo, f->shift, f->s1, f->s2);
  return cudaGetLastError();
}

cudaError_t launch_fit_factor(mhar_ctx* c, FitScratch* f, long long samples, int rank,
                              int power_iters) {
  const int n = c->n;
  cov_finalize_kernel<<<blocks_for(static_cast<long long>(n) * n, 256), 256, 0, c->stream>>>(
      n, static_cast<double>(samples), f->s1, f->s2, f->sigma, f->flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int rows_per_block = 8;
  if (rank > 0) {
    omega_kernel<<<blocks_for(static_cast<long long>(kMaxPcRank) * ((n + 3) / 4), 256), 256, 0,
                   c->stream>>>(c->opts.seed, n, rank, f->Q);
    symm_block_kernel<<<blocks_for(n, rows_per_block), rows_per_block * 32, 0, c->stream>>>(
        n, f->sigma, f->Q, f->Y);
    for (int it = 0; it < power_iters; ++it) {
      orth_kernel<<<1, kFitThreads, 0, c->stream>>>(n, rank, f->Y, f->Q);
      symm_block_kernel<<<blocks_for(n, rows_per_block), rows_per_block * 32, 0, c->stream>>>(
          n, f->sigma, f->Q, f->Y);
    }
    orth_kernel<<<1, kFitThreads, 0, c->stream>>>(n, rank, f->Y, f->Q);
    symm_block_kernel<<<blocks_for(n, rows_per_block), rows_per_block * 32, 0, c->stream>>>(
        n, f->sigma, f->Q, f->Y);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  ritz_kernel<<<1, kFitThreads, 0, c->stream>>>(n, c->n_ld, rank, f->Q, f->Y, f->sigma,
                                                c->d.pc_delta64, c->d.pc_U64, c->d.pc_delta32,
                                                c->d.pc_U32, nullptr, f->flag);
  return cudaGetLastError();
}

}  // namespace mhar
