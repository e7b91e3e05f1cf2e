// mhar_api.cu -- host side of libmhar: the C ABI declared in include/mhar.h.
//
// The context owns every device buffer (cudaMalloc), a stream, and two CUDA
// graphs of the per-iteration kernels (a chunk of graph_chunk iterations and a
// single iteration) that are replayed by mhar_run.  Kernels read the
// iteration index from a device counter, so one captured graph serves every
// replay; the last node of each graph advances the counter.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "mhar_device.cuh"
#include "mhar_internal.h"

thread_local char g_null_err[512] = {0};

namespace mhar {
void set_null_error(const char* msg) {
  if (!msg) {
    g_null_err[0] = 0;
    return;
  }
  snprintf(g_null_err, sizeof(g_null_err), "%s", msg);
}
}  // namespace mhar

namespace {

void remember_create_error(const char* msg) { mhar::set_null_error(msg); }

void set_err(mhar_ctx* c, const char* fmt, ...) {
  if (!c) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
}

int cuda_fail(mhar_ctx* c, cudaError_t e, const char* what) {
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();  // a failed launch must not be reported again by a later check
  return MHAR_E_CUDA;
}

#define MHAR_CUDA(call, what)                    \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

unsigned long long host_key(double f) {
  unsigned long long u;
  std::memcpy(&u, &f, sizeof(u));
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
double host_unkey(unsigned long long k) {
  const unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  double f;
  std::memcpy(&f, &u, sizeof(f));
  return f;
}

template <typename T>
int dmalloc(mhar_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
  e = cudaMemsetAsync(*p, 0, count * sizeof(T), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
  return MHAR_OK;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

bool all_finite(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Tensor-core modes (FP16-pair operands).
bool mixed(const mhar_ctx* c) {
  return c->opts.precision == MHAR_MIXED_F16X3 || c->opts.precision == MHAR_MIXED_RECOMPUTE;
}
// Stored-slack mode (slack array, refresh).
bool stored(const mhar_ctx* c) { return c->opts.precision == MHAR_MIXED_F16X3; }
bool recompute(const mhar_ctx* c) { return c->opts.precision == MHAR_MIXED_RECOMPUTE; }

void free_all(mhar_ctx* c) {
  mhar::DeviceBuffers& d = c->d;
  void* ptrs[] = {d.A64, d.b64, d.A32, d.b32, d.kr32, d.AE64, d.Q64, d.Q32, d.Q32lo, d.bE64,
                  d.wE64, d.Lchol, d.Ah, d.Al, d.row_scale, d.bS, d.rows, d.rowk, d.nx_ref, d.theta_acc,
                  d.refresh_step, d.X64, d.Xhi, d.Xlo, d.D64, d.D32, d.Dh, d.Dl, d.S, d.corr, d.corrn, d.Xh, d.Xl, d.wscale, d.Dh2, d.Dl2,
                  d.key_lo, d.key_hi, d.lmin, d.lmax, d.theta, d.status, d.counters, d.step,
                  d.emit, d.check, d.pc_delta64, d.pc_U64, d.pc_delta32, d.pc_U32, d.sigma};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d = mhar::DeviceBuffers();
}

// Projector set-up on the device (Section 3.2).  With L the Cholesky factor
// of A_E A_E^T and Q = L^{-1} A_E (orthonormal rows spanning the row space of
// A_E), P = I - A_E^T (A_E A_E^T)^{-1} A_E = I - Q^T Q, and the re-projection
// onto A_E x = b_E is x - Q^T (Q x - w) with w = L^{-1} b_E.  The walkers then
// need no triangular solves.  Q is taken by CholeskyQR2 (Fukaya, Nakatsukasa,
// Yanagisawa and Yamamoto, "CholeskyQR2: a simple and communication-avoiding
// algorithm for computing a tall-skinny QR factorization", 2014): the Cholesky
// QR step twice, the second on the first's Q, which leaves the rows of Q
// orthonormal to FP64 rounding while cond(A_E) stays below about 1e7.  All of
// it in FP64 on the device, in global memory, for any mE < n.

constexpr int kSetupThreads = 256;

// G[r][q] = M_r . M_q for q <= r (lower triangle), one block per entry.
__global__ void gram_kernel(int mE, int n, int n_ld, const double* M, double* G) {
  const int r = blockIdx.x, q = blockIdx.y;
  if (q > r) return;
  __shared__ double part[kSetupThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    s += M[static_cast<size_t>(r) * n_ld + i] * M[static_cast<size_t>(q) * n_ld + i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
    G[static_cast<size_t>(r) * mE + q] = t;
  }
}

// In-place Cholesky factor of the lower triangle of G (one block, column by
// column: the pivot by a block reduction, the column below it in parallel).
// ok[0] = 0 when a pivot falls to rel times its diagonal entry or below: A_E
// is rank-deficient, or too ill-conditioned for the factor to mean anything.
__global__ void cholesky_kernel(int mE, double* G, double rel, int* ok) {
  __shared__ double part[kSetupThreads / 32];
  __shared__ double piv;
  for (int j = 0; j < mE; ++j) {
    double* Gj = G + static_cast<size_t>(j) * mE;
    double s = 0.0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) s += Gj[k] * Gj[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
      const double dsum = Gj[j] - t;
      piv = (dsum > rel * Gj[j]) ? sqrt(dsum) : 0.0;
      Gj[j] = piv;
    }
    __syncthreads();
    const double ljj = piv;
    if (!(ljj > 0.0)) {
      if (threadIdx.x == 0) ok[0] = 0;
      return;
    }
    for (int i = j + 1 + threadIdx.x; i < mE; i += blockDim.x) {
      double* Gi = G + static_cast<size_t>(i) * mE;
      double t = Gi[j];
      for (int k = 0; k < j; ++k) t -= Gi[k] * Gj[k];
      Gi[j] = t / ljj;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ok[0] = 1;
}

// M <- L^{-1} M in place (forward substitution), one thread per column of M
// (mE rows, ncol columns, leading dimension ld); L lower, mE x mE.
__global__ void trsm_kernel(int mE, int ncol, int ld, const double* L, double* M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncol) return;
  for (int r = 0; r < mE; ++r) {
    const double* Lr = L + static_cast<size_t>(r) * mE;
    double t = M[static_cast<size_t>(r) * ld + i];
    for (int k = 0; k < r; ++k) t -= Lr[k] * M[static_cast<size_t>(k) * ld + i];
    M[static_cast<size_t>(r) * ld + i] = t / Lr[r];
  }
}

// hi = fl32(v), lo = fl32(v - hi).
__global__ void to_f32_pair_kernel(size_t count, const double* src, float* hi, float* lo) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i < count) {
    const float h = static_cast<float>(src[i]);
    hi[i] = h;
    lo[i] = static_cast<float>(src[i] - static_cast<double>(h));
  }
}

__global__ void broadcast_points_kernel(int mode, int z, int n, int n_ld, const double* x0,
                                        double* X64, float* Xhi, float* Xlo) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(z) * n) return;
  const int k = static_cast<int>(idx / n), i = static_cast<int>(idx - static_cast<long long>(k) * n);
  const size_t dst = static_cast<size_t>(k) * n_ld + i;
  const double v = x0[i];
  if (mode == 0) {
    X64[dst] = v;
  } else {
    const float h = static_cast<float>(v);
    Xhi[dst] = h;
    Xlo[dst] = static_cast<float>(v - static_cast<double>(h));
  }
}

// Recompute mode with nothing between the draw and the chord: the chord
// kernel draws the next directions itself (preconditioned ones too in the
// tensor-memory-operand kernel).
bool tail_draws(const mhar_ctx* c) {
  return recompute(c) && c->mE == 0 && (c->pc_rank < 0 || c->use_ts);
}

// FP32 and tensor-core modes with equalities and no preconditioner: the
// projection kernel draws the directions itself (one launch for both).
bool projection_draws(const mhar_ctx* c) {
  return c->mE > 0 && c->pc_rank < 0 && c->opts.precision != MHAR_FP64;
}

// Launches of one iteration's chord step (enqueue_chord): the stream-K chord
// kernel is followed by its walker update kernel, the FP32 / FP64 chord by
// the update kernel unless one warp per walker does both.
int chord_launches(const mhar_ctx* c) {
  if (recompute(c)) return (!c->use_ts && c->use_sk) ? 2 : 1;
  return (mixed(c) || mhar::simt_warp_path(c)) ? 1 : 2;
}

int kernels_per_iteration(const mhar_ctx* c) {
  const int chord = chord_launches(c);
  if (tail_draws(c)) return chord;
  return (projection_draws(c) ? 0 : 1) + (c->mE > 0 ? 1 : 0) + (c->pc_rank >= 0 ? 1 : 0) + chord;
}

int emit_count(const mhar_ctx* c) {
  return c->opts.emit_walkers > 0 ? c->opts.emit_walkers : c->z;
}

// Direction draw of one iteration (Section 4.3); in recompute mode the same
// launch first applies the previous iteration's moves and re-splits X.
cudaError_t enqueue_directions(mhar_ctx* c, int j) {
  if (tail_draws(c)) return cudaSuccess;  // drawn by the previous chord kernel
  const bool fused = projection_draws(c);
  cudaError_t e = cudaSuccess;
  if (!fused)
    e = recompute(c) ? mhar::launch_prep_walkers(c, j, 4) : mhar::launch_directions(c, j);
  // Preconditioned draw d = delta .* h + U g; the tensor-core modes split it
  // into the FP16 pair here unless the projection still has to run.
  if (e == cudaSuccess && c->pc_rank >= 0)
    e = mhar::launch_precondition(c, j, (mixed(c) && c->mE == 0) ? 1 : 0);
  if (e == cudaSuccess && c->mE > 0) e = mhar::launch_projection(c, j, fused ? 1 : 0);
  return e;
}

// The kernels of one iteration after the direction draw (Sections 4.4-4.5).
cudaError_t enqueue_chord(mhar_ctx* c, int j) {
  if (stored(c)) return mhar::launch_chord_tc(c, j);
  if (recompute(c)) {
    if (c->use_ts) return mhar::launch_recompute_ts(c, j);
    return c->use_sk ? mhar::launch_recompute_sk(c, j) : mhar::launch_recompute_tc(c, j);
  }
  if (mhar::simt_warp_path(c)) return mhar::launch_chord_update_warp(c, j);
  cudaError_t e = mhar::launch_chord_simt(c);
  return e == cudaSuccess ? mhar::launch_update_simt(c, j) : e;
}

// Recompute mode: each chord kernel moves its walkers and leaves the FP16
// operands of the next iteration in place, so X is always current.  After the
// host changed the state (creation, set_state, a new preconditioner) one
// preparation launch rebuilds the operands: the split of X, and the
// directions when the chord kernel draws them.
int ensure_operands(mhar_ctx* c) {
  if (!recompute(c) || c->operands_fresh) return MHAR_OK;
  MHAR_CUDA(mhar::launch_prep_walkers(c, 0, tail_draws(c) ? 6 : 2), "operand preparation");
  ++c->launches;
  if (tail_draws(c) && c->pc_rank >= 0) {  // preconditioned first directions
    MHAR_CUDA(mhar::launch_precondition(c, 0, 1), "operand preparation");
    ++c->launches;
  }
  c->operands_fresh = true;
  return MHAR_OK;
}

int enqueue_iterations(mhar_ctx* c, int count) {
  for (int j = 0; j < count; ++j) {
    MHAR_CUDA(enqueue_directions(c, j), "direction kernels");
    MHAR_CUDA(enqueue_chord(c, j), "chord kernels");
  }
  MHAR_CUDA(mhar::launch_advance(c, count), "advance kernel");
  return MHAR_OK;
}

int capture(mhar_ctx* c, int count, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  MHAR_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "begin capture");
  int rc = enqueue_iterations(c, count);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != MHAR_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  return MHAR_OK;
}

int advance(mhar_ctx* c, int64_t count) {
  int frc = ensure_operands(c);
  if (frc) return frc;
  if (c->opts.graph_chunk <= 0) {
    while (count > 0) {
      const int now = count > (1 << 20) ? (1 << 20) : static_cast<int>(count);
      int rc = enqueue_iterations(c, now);
      if (rc != MHAR_OK) return rc;
      c->launches += static_cast<int64_t>(now) * kernels_per_iteration(c) + 1;
      count -= now;
    }
    return MHAR_OK;
  }
  if (!c->g_one) {
    int rc = capture(c, 1, &c->g_one);
    if (rc != MHAR_OK) return rc;
    rc = capture(c, c->opts.graph_chunk, &c->g_chunk);
    if (rc != MHAR_OK) return rc;
    c->graph_len = c->opts.graph_chunk;
    c->launches_one = kernels_per_iteration(c) + 1;
    c->launches_chunk = static_cast<int64_t>(c->graph_len) * kernels_per_iteration(c) + 1;
  }
  while (count >= c->graph_len) {
    MHAR_CUDA(cudaGraphLaunch(c->g_chunk, c->stream), "graph launch");
    c->launches += c->launches_chunk;
    count -= c->graph_len;
  }
  while (count-- > 0) {
    MHAR_CUDA(cudaGraphLaunch(c->g_one, c->stream), "graph launch");
    c->launches += c->launches_one;
  }
  return MHAR_OK;
}

// Stored-slack mode: S = b - A X from the current points.  `periodic`: the
// refresh of a run, whose tracked slack it also checks against the tracked
// error bound (MHAR_ST_DRIFT when exceeded); otherwise the slack is new
// (creation, a new state or preconditioner) and there is nothing to check.
int refresh(mhar_ctx* c, bool periodic = false) {
  if (c->mE > 0) {
    MHAR_CUDA(mhar::launch_reproject(c), "re-projection kernel");
    ++c->launches;
  }
  if (c->opts.refresh_fp64) {
    MHAR_CUDA(mhar::launch_refresh_simt(c), "slack refresh kernel");
    ++c->launches;
  } else {
    MHAR_CUDA(mhar::launch_refresh_tc(c, periodic), "tensor-core slack refresh");
    c->launches += 2;
  }
  MHAR_CUDA(mhar::launch_stored_reset(c), "slack error reset");
  ++c->launches;
  c->since_refresh = 0;
  return MHAR_OK;
}

int emit_to(mhar_ctx* c, double* out, bool out_device, int walkers) {
  ++c->launches;
  if (out_device) {
    MHAR_CUDA(mhar::launch_emit(c, out, walkers), "emit kernel");
  } else {
    MHAR_CUDA(mhar::launch_emit(c, c->d.emit, walkers), "emit kernel");
    MHAR_CUDA(cudaMemcpyAsync(out, c->d.emit, sizeof(double) * walkers * c->n,
                              cudaMemcpyDeviceToHost, c->stream),
              "sample copy");
  }
  return MHAR_OK;
}

void drop_graphs(mhar_ctx* c) {
  if (c->g_chunk) cudaGraphExecDestroy(c->g_chunk);
  if (c->g_one) cudaGraphExecDestroy(c->g_one);
  c->g_chunk = nullptr;
  c->g_one = nullptr;
  c->graph_len = 0;
}

// Makes (delta, U, sigma) current: padded copies are on the device already;
// re-splits A with the new coordinate scales and, in the stored-slack mode,
// recomputes the slack from the points.
int adopt_preconditioner(mhar_ctx* c, int rank) {
  c->pc_rank = rank;
  c->operands_fresh = false;
  drop_graphs(c);
  if (mixed(c)) {
    MHAR_CUDA(mhar::launch_prepare_tc_operands(c), "operand preparation kernel");
    ++c->launches;
    if (stored(c)) {
      int rc = refresh(c);
      if (rc) return rc;
    }
  }
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "preconditioner sync");
  return MHAR_OK;
}

int alloc_preconditioner(mhar_ctx* c) {
  mhar::DeviceBuffers& d = c->d;
  const size_t nl = static_cast<size_t>(c->n_ld);
  int rc;
  if (!d.pc_delta64 &&
      ((rc = dmalloc(c, &d.pc_delta64, nl)) || (rc = dmalloc(c, &d.pc_U64, nl * mhar::kMaxPcRank)) ||
       (rc = dmalloc(c, &d.pc_delta32, nl)) || (rc = dmalloc(c, &d.pc_U32, nl * mhar::kMaxPcRank))))
    return rc;
  if (mixed(c) && !d.D32 && (rc = dmalloc(c, &d.D32, static_cast<size_t>(c->z) * c->n_ld)))
    return rc;
  return MHAR_OK;
}

int set_sigma(mhar_ctx* c, const std::vector<float>& sig) {
  for (float v : sig) {
    // The FP32 / tensor-core projection takes 1 / sigma as the negated
    // exponent (mhar_device.cuh, pow2_recip).
    int e = 0;
    if (!(std::frexp(v, &e) == 0.5f && e >= -125 && e <= 127)) {
      set_err(c, "a coordinate scale outside the powers of two 2^-126 .. 2^126");
      return MHAR_E_UNSUPPORTED;
    }
  }
  c->sigma_host = sig;
  if (!c->d.sigma) return MHAR_OK;
  c->unit_sigma = true;
  for (float v : sig) c->unit_sigma = c->unit_sigma && v == 1.0f;
  MHAR_CUDA(cudaMemcpyAsync(c->d.sigma, sig.data(), sizeof(float) * sig.size(),
                            cudaMemcpyHostToDevice, c->stream), "copy sigma");
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "sigma sync");
  return MHAR_OK;
}

// Column scales of A: sigma_j = 2^-e_j with max_i |a_ij| = f 2^e_j, f in
// [0.5, 1), then divided by the largest of them (so max sigma = 1) and kept
// >= 2^-13, so that a unit normal divided by sigma stays inside the FP16
// range (|h| <= 6.8 for the 32-bit uniforms of the draw).  All-zero columns
// get 1.  n_ld entries, 1 beyond n.
std::vector<float> column_scales(const double* A, int m, int n, int n_ld) {
  std::vector<double> colmax(n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j)
      colmax[j] = std::max(colmax[j], std::fabs(A[static_cast<size_t>(i) * n + j]));
  std::vector<float> sig(n_ld, 1.0f);
  double smax = 0.0;
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    if (colmax[j] > 0.0) {
      int e = 0;
      std::frexp(colmax[j], &e);
      v = std::ldexp(1.0, -e);
    }
    sig[j] = static_cast<float>(v);
    smax = std::max(smax, v);
  }
  for (int j = 0; j < n; ++j)
    sig[j] = std::max(static_cast<float>(sig[j] / smax), 0x1p-13f);
  return sig;
}

// Typical 2-norm and max-norm of a scaled direction d / sigma when d_i has
// variance var_i (1 for isotropic directions): sqrt(sum var_i / sigma_i^2)
// and 3 max sqrt(var_i) / sigma_i.  They only choose the bound form of each
// 32-row block (row_blocks_kernel); the bounds themselves use the actual
// norms of every walker's direction.
void direction_norms(mhar_ctx* c, const std::vector<double>& var) {
  const std::vector<float>& sig = c->sigma_host;
  double s2 = 0.0, mx = 0.0;
  for (int i = 0; i < c->n; ++i) {
    const double v = var.empty() ? 1.0 : var[i];
    const double r = std::sqrt(v) / static_cast<double>(sig[i]);
    s2 += r * r;
    mx = std::max(mx, r);
  }
  c->dir_norm2 = std::max(std::sqrt(s2), 1e-30);
  c->dir_norminf = std::max(3.0 * mx, 1e-30);
}

// Coordinate scales with a preconditioner (delta: n_ld values, U: n_ld x 32,
// zero beyond its rank).  Tensor-core modes: A's column scales times one
// power of two c that brings the largest typical |d_i| / sigma_i near 1; then
// each sigma_i at most 2^8 sd_i (so d_i / sigma_i is well above the FP16
// subnormals) and at least 6.8 l1_i / 65504 rounded up (|d_i| <= 6.8 (delta_i
// + sum_q |U_iq|) for the 32-bit uniforms of the draw, so the scaled
// direction stays inside the FP16 range); sd_i^2 = delta_i^2 + (U U^T)_ii,
// l1_i = delta_i + sum_q |U_iq|.  The CUDA-core modes keep A's column scales
// (their margins only need some sigma).
int precond_scales(mhar_ctx* c, const double* delta, const double* U) {
  const int n = c->n, R = mhar::kMaxPcRank;
  std::vector<double> sd(n, 0.0), l1(n, 0.0), var(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double v = delta[i] * delta[i], a1 = delta[i];
    for (int q = 0; q < R; ++q) {
      const double u = U[static_cast<size_t>(i) * R + q];
      v += u * u;
      a1 += std::fabs(u);
    }
    var[i] = v;
    sd[i] = std::sqrt(v);
    l1[i] = a1;
  }
  std::vector<float> sig = c->sigma_A;
  if (mixed(c)) {
    double rmax = 0.0;
    for (int i = 0; i < n; ++i) rmax = std::max(rmax, sd[i] / c->sigma_A[i]);
    int ec = 0;
    if (rmax > 0.0 && std::isfinite(rmax)) std::frexp(rmax, &ec);
    for (int i = 0; i < n; ++i) {
      double v = std::ldexp(static_cast<double>(c->sigma_A[i]), ec);
      if (sd[i] > 0.0) {
        int e = 0;
        std::frexp(sd[i] * 256.0, &e);
        v = std::min(v, std::ldexp(1.0, e - 1));
      }
      const double lo = 6.8 * l1[i] / 65504.0;
      if (lo > 0.0) {
        int e = 0;
        std::frexp(lo, &e);
        v = std::max(v, std::ldexp(1.0, e));
      }
      sig[i] = static_cast<float>(v);
    }
  }
  int rc = set_sigma(c, sig);
  if (rc) return rc;
  direction_norms(c, var);
  return MHAR_OK;
}

// FP32 mode: b lowered by 3 u |b_i| and the row bounds of chord_simt_kernel
// (kernels_simt.cu), K_i,2 = gamma ||a_i sigma||_2 and K_i,1 = gamma
// ||a_i sigma||_1 with gamma = gamma_{nnz_i + 4} (products of exact zeros add
// nothing), and ||a_i sigma||_2 itself.  kr[3 i .. 3 i + 2].
void simt_bounds(const double* A, const double* b, int m, int n, const std::vector<float>& sig,
                 std::vector<float>* bm, std::vector<float>* kr) {
  const double u = 0x1p-24;
  bm->resize(m);
  kr->resize(3 * static_cast<size_t>(m));
  auto up = [](double v) {
    float f = static_cast<float>(v);
    if (static_cast<double>(f) < v) f = std::nextafter(f, INFINITY);
    return f;
  };
  for (int i = 0; i < m; ++i) {
    double s2 = 0.0, s1 = 0.0;
    int nnz = 0;
    for (int j = 0; j < n; ++j) {
      const double v = A[static_cast<size_t>(i) * n + j] * static_cast<double>(sig[j]);
      s2 += v * v;
      s1 += std::fabs(v);
      nnz += v != 0.0;
    }
    const double k = static_cast<double>(nnz + 4);
    const double gamma = k * u / (1.0 - k * u) * (1.0 + 1e-6);
    (*kr)[3 * i] = up(gamma * std::sqrt(s2));
    (*kr)[3 * i + 1] = up(gamma * s1);
    (*kr)[3 * i + 2] = up(std::sqrt(s2) * (1.0 + 1e-6));
    const double lb = b[i] - 3.0 * u * std::fabs(b[i]);
    float bt = static_cast<float>(lb);
    if (static_cast<double>(bt) > lb) bt = std::nextafter(bt, -INFINITY);
    (*bm)[i] = bt;
  }
}

int reset_drift(mhar_ctx* c) {
  const unsigned long long k0 = host_key(0.0);
  MHAR_CUDA(cudaMemcpyAsync(reinterpret_cast<unsigned long long*>(c->d.check) + 2, &k0, sizeof(k0),
                            cudaMemcpyHostToDevice, c->stream),
            "drift reset");
  return MHAR_OK;
}

// FP64 audit of the running walkers (opts.audit_every): folds into the
// running maxima at check keys 3 and 4.
int audit(mhar_ctx* c) {
  const int w = c->opts.audit_walkers > 0 ? c->opts.audit_walkers : c->z;
  MHAR_CUDA(mhar::launch_check(c, w, reinterpret_cast<unsigned long long*>(c->d.check) + 3),
            "audit kernel");
  ++c->launches;
  ++c->audits;
  c->since_audit = 0;
  return MHAR_OK;
}

}  // namespace

namespace {

// ---- the preconditioner fit, in parts (mhar_fit_preconditioner, and the
// moments / factor halves used to pool a fit over several shards) ------------
bool fit_args_ok(mhar_ctx* c, int64_t warmup, int32_t snapshots) {
  if (warmup < 1 || snapshots < 1 || snapshots > warmup ||
      static_cast<int64_t>(c->z) * snapshots < 2) {
    set_err(c, "bad fit arguments (warmup=%lld snapshots=%d, z=%d)",
            static_cast<long long>(warmup), snapshots, c->z);
    return false;
  }
  return true;
}

bool factor_args_ok(mhar_ctx* c, int32_t rank, int32_t power_iters) {
  if (rank < 0 || rank > std::min(mhar::kMaxPcRank, c->n) || power_iters < 0 || power_iters > 64) {
    set_err(c, "bad fit arguments (rank=%d power_iters=%d, n=%d)", rank, power_iters, c->n);
    return false;
  }
  return true;
}

void fit_release(mhar_ctx* c, mhar::FitScratch* f) {
  cudaStreamSynchronize(c->stream);
  void* ptrs[] = {f->shift, f->s1, f->s2, f->sigma, f->Y, f->Q, f->flag};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  *f = mhar::FitScratch();
}

int fit_alloc(mhar_ctx* c, mhar::FitScratch* f) {
  const size_t n = static_cast<size_t>(c->n), nn = n * n;
  int rc;
  if ((rc = dmalloc(c, &f->shift, n)) || (rc = dmalloc(c, &f->s1, n)) || (rc = dmalloc(c, &f->s2, nn)) ||
      (rc = dmalloc(c, &f->sigma, nn)) || (rc = dmalloc(c, &f->Y, n * mhar::kMaxPcRank)) ||
      (rc = dmalloc(c, &f->Q, n * mhar::kMaxPcRank)) || (rc = dmalloc(c, &f->flag, 1)) ||
      (rc = alloc_preconditioner(c))) {
    fit_release(c, f);
    return rc;
  }
  return MHAR_OK;
}

// Warm-up and moments on the device: `snapshots` snapshots spread over the
// last half of `warmup` iterations; the moments are taken about `shift`
// (host, n) or, when it is NULL, about walker 0's point at the first snapshot.
int fit_moments_device(mhar_ctx* c, int64_t warmup, int32_t snapshots, const double* shift,
                       mhar::FitScratch* f) {
  const int64_t gap = std::max<int64_t>(1, warmup / (2 * static_cast<int64_t>(snapshots)));
  const int64_t first = warmup - (snapshots - 1) * gap;
  if (shift)
    MHAR_CUDA(cudaMemcpyAsync(f->shift, shift, sizeof(double) * c->n, cudaMemcpyHostToDevice,
                              c->stream), "copy shift");
  int rc = MHAR_OK;
  for (int s = 0; s < snapshots && rc == MHAR_OK; ++s) {
    rc = mhar_run(c, s == 0 ? first : gap, 0, nullptr);
    if (rc != MHAR_OK) break;
    cudaError_t e = cudaSuccess;
    if (s == 0 && !shift) e = mhar::launch_fit_shift(c, f);
    if (e == cudaSuccess) e = mhar::launch_fit_accumulate(c, f);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "covariance kernel");
    c->launches += (s == 0 && !shift) ? 2 : 1;
  }
  return rc;
}

// Sigma from the moments of `samples` points, then (delta, U) into the
// context's preconditioner buffers.
int fit_factor_device(mhar_ctx* c, mhar::FitScratch* f, long long samples, int rank,
                      int power_iters) {
  cudaError_t e = mhar::launch_fit_factor(c, f, samples, rank, power_iters);
  if (e != cudaSuccess) return cuda_fail(c, e, "preconditioner fit kernels");
  c->launches += rank > 0 ? 5 + 2 * power_iters : 2;
  int flag = 0;
  e = cudaMemcpyAsync(&flag, f->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fit sync");
  if (flag) {
    set_err(c, "the warm-up covariance is not finite");
    return MHAR_E_NONFINITE;
  }
  return MHAR_OK;
}

// The coordinate scales follow the fitted (delta, U) by the rule of
// mhar_set_preconditioner; then the walk adopts it.
int fit_adopt(mhar_ctx* c, int rank) {
  std::vector<double> d64(c->n_ld), u64(static_cast<size_t>(c->n_ld) * mhar::kMaxPcRank);
  MHAR_CUDA(cudaMemcpy(d64.data(), c->d.pc_delta64, sizeof(double) * d64.size(),
                       cudaMemcpyDeviceToHost), "copy delta");
  MHAR_CUDA(cudaMemcpy(u64.data(), c->d.pc_U64, sizeof(double) * u64.size(),
                       cudaMemcpyDeviceToHost), "copy U");
  int rc = precond_scales(c, d64.data(), u64.data());
  if (rc) return rc;
  return adopt_preconditioner(c, rank);
}

}  // namespace

extern "C" {

int mhar_status_code(int32_t status_bits, int32_t wait_expired) {
  if (wait_expired) return MHAR_E_TIMEOUT;
  if (status_bits & MHAR_ST_NONFINITE) return MHAR_E_NONFINITE;
  if (status_bits & MHAR_ST_DRIFT) return MHAR_E_INFEASIBLE_DRIFT;
  if (status_bits & MHAR_ST_UNBOUNDED) return MHAR_E_UNBOUNDED;
  return MHAR_OK;
}

void mhar_default_opts(mhar_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->seed = 0;
  o->precision = MHAR_FP64;
  o->refresh_k = 64;
  o->out_on_device = 0;
  o->walker0 = 0;
  o->stream = nullptr;
  o->graph_chunk = 16;
}

const char* mhar_strerror(int code) {
  switch (code) {
    case MHAR_OK: return "MHAR_OK";
    case MHAR_E_ARG: return "MHAR_E_ARG";
    case MHAR_E_X0_INFEASIBLE: return "MHAR_E_X0_INFEASIBLE";
    case MHAR_E_UNBOUNDED: return "MHAR_E_UNBOUNDED";
    case MHAR_E_NONFINITE: return "MHAR_E_NONFINITE";
    case MHAR_E_CUDA: return "MHAR_E_CUDA";
    case MHAR_E_RANK: return "MHAR_E_RANK";
    case MHAR_E_UNSUPPORTED: return "MHAR_E_UNSUPPORTED";
    case MHAR_E_TIMEOUT: return "MHAR_E_TIMEOUT";
    case MHAR_E_INFEASIBLE_DRIFT: return "MHAR_E_INFEASIBLE_DRIFT";
    default: return "MHAR_E_UNKNOWN";
  }
}

const char* mhar_kernel_name(const mhar_ctx* c) {
  if (!c) return "none";
  if (recompute(c)) return c->use_ts ? "recompute_ts_kernel" : (c->use_sk ? "recompute_sk_kernel" : "recompute_tc_kernel");
  if (stored(c)) return "walker_tc_kernel";
  return mhar::simt_warp_path(c) ? "chord_warp_kernel" : "chord_simt_kernel";
}

const char* mhar_last_error(const mhar_ctx* c) {
  if (!c) return g_null_err[0] ? g_null_err : "no error";
  return c->err[0] ? c->err : "no error";
}

void mhar_destroy(mhar_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->g_chunk) cudaGraphExecDestroy(c->g_chunk);
  if (c->g_one) cudaGraphExecDestroy(c->g_one);
  if (c->sk) mhar::sk_destroy(c);
  if (c->tc) mhar::tc_plan_destroy(c);
  free_all(c);
  if (c->stream && c->stream != static_cast<cudaStream_t>(c->opts.stream))
    cudaStreamDestroy(c->stream);
  delete c;
}

static int create_impl(mhar_ctx* c, const double* A, const double* b, const double* AE,
                       const double* bE, const double* x0) {
  const int m = c->m, n = c->n, mE = c->mE, z = c->z;
  // Device must be sm_103 (the only architecture this library is built for).
  MHAR_CUDA(cudaGetDevice(&c->device), "cudaGetDevice");
  cudaDeviceProp prop;
  MHAR_CUDA(cudaGetDeviceProperties(&prop, c->device), "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3)) {
    set_err(c, "device %d is sm_%d%d; libmhar is built for sm_103a only", c->device, prop.major,
            prop.minor);
    return MHAR_E_CUDA;
  }
  if (c->opts.stream) {
    c->stream = static_cast<cudaStream_t>(c->opts.stream);
  } else {
    MHAR_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream create");
  }

  // Strict interiority of x0 and the equality residual, in FP64 on the host
  // (a one-off input check, not part of the sampling path).
  double worst = INFINITY;
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int k = 0; k < n; ++k) s -= A[static_cast<size_t>(i) * n + k] * x0[k];
    worst = s < worst ? s : worst;
  }
  if (!(worst > 0.0)) {
    set_err(c, "x0 is not strictly inside A x <= b (min slack %.3e)", worst);
    return MHAR_E_X0_INFEASIBLE;
  }
  if (mE > 0) {
    double bmax = 0.0, res = 0.0;
    for (int e = 0; e < mE; ++e) {
      double s = -bE[e];
      for (int k = 0; k < n; ++k) s += AE[static_cast<size_t>(e) * n + k] * x0[k];
      res = std::fmax(res, std::fabs(s));
      bmax = std::fmax(bmax, std::fabs(bE[e]));
    }
    if (res > 1e-9 * (1.0 + bmax)) {
      set_err(c, "x0 violates A_E x = b_E (residual %.3e)", res);
      return MHAR_E_X0_INFEASIBLE;
    }
  }

  c->n_ld = round_up(n, 32);
  c->k_pad = round_up(n, mhar::kTcKChunk);
  c->kdim = round_up(n, mhar::kTcK);
  c->m_pad = round_up(m, mhar::kTcM);
  const int z_ld = round_up(z, 128);
  const int mode = c->opts.precision == MHAR_FP64 ? 0 : 1;
  mhar::DeviceBuffers& d = c->d;
  int rc;

  // Problem data, padded to the leading dimensions.
  std::vector<double> Ap(static_cast<size_t>(m) * c->n_ld, 0.0);
  for (int i = 0; i < m; ++i)
    std::memcpy(&Ap[static_cast<size_t>(i) * c->n_ld], A + static_cast<size_t>(i) * n,
                sizeof(double) * n);
  if ((rc = dmalloc(c, &d.A64, Ap.size())) || (rc = dmalloc(c, &d.b64, m))) return rc;
  MHAR_CUDA(cudaMemcpyAsync(d.A64, Ap.data(), sizeof(double) * Ap.size(), cudaMemcpyHostToDevice,
                            c->stream), "copy A");
  MHAR_CUDA(cudaMemcpyAsync(d.b64, b, sizeof(double) * m, cudaMemcpyHostToDevice, c->stream),
            "copy b");
  // Column scales of A (every mode) and the CUDA-core modes' rounding bounds.
  c->sigma_A = column_scales(A, m, n, c->n_ld);
  if ((rc = dmalloc(c, &d.sigma, c->n_ld)) || (rc = set_sigma(c, c->sigma_A))) return rc;
  direction_norms(c, {});
  if (c->opts.precision == MHAR_FP32) {
    std::vector<float> Af(Ap.begin(), Ap.end());
    std::vector<float> bf, kr;
    simt_bounds(A, b, m, n, c->sigma_A, &bf, &kr);
    if ((rc = dmalloc(c, &d.A32, Af.size())) || (rc = dmalloc(c, &d.b32, m)) ||
        (rc = dmalloc(c, &d.kr32, kr.size())))
      return rc;
    MHAR_CUDA(cudaMemcpyAsync(d.A32, Af.data(), sizeof(float) * Af.size(), cudaMemcpyHostToDevice,
                              c->stream), "copy A32");
    MHAR_CUDA(cudaMemcpyAsync(d.b32, bf.data(), sizeof(float) * m, cudaMemcpyHostToDevice,
                              c->stream), "copy b32");
    MHAR_CUDA(cudaMemcpyAsync(d.kr32, kr.data(), sizeof(float) * kr.size(),
                              cudaMemcpyHostToDevice, c->stream), "copy bounds");
    MHAR_CUDA(cudaStreamSynchronize(c->stream), "sync");
  }

  if (mE > 0) {
    std::vector<double> AEp(static_cast<size_t>(mE) * c->n_ld, 0.0);
    for (int e = 0; e < mE; ++e)
      std::memcpy(&AEp[static_cast<size_t>(e) * c->n_ld], AE + static_cast<size_t>(e) * n,
                  sizeof(double) * n);
    if ((rc = dmalloc(c, &d.AE64, AEp.size())) || (rc = dmalloc(c, &d.Q64, AEp.size())) ||
        (rc = dmalloc(c, &d.Q32, AEp.size())) || (rc = dmalloc(c, &d.Q32lo, AEp.size())) ||
        (rc = dmalloc(c, &d.bE64, mE)) ||
        (rc = dmalloc(c, &d.wE64, mE)) || (rc = dmalloc(c, &d.Lchol, static_cast<size_t>(mE) * mE)))
      return rc;
    MHAR_CUDA(cudaMemcpyAsync(d.AE64, AEp.data(), sizeof(double) * AEp.size(),
                              cudaMemcpyHostToDevice, c->stream), "copy AE");
    MHAR_CUDA(cudaMemcpyAsync(d.bE64, bE, sizeof(double) * mE, cudaMemcpyHostToDevice, c->stream),
              "copy bE");
    MHAR_CUDA(cudaStreamSynchronize(c->stream), "sync");
  }

  // Walker state and bookkeeping.
  if ((rc = dmalloc(c, &d.key_lo, z)) || (rc = dmalloc(c, &d.key_hi, z)) ||
      (rc = dmalloc(c, &d.lmin, z)) || (rc = dmalloc(c, &d.lmax, z)) ||
      (rc = dmalloc(c, &d.theta, z)) || (rc = dmalloc(c, &d.status, 2)) ||
      (rc = dmalloc(c, &d.counters, 2)) || (rc = dmalloc(c, &d.step, 1)) ||
      (rc = dmalloc(c, &d.emit, static_cast<size_t>(z) * n)) || (rc = dmalloc(c, &d.check, 6)))
    return rc;
  {
    // Audit keys: running max violation from -inf, running residual from 0.
    const unsigned long long init[2] = {host_key(-INFINITY), host_key(0.0)};
    MHAR_CUDA(cudaMemcpyAsync(reinterpret_cast<unsigned long long*>(d.check) + 3, init, sizeof(init),
                              cudaMemcpyHostToDevice, c->stream), "audit init");
  }
  const size_t zn = static_cast<size_t>(z) * c->n_ld;
  if (mode == 0) {
    if ((rc = dmalloc(c, &d.X64, zn)) || (rc = dmalloc(c, &d.D64, zn))) return rc;
  } else {
    if ((rc = dmalloc(c, &d.Xhi, zn)) || (rc = dmalloc(c, &d.Xlo, zn))) return rc;
    if (c->opts.precision == MHAR_FP32 || mE > 0)
      if ((rc = dmalloc(c, &d.D32, zn))) return rc;
    if (mE > 0 && ((rc = dmalloc(c, &d.corr, static_cast<size_t>(z) * mE)) ||
                   (rc = dmalloc(c, &d.corrn, z))))
      return rc;
  }
  if (mixed(c)) {
    const size_t opnd = static_cast<size_t>(c->m_pad) * c->k_pad;
    const size_t dsz = static_cast<size_t>(z_ld) * c->k_pad;
    if ((rc = dmalloc(c, &d.Ah, opnd)) || (rc = dmalloc(c, &d.Al, opnd)) ||
        (rc = dmalloc(c, &d.row_scale, c->m_pad)) || (rc = dmalloc(c, &d.bS, c->m_pad)) ||
        (rc = dmalloc(c, &d.rows, static_cast<size_t>(4) * c->m_pad)) ||
        (rc = dmalloc(c, &d.rowk, static_cast<size_t>(4) * c->m_pad)) ||
        (rc = dmalloc(c, &d.Dh, dsz)) || (rc = dmalloc(c, &d.Dl, dsz)) ||
        (rc = dmalloc(c, &d.Xh, dsz)) || (rc = dmalloc(c, &d.Xl, dsz)) ||
        (rc = dmalloc(c, &d.wscale, z_ld)))
      return rc;
    if (stored(c) && ((rc = dmalloc(c, &d.S, static_cast<size_t>(c->m_pad) * z_ld)) ||
                      (rc = dmalloc(c, &d.nx_ref, z)) || (rc = dmalloc(c, &d.theta_acc, z)) ||
                      (rc = dmalloc(c, &d.refresh_step, 1))))
      return rc;
    if (recompute(c) && ((rc = dmalloc(c, &d.Dh2, dsz)) || (rc = dmalloc(c, &d.Dl2, dsz))))
      return rc;
  }

  // Projector on the device: Q and w by CholeskyQR2.
  if (mE > 0) {
    int* ok = d.status + 1;
    const size_t qn = static_cast<size_t>(mE) * c->n_ld;
    MHAR_CUDA(cudaMemcpyAsync(d.Q64, d.AE64, sizeof(double) * qn, cudaMemcpyDeviceToDevice,
                              c->stream), "copy Q");
    MHAR_CUDA(cudaMemcpyAsync(d.wE64, d.bE64, sizeof(double) * mE, cudaMemcpyDeviceToDevice,
                              c->stream), "copy w");
    for (int pass = 0; pass < 2; ++pass) {
      gram_kernel<<<dim3(mE, mE), kSetupThreads, 0, c->stream>>>(mE, n, c->n_ld, d.Q64, d.Lchol);
      MHAR_CUDA(cudaGetLastError(), "projector Gram kernel");
      // A pivot below 1e-14 of its diagonal entry: cond(A_E) beyond about 1e7.
      cholesky_kernel<<<1, kSetupThreads, 0, c->stream>>>(mE, d.Lchol, 1e-14, ok);
      MHAR_CUDA(cudaGetLastError(), "projector Cholesky kernel");
      int okh = 0;
      MHAR_CUDA(cudaMemcpyAsync(&okh, ok, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy");
      MHAR_CUDA(cudaStreamSynchronize(c->stream), "sync");
      MHAR_CUDA(cudaMemsetAsync(ok, 0, sizeof(int), c->stream), "memset");
      if (!okh) {
        set_err(c, "A_E A_E^T is not positive definite (rank-deficient or ill-conditioned "
                   "equalities, cond(A_E) > ~1e7)");
        return MHAR_E_RANK;
      }
      trsm_kernel<<<(c->n_ld + 127) / 128, 128, 0, c->stream>>>(mE, c->n_ld, c->n_ld, d.Lchol,
                                                                 d.Q64);
      trsm_kernel<<<1, 32, 0, c->stream>>>(mE, 1, 1, d.Lchol, d.wE64);
      MHAR_CUDA(cudaGetLastError(), "projector solve kernel");
    }
    to_f32_pair_kernel<<<static_cast<unsigned>((qn + 255) / 256), 256, 0, c->stream>>>(
        qn, d.Q64, d.Q32, d.Q32lo);
    MHAR_CUDA(cudaGetLastError(), "projector conversion kernel");
    MHAR_CUDA(mhar::projection_smem_attr(mE, n), "projection kernel attributes");
  }

  // Algorithm 2: every column of X starts at x0.
  double* x0d = nullptr;
  if ((rc = dmalloc(c, &x0d, n))) return rc;
  MHAR_CUDA(cudaMemcpyAsync(x0d, x0, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream),
            "copy x0");
  broadcast_points_kernel<<<(static_cast<long long>(z) * n + 255) / 256, 256, 0, c->stream>>>(
      mode, z, n, c->n_ld, x0d, d.X64, d.Xhi, d.Xlo);
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(c->stream);
  cudaFree(x0d);
  if (e != cudaSuccess) return cuda_fail(c, e, "broadcast kernel");
  MHAR_CUDA(mhar::launch_set_points(c, nullptr), "init keys");

  if (mixed(c)) {
    MHAR_CUDA(mhar::launch_prepare_tc_operands(c), "operand preparation kernel");
    if ((rc = mhar::tc_plan_create(c))) return rc;
    if (recompute(c)) {
      c->operands_fresh = false;
      c->use_ts = mhar::ts_eligible(c) && c->opts.smem_operands == 0;
      c->use_sk = !c->use_ts &&
                  (c->opts.schedule == 2 ||
                   (c->opts.schedule == 0 && mhar::rc_prefers_stream_k(c) &&
                    (c->k_pad / mhar::kTcKChunk > 2 || c->m_pad > 32768)));
      if (c->use_ts)
        rc = mhar::ts_prepare(c);
      else
        rc = c->use_sk ? mhar::sk_prepare(c) : mhar::rc_prepare(c);
      if (rc) return rc;
    }
    if (stored(c) && ((rc = reset_drift(c)) || (rc = refresh(c)))) return rc;
  }
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "create sync");
  return MHAR_OK;
}

int mhar_create(const double* A, const double* b, int m, int n, const double* AE, const double* bE,
                int mE, const double* x0, int z, const mhar_opts* opts, mhar_ctx** out) {
  if (!out) return MHAR_E_ARG;
  *out = nullptr;
  mhar_ctx* c = new (std::nothrow) mhar_ctx();
  if (!c) return MHAR_E_ARG;
  if (opts) c->opts = *opts; else mhar_default_opts(&c->opts);
  if (z <= 0) z = (m > n ? m : n) + 1;  // Algorithm 2's default padding
  c->m = m; c->n = n; c->mE = mE; c->z = z;
  int rc = MHAR_OK;
  if (!A || !b || !x0 || m < 1 || n < 1 || mE < 0 || (mE > 0 && (!AE || !bE))) {
    set_err(c, "bad pointer or size (m=%d n=%d mE=%d)", m, n, mE);
    rc = MHAR_E_ARG;
  } else if (mE >= n || mE > 25600) {
    set_err(c, "the library handles 0 <= mE < n and mE <= 25600 (got mE=%d, n=%d)", mE, n);
    rc = MHAR_E_UNSUPPORTED;
  } else if (c->opts.precision < MHAR_FP64 || c->opts.precision > MHAR_MIXED_RECOMPUTE ||
             c->opts.refresh_k < 0 || c->opts.graph_chunk < 0 || c->opts.emit_walkers < 0 ||
             c->opts.emit_walkers > z || c->opts.schedule < 0 || c->opts.schedule > 2 ||
             c->opts.audit_every < 0 || c->opts.audit_walkers < 0 ||
             c->opts.audit_walkers > z || c->opts.reserved != 0) {
    set_err(c, "bad option (precision=%d refresh_k=%d graph_chunk=%d emit_walkers=%d)",
            c->opts.precision, c->opts.refresh_k, c->opts.graph_chunk, c->opts.emit_walkers);
    rc = MHAR_E_ARG;
  } else if (!all_finite(A, static_cast<size_t>(m) * n) || !all_finite(b, m) ||
             !all_finite(x0, n) || (mE > 0 && (!all_finite(AE, static_cast<size_t>(mE) * n) ||
                                               !all_finite(bE, mE)))) {
    set_err(c, "non-finite input");
    rc = MHAR_E_NONFINITE;
  } else {
    rc = create_impl(c, A, b, AE, bE, x0);
  }
  if (rc != MHAR_OK) {
    // The message survives the context for mhar_last_error(NULL).
    remember_create_error(c->err);
    mhar_destroy(c);
    return rc;
  }
  *out = c;
  return MHAR_OK;
}

int mhar_run(mhar_ctx* c, int64_t steps, int64_t thin, double* out) {
  if (!c) return MHAR_E_ARG;
  if (steps < 0 || thin < 0) {
    set_err(c, "steps and thin must be >= 0");
    return MHAR_E_ARG;
  }
  const int64_t nsamp = thin > 0 ? steps / thin : 0;
  if (nsamp > 0 && !out) {
    set_err(c, "out is NULL but %lld samples are due", static_cast<long long>(nsamp));
    return MHAR_E_ARG;
  }
  if (steps == 0) return MHAR_OK;
  MHAR_CUDA(cudaMemsetAsync(c->d.status, 0, 2 * sizeof(int), c->stream), "status reset");
  int rc;
  if (stored(c) && (rc = reset_drift(c))) return rc;
  int64_t done = 0, emitted = 0;
  const int64_t k = stored(c) ? c->opts.refresh_k : 0;
  const int64_t au = c->opts.audit_every;
  while (done < steps) {
    int64_t adv = steps - done;
    if (thin > 0) adv = std::min<int64_t>(adv, thin - (done % thin));
    if (k > 0) adv = std::min<int64_t>(adv, k - c->since_refresh);
    if (au > 0) adv = std::min<int64_t>(adv, au - c->since_audit);
    if ((rc = advance(c, adv))) return rc;
    done += adv;
    c->step += static_cast<uint64_t>(adv);
    if (au > 0) {
      c->since_audit += adv;
      if (c->since_audit >= au && (rc = audit(c))) return rc;
    }
    if (k > 0) {
      c->since_refresh += adv;
      if (c->since_refresh >= k && (rc = refresh(c, true))) return rc;
    }
    if (thin > 0 && done % thin == 0 && emitted < nsamp) {
      if ((rc = emit_to(c, out + static_cast<size_t>(emitted) * emit_count(c) * c->n,
                        c->opts.out_on_device != 0, emit_count(c))))
        return rc;
      ++emitted;
    }
  }
  int st[2] = {0, 0};
  MHAR_CUDA(cudaMemcpyAsync(st, c->d.status, sizeof(st), cudaMemcpyDeviceToHost, c->stream),
            "status copy");
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "run sync");
  if (stored(c)) {
    unsigned long long kd = 0;
    MHAR_CUDA(cudaMemcpy(&kd, reinterpret_cast<unsigned long long*>(c->d.check) + 2, sizeof(kd),
                         cudaMemcpyDeviceToHost), "drift copy");
    c->last_drift = host_unkey(kd);
  }
  c->status_bits |= st[0];
  const int code = mhar_status_code(st[0], st[1]);
  switch (code) {
    case MHAR_E_TIMEOUT: set_err(c, "a tensor-core pipeline wait expired"); break;
    case MHAR_E_NONFINITE: set_err(c, "non-finite slack or direction met"); break;
    case MHAR_E_INFEASIBLE_DRIFT:
      set_err(c, "a refresh found the tracked slack beyond its error bound");
      break;
    case MHAR_E_UNBOUNDED:
      set_err(c, "a walker met a chord open on one side: the body is unbounded");
      break;
    default: break;
  }
  return code;
}

int mhar_get_state(const mhar_ctx* cc, double* X, uint64_t* step) {
  mhar_ctx* c = const_cast<mhar_ctx*>(cc);
  if (!c) return MHAR_E_ARG;
  if (X) {
    int rc = emit_to(c, X, false, c->z);
    if (rc) return rc;
  }
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "state sync");
  if (step) *step = c->step;
  return MHAR_OK;
}

int mhar_set_state(mhar_ctx* c, const double* X, uint64_t step) {
  if (!c || !X) return MHAR_E_ARG;
  const size_t zn = static_cast<size_t>(c->z) * c->n;
  if (!all_finite(X, zn)) {
    set_err(c, "non-finite point");
    return MHAR_E_NONFINITE;
  }
  MHAR_CUDA(cudaMemcpyAsync(c->d.emit, X, sizeof(double) * zn, cudaMemcpyHostToDevice, c->stream),
            "copy X");
  MHAR_CUDA(mhar::launch_set_points(c, c->d.emit), "set points kernel");
  c->operands_fresh = false;
  MHAR_CUDA(cudaMemcpyAsync(c->d.step, &step, sizeof(step), cudaMemcpyHostToDevice, c->stream),
            "copy step");
  c->step = step;
  if (stored(c)) {
    int rc;
    if ((rc = refresh(c))) return rc;
  }
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "set_state sync");
  return MHAR_OK;
}

int mhar_get_chord(const mhar_ctx* cc, double* lmin, double* lmax, double* theta) {
  mhar_ctx* c = const_cast<mhar_ctx*>(cc);
  if (!c) return MHAR_E_ARG;
  const size_t bytes = sizeof(double) * c->z;
  if (lmin) MHAR_CUDA(cudaMemcpyAsync(lmin, c->d.lmin, bytes, cudaMemcpyDeviceToHost, c->stream), "copy");
  if (lmax) MHAR_CUDA(cudaMemcpyAsync(lmax, c->d.lmax, bytes, cudaMemcpyDeviceToHost, c->stream), "copy");
  if (theta) MHAR_CUDA(cudaMemcpyAsync(theta, c->d.theta, bytes, cudaMemcpyDeviceToHost, c->stream), "copy");
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "chord sync");
  return MHAR_OK;
}

int mhar_set_preconditioner(mhar_ctx* c, const double* delta, const double* U, int32_t rank) {
  if (!c) return MHAR_E_ARG;
  int rc = MHAR_OK;
  if (!delta) {
    if (c->pc_rank < 0) return MHAR_OK;
    if ((rc = set_sigma(c, c->sigma_A))) return rc;
    direction_norms(c, {});
    return adopt_preconditioner(c, -1);
  }
  if (rank < 0 || rank > mhar::kMaxPcRank || (rank > 0 && !U)) {
    set_err(c, "preconditioner rank must be 0..%d with U given when rank > 0 (got %d)",
            mhar::kMaxPcRank, rank);
    return MHAR_E_ARG;
  }
  const int n = c->n, nl = c->n_ld, R = mhar::kMaxPcRank;
  if (!all_finite(delta, n) || (rank > 0 && !all_finite(U, static_cast<size_t>(n) * rank))) {
    set_err(c, "non-finite preconditioner entry");
    return MHAR_E_NONFINITE;
  }
  for (int i = 0; i < n; ++i)
    if (delta[i] < 0.0) {
      set_err(c, "delta[%d] < 0", i);
      return MHAR_E_ARG;
    }
  if ((rc = alloc_preconditioner(c))) return rc;
  std::vector<double> d64(nl, 0.0), u64(static_cast<size_t>(nl) * R, 0.0);
  for (int i = 0; i < n; ++i) {
    d64[i] = delta[i];
    for (int q = 0; q < rank; ++q)
      u64[static_cast<size_t>(i) * R + q] = U[static_cast<size_t>(i) * rank + q];
  }
  std::vector<float> d32(d64.begin(), d64.end()), u32(u64.begin(), u64.end());
  mhar::DeviceBuffers& d = c->d;
  MHAR_CUDA(cudaMemcpy(d.pc_delta64, d64.data(), sizeof(double) * nl, cudaMemcpyHostToDevice), "copy delta");
  MHAR_CUDA(cudaMemcpy(d.pc_U64, u64.data(), sizeof(double) * u64.size(), cudaMemcpyHostToDevice), "copy U");
  MHAR_CUDA(cudaMemcpy(d.pc_delta32, d32.data(), sizeof(float) * nl, cudaMemcpyHostToDevice), "copy delta");
  MHAR_CUDA(cudaMemcpy(d.pc_U32, u32.data(), sizeof(float) * u32.size(), cudaMemcpyHostToDevice), "copy U");
  if ((rc = precond_scales(c, d64.data(), u64.data()))) return rc;
  return adopt_preconditioner(c, rank);
}

int mhar_get_preconditioner(const mhar_ctx* cc, double* delta, double* U, int32_t* rank) {
  mhar_ctx* c = const_cast<mhar_ctx*>(cc);
  if (!c) return MHAR_E_ARG;
  if (rank) *rank = c->pc_rank;
  if (c->pc_rank < 0) return MHAR_OK;
  const int n = c->n, R = mhar::kMaxPcRank, r = c->pc_rank;
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "preconditioner sync");
  if (delta) MHAR_CUDA(cudaMemcpy(delta, c->d.pc_delta64, sizeof(double) * n, cudaMemcpyDeviceToHost), "copy delta");
  if (U && r > 0) {
    std::vector<double> u64(static_cast<size_t>(n) * R);
    MHAR_CUDA(cudaMemcpy(u64.data(), c->d.pc_U64, sizeof(double) * u64.size(), cudaMemcpyDeviceToHost), "copy U");
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < r; ++q) U[static_cast<size_t>(i) * r + q] = u64[static_cast<size_t>(i) * R + q];
  }
  return MHAR_OK;
}

int mhar_fit_preconditioner(mhar_ctx* c, int64_t warmup, int32_t snapshots, int32_t rank,
                            int32_t power_iters) {
  if (!c) return MHAR_E_ARG;
  if (!fit_args_ok(c, warmup, snapshots) || !factor_args_ok(c, rank, power_iters)) return MHAR_E_ARG;
  mhar::FitScratch f;
  int rc = fit_alloc(c, &f);
  if (rc == MHAR_OK) rc = fit_moments_device(c, warmup, snapshots, nullptr, &f);
  if (rc == MHAR_OK)
    rc = fit_factor_device(c, &f, static_cast<long long>(c->z) * snapshots, rank, power_iters);
  fit_release(c, &f);
  if (rc != MHAR_OK) return rc;
  return fit_adopt(c, rank);
}

int mhar_fit_moments(mhar_ctx* c, int64_t warmup, int32_t snapshots, const double* shift,
                     double* s1, double* s2, int64_t* count) {
  if (!c) return MHAR_E_ARG;
  if (!s1 || !s2 || !count) {
    set_err(c, "s1, s2 and count must not be NULL");
    return MHAR_E_ARG;
  }
  if (!fit_args_ok(c, warmup, snapshots)) return MHAR_E_ARG;
  if (shift && !all_finite(shift, static_cast<size_t>(c->n))) {
    set_err(c, "shift is not finite");
    return MHAR_E_NONFINITE;
  }
  mhar::FitScratch f;
  int rc = fit_alloc(c, &f);
  if (rc == MHAR_OK) rc = fit_moments_device(c, warmup, snapshots, shift, &f);
  const size_t n = static_cast<size_t>(c->n);
  if (rc == MHAR_OK) {
    cudaError_t e = cudaMemcpyAsync(s1, f.s1, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s2, f.s2, sizeof(double) * n * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "copy moments");
  }
  fit_release(c, &f);
  if (rc != MHAR_OK) return rc;
  // Only the upper triangle (j >= i) is accumulated; the rest is returned as
  // its mirror so that s2 is the full symmetric sum.
  for (size_t i = 0; i < n; ++i)
    for (size_t j = 0; j < i; ++j) s2[i * n + j] = s2[j * n + i];
  *count = static_cast<int64_t>(c->z) * snapshots;
  return MHAR_OK;
}

int mhar_fit_from_moments(mhar_ctx* c, const double* s1, const double* s2, int64_t count,
                          int32_t rank, int32_t power_iters) {
  if (!c) return MHAR_E_ARG;
  if (!s1 || !s2 || count < 2) {
    set_err(c, "s1 and s2 must not be NULL and count must be at least 2 (got %lld)",
            static_cast<long long>(count));
    return MHAR_E_ARG;
  }
  if (!factor_args_ok(c, rank, power_iters)) return MHAR_E_ARG;
  const size_t n = static_cast<size_t>(c->n);
  if (!all_finite(s1, n) || !all_finite(s2, n * n)) {
    set_err(c, "the moments are not finite");
    return MHAR_E_NONFINITE;
  }
  mhar::FitScratch f;
  int rc = fit_alloc(c, &f);
  if (rc == MHAR_OK) {
    cudaError_t e = cudaMemcpyAsync(f.s1, s1, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f.s2, s2, sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "copy moments");
  }
  if (rc == MHAR_OK) rc = fit_factor_device(c, &f, static_cast<long long>(count), rank, power_iters);
  fit_release(c, &f);
  if (rc != MHAR_OK) return rc;
  return fit_adopt(c, rank);
}

int mhar_get_stats(const mhar_ctx* c, mhar_stats* s) {
  if (!c || !s) return MHAR_E_ARG;
  std::memset(s, 0, sizeof(*s));
  unsigned long long cnt[2] = {0, 0};
  cudaError_t e = cudaMemcpy(cnt, c->d.counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return MHAR_E_CUDA;
  s->step = c->step;
  s->walker_steps = static_cast<int64_t>(c->step) * c->z;
  s->stalls = static_cast<int64_t>(cnt[0]);
  s->unbounded = static_cast<int64_t>(cnt[1]);
  s->status_bits = c->status_bits;
  s->precision = c->opts.precision;
  s->refresh_drift = c->last_drift;
  s->max_violation = c->max_violation;
  s->eq_residual = c->eq_residual;
  s->kernel_launches = c->launches;
  unsigned long long keys[2];
  e = cudaMemcpy(keys, reinterpret_cast<unsigned long long*>(c->d.check) + 3, sizeof(keys),
                 cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return MHAR_E_CUDA;
  s->run_max_violation = host_unkey(keys[0]);
  s->run_eq_residual = c->mE > 0 ? host_unkey(keys[1]) : 0.0;
  s->audits = c->audits;
  return MHAR_OK;
}

}  // extern "C"

namespace {

// Captures `body` into a graph, replays it once between two events on the
// context's stream and returns the elapsed device milliseconds.
template <typename F>
cudaError_t time_graph(mhar_ctx* c, F body, float* ms) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t eb = body();
    e = cudaStreamEndCapture(c->stream, &g);
    if (eb != cudaSuccess) e = eb;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (e == cudaSuccess) e = cudaGraphUpload(ge, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" {

int mhar_time_kernels(mhar_ctx* c, int iters, double* ms) {
  if (!c || !ms || iters < 1 || iters > 4096) return MHAR_E_ARG;
  int orc = ensure_operands(c);
  if (orc) return orc;
  // (1) `iters` real iterations, replayed back to back from one graph.
  auto full = [&]() -> cudaError_t {
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = enqueue_directions(c, it);
      if (e == cudaSuccess) e = enqueue_chord(c, it);
      if (e != cudaSuccess) return e;
    }
    return mhar::launch_advance(c, iters);
  };
  // (2) the direction kernels alone, `iters` times for the current iteration
  // (idempotent: they rewrite the same directions).
  auto dirs = [&]() -> cudaError_t {
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = enqueue_directions(c, 0);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  float t_full = 0.f, t_dir = 0.f, t_ref = 0.f;
  cudaError_t e = time_graph(c, full, &t_full);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel timing");
  c->launches += static_cast<int64_t>(iters) * kernels_per_iteration(c) + 1;
  c->step += static_cast<uint64_t>(iters);
  if (!tail_draws(c)) {  // otherwise the draw is part of the chord kernel
    e = time_graph(c, dirs, &t_dir);
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel timing");
    c->launches += static_cast<int64_t>(iters) * (kernels_per_iteration(c) - chord_launches(c));
  }
  if (stored(c)) {
    auto ref = [&]() -> cudaError_t {
      cudaError_t e2 = cudaSuccess;
      if (c->mE > 0) e2 = mhar::launch_reproject(c);
      if (e2 == cudaSuccess)
        e2 = c->opts.refresh_fp64 ? mhar::launch_refresh_simt(c) : mhar::launch_refresh_tc(c, false);
      if (e2 == cudaSuccess) e2 = mhar::launch_stored_reset(c);
      return e2;
    };
    e = time_graph(c, ref, &t_ref);
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel timing");
    c->launches += (c->mE > 0 ? 1 : 0) + (c->opts.refresh_fp64 ? 1 : 2) + 1;
    c->since_refresh = 0;
  }
  ms[0] = t_dir / iters;
  ms[1] = (t_full - t_dir) / iters;
  ms[2] = t_ref;
  return MHAR_OK;
}

int mhar_set_audit(mhar_ctx* c, int32_t every, int32_t walkers) {
  if (!c) return MHAR_E_ARG;
  if (every < 0 || walkers < 0 || walkers > c->z) {
    set_err(c, "bad audit setting (every=%d walkers=%d, z=%d)", every, walkers, c->z);
    return MHAR_E_ARG;
  }
  c->opts.audit_every = every;
  c->opts.audit_walkers = walkers;
  c->since_audit = 0;
  return MHAR_OK;
}

int mhar_check(mhar_ctx* c, mhar_stats* s) {
  if (!c) return MHAR_E_ARG;
  const unsigned long long init[2] = {host_key(-INFINITY), host_key(0.0)};
  MHAR_CUDA(cudaMemcpyAsync(c->d.check, init, sizeof(init), cudaMemcpyHostToDevice, c->stream),
            "check init");
  MHAR_CUDA(mhar::launch_check(c, c->z, reinterpret_cast<unsigned long long*>(c->d.check)),
            "check kernel");
  unsigned long long res[2];
  MHAR_CUDA(cudaMemcpyAsync(res, c->d.check, sizeof(res), cudaMemcpyDeviceToHost, c->stream),
            "check copy");
  MHAR_CUDA(cudaStreamSynchronize(c->stream), "check sync");
  c->max_violation = host_unkey(res[0]);
  c->eq_residual = c->mE > 0 ? host_unkey(res[1]) : 0.0;
  return s ? mhar_get_stats(c, s) : MHAR_OK;
}

}  // extern "C"

// ---- batches of problems ----------------------------------------------------------
// Buckets of a batch's problems by the 64-column K chunks of their operands:
// 1, 2, 3-4, 5-8, more.  The walker operands stay in shared memory for the
// first two, and the MMA run of a row tile grows with the chunks, so the
// balance between a unit's set-up and walker-side work and its MMAs, and
// with it the best launch shape, changes from bucket to bucket.
constexpr int kBatchBuckets = 5;

int batch_bucket_of(const mhar_ctx* c) {
  const int kc = c->k_pad / mhar::kTcKChunk;
  return kc <= 1 ? 0 : kc == 2 ? 1 : kc <= 4 ? 2 : kc <= 8 ? 3 : 4;
}

// One bucket in per-bucket mode: its problems, its launch shape and unit
// table (or persistent plan), and a stream of its own.
struct BatchBucket {
  int cls = 0;                      // bucket index (batch_bucket_of)
  std::vector<mhar_ctx*> ctx;
  int max_tiles = 1;                // largest row-tile count of its problems
  int64_t work = 0;                 // sum of m_tiles x k_chunks x strips
  int C = -1;                       // shape; -1: tables not built
  void* table = nullptr;
  int units = 0;
  void* sk = nullptr;
  void* upd = nullptr;              // the walker update of its problems
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

struct mhar_batch {
  std::vector<mhar_ctx*> ctx;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int z = 0;
  int C = 1;                    // cluster size; 0: the persistent stream-K launch
  void* table = nullptr;
  int units = 0;
  void* sk = nullptr;           // stream-K plan (C == 0)
  void* upd = nullptr;          // the walker update of every problem
  uint64_t** steps = nullptr;   // device array of every problem's step counter
  cudaGraphExec_t g_chunk = nullptr;
  cudaGraphExec_t g_one = nullptr;
  int graph_len = 16;
  int64_t launches = 0;
  int64_t walker_steps = 0;
  int64_t since_audit = 0;
  bool per_bucket = false;          // every bucket launched with its own shape
  std::vector<BatchBucket> buckets; // the non-empty buckets
  std::vector<int> bucket_of;       // bucket index of every problem
  cudaEvent_t fork = nullptr;
  mhar_opts opts{};
  char err[512] = {0};
};

namespace {

void batch_err(mhar_batch* b, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->err, sizeof(b->err), fmt, ap);
  va_end(ap);
}

int batch_cuda(mhar_batch* b, cudaError_t e, const char* what) {
  batch_err(b, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return MHAR_E_CUDA;
}

void batch_drop_graphs(mhar_batch* b) {
  if (b->g_chunk) cudaGraphExecDestroy(b->g_chunk);
  if (b->g_one) cudaGraphExecDestroy(b->g_one);
  b->g_chunk = b->g_one = nullptr;
}

void bucket_release(BatchBucket& k) {
  if (k.table) cudaFree(k.table);
  k.table = nullptr;
  k.units = 0;
  mhar::batch_sk_destroy(k.sk);
  k.sk = nullptr;
  k.C = -1;
}

// The bucket's launch with shape C (C as for the whole batch).
int bucket_build(mhar_batch* b, BatchBucket& k, int C) {
  batch_drop_graphs(b);
  bucket_release(k);
  const int n = static_cast<int>(k.ctx.size());
  const int rc = C == 0 ? mhar::batch_sk_build(k.ctx.data(), n, &k.sk, b->err, sizeof(b->err))
                        : mhar::batch_table_build(k.ctx.data(), n, C, &k.table, &k.units, b->err,
                                                  sizeof(b->err));
  if (rc == MHAR_OK) k.C = C;
  return rc;
}

// Problems into their buckets, with a stream and an event per bucket.
int batch_buckets_init(mhar_batch* b) {
  int index[kBatchBuckets];
  for (int& i : index) i = -1;
  b->bucket_of.resize(b->ctx.size());
  for (size_t q = 0; q < b->ctx.size(); ++q) {
    mhar_ctx* c = b->ctx[q];
    const int cls = batch_bucket_of(c);
    if (index[cls] < 0) {
      index[cls] = static_cast<int>(b->buckets.size());
      b->buckets.emplace_back();
      b->buckets.back().cls = cls;
    }
    BatchBucket& k = b->buckets[index[cls]];
    k.ctx.push_back(c);
    const int tiles = mhar::tc_plan_m_tiles(c);
    k.max_tiles = std::max(k.max_tiles, tiles);
    k.work += static_cast<int64_t>(tiles) * (c->k_pad / mhar::kTcKChunk) * mhar::tc_plan_strips(c);
    b->bucket_of[q] = cls;
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (BatchBucket& k : b->buckets) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&k.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return batch_cuda(b, e, "bucket streams");
  int rc = mhar::update_plan_build(b->ctx.data(), static_cast<int>(b->ctx.size()), &b->upd, b->err,
                                   sizeof(b->err));
  for (BatchBucket& k : b->buckets)
    if (rc == MHAR_OK)
      rc = mhar::update_plan_build(k.ctx.data(), static_cast<int>(k.ctx.size()), &k.upd, b->err,
                                   sizeof(b->err));
  return rc;
}

// The largest shape allowed for a bucket at or below C (cluster sizes may
// not exceed its problems' row tiles).
int bucket_clamp(const BatchBucket& k, int C) {
  while (C > 1 && C > k.max_tiles) C /= 2;
  return C;
}

int batch_set_shape(mhar_batch* b, int C) {
  b->per_bucket = false;
  batch_drop_graphs(b);
  for (BatchBucket& k : b->buckets) bucket_release(k);
  if (b->table) cudaFree(b->table);
  b->table = nullptr;
  mhar::batch_sk_destroy(b->sk);
  b->sk = nullptr;
  int rc = C == 0 ? mhar::batch_sk_build(b->ctx.data(), static_cast<int>(b->ctx.size()), &b->sk,
                                         b->err, sizeof(b->err))
                  : mhar::batch_table_build(b->ctx.data(), static_cast<int>(b->ctx.size()), C,
                                            &b->table, &b->units, b->err, sizeof(b->err));
  if (rc == MHAR_OK) b->C = C;
  return rc;
}

cudaError_t batch_enqueue(mhar_batch* b, int count) {
  if (b->per_bucket) {
    // Every bucket on its own stream, forked from and joined back into the
    // batch's stream: the buckets run concurrently, each bucket's iterations
    // in order, and the step counters advance after all of them.
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (BatchBucket& k : b->buckets) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(k.stream, b->fork, 0);
      for (int j = 0; j < count && e == cudaSuccess; ++j) {
        e = k.C == 0 ? mhar::launch_recompute_batch_sk(k.sk, j, k.stream)
                     : mhar::launch_recompute_batch(k.table, k.units, k.C, j, k.stream);
        if (e == cudaSuccess) e = mhar::launch_update_plan(k.upd, j, k.stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(k.done, k.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, k.done, 0);
    }
    if (e != cudaSuccess) return e;
    return mhar::launch_advance_many(b->steps, static_cast<int>(b->ctx.size()), count, b->stream);
  }
  for (int j = 0; j < count; ++j) {
    cudaError_t e = b->C == 0 ? mhar::launch_recompute_batch_sk(b->sk, j, b->stream)
                              : mhar::launch_recompute_batch(b->table, b->units, b->C, j, b->stream);
    if (e == cudaSuccess) e = mhar::launch_update_plan(b->upd, j, b->stream);
    if (e != cudaSuccess) return e;
  }
  return mhar::launch_advance_many(b->steps, static_cast<int>(b->ctx.size()), count, b->stream);
}

int batch_capture(mhar_batch* b, int count, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return batch_cuda(b, e, "begin capture");
  cudaError_t eb = batch_enqueue(b, count);
  e = cudaStreamEndCapture(b->stream, &g);
  if (eb != cudaSuccess) e = eb;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e == cudaSuccess ? MHAR_OK : batch_cuda(b, e, "batch graph");
}

int batch_advance(mhar_batch* b, int64_t count) {
  for (mhar_ctx* c : b->ctx) {
    int rc = ensure_operands(c);
    if (rc) {
      batch_err(b, "%s", c->err);
      return rc;
    }
  }
  if (!b->g_one) {
    int rc = batch_capture(b, 1, &b->g_one);
    if (rc == MHAR_OK) rc = batch_capture(b, b->graph_len, &b->g_chunk);
    if (rc) return rc;
  }
  const int64_t n = count;
  // Each bucket's (or the batch's) chord kernel and walker update.
  const int64_t per_iter = 2 * (b->per_bucket ? static_cast<int64_t>(b->buckets.size()) : 1);
  while (count >= b->graph_len) {
    cudaError_t e = cudaGraphLaunch(b->g_chunk, b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "graph launch");
    count -= b->graph_len;
    b->launches += b->graph_len * per_iter + 1;
  }
  while (count-- > 0) {
    cudaError_t e = cudaGraphLaunch(b->g_one, b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "graph launch");
    b->launches += per_iter + 1;
  }
  for (mhar_ctx* c : b->ctx) c->step += static_cast<uint64_t>(n);
  b->walker_steps += n * b->z * static_cast<int64_t>(b->ctx.size());
  return MHAR_OK;
}

// Device time of `iters` iterations with the current shape(s), after one
// untimed iteration that captures the graphs.  The iterations are real:
// every walk advances.
int batch_time(mhar_batch* b, int iters, float* ms) {
  int rc = batch_advance(b, 1);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
  if (e == cudaSuccess) {
    rc = batch_advance(b, iters);
    if (rc == MHAR_OK) e = cudaEventRecord(e1, b->stream);
  }
  if (rc == MHAR_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (rc == MHAR_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  return e == cudaSuccess ? MHAR_OK : batch_cuda(b, e, "tuning");
}

// Per-bucket mode; buckets without a table yet take shape C0 (clamped).
int batch_enter_buckets(mhar_batch* b, int C0) {
  if (b->table) cudaFree(b->table);
  b->table = nullptr;
  mhar::batch_sk_destroy(b->sk);
  b->sk = nullptr;
  batch_drop_graphs(b);
  for (BatchBucket& k : b->buckets) {
    if (k.C >= 0) continue;
    const int rc = bucket_build(b, k, bucket_clamp(k, C0));
    if (rc) return rc;
  }
  b->per_bucket = true;
  return MHAR_OK;
}

}  // namespace

extern "C" {

int mhar_batch_create(const mhar_problem* problems, int32_t count, int32_t z,
                      const mhar_opts* opts, mhar_batch** out) {
  if (!out) return MHAR_E_ARG;
  *out = nullptr;
  if (!problems || count < 1 || z < 1) return MHAR_E_ARG;
  mhar_batch* b = new (std::nothrow) mhar_batch();
  if (!b) return MHAR_E_ARG;
  if (opts) b->opts = *opts; else mhar_default_opts(&b->opts);
  b->z = z;
  int rc = MHAR_OK;
  if (b->opts.stream) {
    b->stream = static_cast<cudaStream_t>(b->opts.stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = batch_cuda(b, e, "stream create");
    b->own_stream = true;
  }
  for (int q = 0; q < count && rc == MHAR_OK; ++q) {
    const mhar_problem& pr = problems[q];
    mhar_opts o = b->opts;
    o.seed = b->opts.seed + static_cast<uint64_t>(q);
    o.precision = MHAR_MIXED_RECOMPUTE;
    o.smem_operands = 1;
    o.stream = b->stream;
    o.graph_chunk = 0;
    mhar_ctx* c = nullptr;
    rc = mhar_create(pr.A, pr.b, pr.m, pr.n, nullptr, nullptr, 0, pr.x0, z, &o, &c);
    if (rc != MHAR_OK) {
      batch_err(b, "problem %d: %s", q, mhar_strerror(rc));
      break;
    }
    b->ctx.push_back(c);
  }
  if (rc == MHAR_OK) {
    std::vector<uint64_t*> steps;
    for (mhar_ctx* c : b->ctx) steps.push_back(c->d.step);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->steps), sizeof(uint64_t*) * steps.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(b->steps, steps.data(), sizeof(uint64_t*) * steps.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = batch_cuda(b, e, "step table");
  }
  if (rc == MHAR_OK) rc = batch_buckets_init(b);
  if (rc == MHAR_OK) {
    // Default shape: one CTA per unit when the units alone fill the GPU.
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx[0]->device);
    int strips = 0;
    for (mhar_ctx* c : b->ctx) strips += mhar::tc_plan_strips(c);
    int C = 1;
    while (C < 8 && strips * C * 2 <= sms) C *= 2;
    rc = batch_set_shape(b, C);
  }
  if (rc != MHAR_OK) {
    remember_create_error(b->err);
    mhar_batch_destroy(b);
    return rc;
  }
  *out = b;
  return MHAR_OK;
}

int mhar_batch_tune(mhar_batch* b, int32_t iters, int32_t* cluster) {
  if (!b || iters < 1 || iters > 1024) return MHAR_E_ARG;
  int max_tiles = 1;
  for (mhar_ctx* c : b->ctx)
    max_tiles = std::max(max_tiles, mhar::tc_plan_m_tiles(c));
  int best_C = b->C;
  float best = INFINITY;
  // (1) One shape for the whole batch: the persistent launch (C = 0), then
  // clusters of 1, 2, 4, 8.
  for (int C = 0; C <= 8; C = C == 0 ? 1 : 2 * C) {
    if (C > max_tiles) break;
    int rc = batch_set_shape(b, C);
    if (rc) return rc;
    float ms = 0.f;
    rc = batch_time(b, iters, &ms);
    if (rc) return rc;
    if (ms < best) {
      best = ms;
      best_C = C;
    }
  }
  // (2) A shape per bucket, by coordinate descent from the best single
  // shape: one bucket at a time (most work first) tries every other shape
  // with the whole batch timed; a change stays only if the batch runs more
  // than 1 % faster.  The mix is kept if it beats the best single shape by
  // more than 1 %.
  bool mix = false;
  if (b->buckets.size() >= 2) {
    for (BatchBucket& k : b->buckets) bucket_release(k);
    int rc = batch_enter_buckets(b, best_C);
    float cur = 0.f;
    if (rc == MHAR_OK) rc = batch_time(b, iters, &cur);
    if (rc) return rc;
    std::vector<BatchBucket*> order;
    for (BatchBucket& k : b->buckets) order.push_back(&k);
    std::stable_sort(order.begin(), order.end(),
                     [](const BatchBucket* x, const BatchBucket* y) { return x->work > y->work; });
    for (BatchBucket* k : order) {
      for (int C = 0; C <= 8; C = C == 0 ? 1 : 2 * C) {
        if (C > k->max_tiles) break;
        const int prev = k->C;
        if (C == prev) continue;
        rc = bucket_build(b, *k, C);
        float ms = 0.f;
        if (rc == MHAR_OK) rc = batch_time(b, iters, &ms);
        if (rc) return rc;
        if (ms < 0.99f * cur) {
          cur = ms;
        } else if ((rc = bucket_build(b, *k, prev))) {
          return rc;
        }
      }
    }
    mix = cur < 0.99f * best;
  }
  if (!mix) {
    const int rc = batch_set_shape(b, best_C);
    if (rc) return rc;
  }
  if (cluster) *cluster = mix ? -1 : best_C;
  return MHAR_OK;
}

int mhar_batch_set_shape(mhar_batch* b, int32_t shape) {
  if (!b) return MHAR_E_ARG;
  int max_tiles = 1;
  for (mhar_ctx* c : b->ctx) max_tiles = std::max(max_tiles, mhar::tc_plan_m_tiles(c));
  if (!(shape == 0 || shape == 1 || shape == 2 || shape == 4 || shape == 8) ||
      (shape > 1 && shape > max_tiles)) {
    batch_err(b, "shape %d: 0 (stream-K) or a cluster size 1, 2, 4, 8 up to %d row tiles",
              shape, max_tiles);
    return MHAR_E_ARG;
  }
  return batch_set_shape(b, shape);
}

int mhar_batch_set_bucket_shape(mhar_batch* b, int32_t bucket, int32_t shape) {
  if (!b) return MHAR_E_ARG;
  BatchBucket* k = nullptr;
  for (BatchBucket& x : b->buckets)
    if (x.cls == bucket) k = &x;
  if (!k || !(shape == 0 || shape == 1 || shape == 2 || shape == 4 || shape == 8) ||
      (shape > 1 && shape > k->max_tiles)) {
    batch_err(b, "bucket %d shape %d: a non-empty bucket 0..%d and 0 (persistent) or a cluster "
              "size 1, 2, 4, 8 up to %d row tiles", bucket, shape, kBatchBuckets - 1,
              k ? k->max_tiles : 0);
    return MHAR_E_ARG;
  }
  if (!b->per_bucket) {
    for (BatchBucket& x : b->buckets) bucket_release(x);
    const int rc = batch_enter_buckets(b, b->C);
    if (rc) return rc;
  }
  return bucket_build(b, *k, shape);
}

int mhar_batch_get_shapes(const mhar_batch* b, int32_t* per_bucket, int32_t* shape,
                          int32_t* bucket_of) {
  if (!b) return MHAR_E_ARG;
  if (per_bucket) *per_bucket = b->per_bucket ? 1 : 0;
  if (shape) {
    for (int i = 0; i < kBatchBuckets; ++i) shape[i] = -1;
    for (const BatchBucket& k : b->buckets) shape[k.cls] = b->per_bucket ? k.C : b->C;
  }
  if (bucket_of)
    for (size_t q = 0; q < b->bucket_of.size(); ++q) bucket_of[q] = b->bucket_of[q];
  return MHAR_OK;
}

int mhar_batch_run(mhar_batch* b, int64_t steps, int64_t thin, double* const* out) {
  if (!b || steps < 0 || thin < 0) return MHAR_E_ARG;
  const int64_t nsamp = thin > 0 ? steps / thin : 0;
  if (nsamp > 0 && !out) {
    batch_err(b, "out is NULL but samples are due");
    return MHAR_E_ARG;
  }
  for (mhar_ctx* c : b->ctx) {
    cudaError_t e = cudaMemsetAsync(c->d.status, 0, 2 * sizeof(int), b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "status reset");
  }
  int64_t done = 0, emitted = 0;
  const int64_t au = b->opts.audit_every;
  while (done < steps) {
    int64_t adv = steps - done;
    if (thin > 0) adv = std::min<int64_t>(adv, thin - (done % thin));
    if (au > 0) adv = std::min<int64_t>(adv, au - b->since_audit);
    int rc = batch_advance(b, adv);
    if (rc) return rc;
    done += adv;
    if (au > 0 && (b->since_audit += adv) >= au) {
      for (mhar_ctx* c : b->ctx) {
        if ((rc = audit(c))) {
          batch_err(b, "audit: %s", c->err);
          return rc;
        }
      }
      b->since_audit = 0;
    }
    if (thin > 0 && done % thin == 0 && emitted < nsamp) {
      for (size_t q = 0; q < b->ctx.size(); ++q) {
        mhar_ctx* c = b->ctx[q];
        if (!out[q]) continue;
        rc = emit_to(c, out[q] + static_cast<size_t>(emitted) * emit_count(c) * c->n,
                     c->opts.out_on_device != 0, emit_count(c));
        if (rc) {
          batch_err(b, "problem %zu: %s", q, c->err);
          return rc;
        }
      }
      ++emitted;
    }
  }
  int worst = MHAR_OK;
  for (size_t q = 0; q < b->ctx.size(); ++q) {
    mhar_ctx* c = b->ctx[q];
    int st[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(st, c->d.status, sizeof(st), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "status copy");
    c->status_bits |= st[0];
    if (st[1]) {
      batch_err(b, "problem %zu: a tensor-core pipeline wait expired", q);
      return MHAR_E_TIMEOUT;
    }
    if ((st[0] & MHAR_ST_NONFINITE) && worst == MHAR_OK) {
      batch_err(b, "problem %zu: non-finite slack or direction met", q);
      worst = MHAR_E_NONFINITE;
    }
    if ((st[0] & MHAR_ST_UNBOUNDED) && worst == MHAR_OK) {
      batch_err(b, "problem %zu: a chord open on one side (unbounded body)", q);
      worst = MHAR_E_UNBOUNDED;
    }
  }
  return worst;
}

int mhar_batch_get_state(const mhar_batch* b, int32_t problem, double* X, uint64_t* step) {
  if (!b || problem < 0 || problem >= static_cast<int>(b->ctx.size())) return MHAR_E_ARG;
  return mhar_get_state(b->ctx[problem], X, step);
}

int mhar_batch_check(mhar_batch* b, int32_t problem, mhar_stats* stats) {
  if (!b || problem < 0 || problem >= static_cast<int>(b->ctx.size())) return MHAR_E_ARG;
  int rc = mhar_check(b->ctx[problem], stats);
  if (rc == MHAR_OK && stats) stats->kernel_launches += b->launches;  // the batch's own launches
  return rc;
}

int mhar_batch_set_audit(mhar_batch* b, int32_t every, int32_t walkers) {
  if (!b) return MHAR_E_ARG;
  for (mhar_ctx* c : b->ctx) {
    const int rc = mhar_set_audit(c, every, walkers);
    if (rc) {
      batch_err(b, "%s", c->err);
      return rc;
    }
  }
  b->opts.audit_every = every;
  b->opts.audit_walkers = walkers;
  b->since_audit = 0;
  return MHAR_OK;
}

const char* mhar_batch_last_error(const mhar_batch* b) {
  if (!b) return "null batch";
  return b->err[0] ? b->err : "no error";
}

void mhar_batch_destroy(mhar_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  if (b->table) cudaFree(b->table);
  mhar::batch_sk_destroy(b->sk);
  for (BatchBucket& k : b->buckets) {
    bucket_release(k);
    mhar::update_plan_destroy(k.upd);
    if (k.done) cudaEventDestroy(k.done);
    if (k.stream) cudaStreamDestroy(k.stream);
  }
  mhar::update_plan_destroy(b->upd);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->steps) cudaFree(b->steps);
  for (mhar_ctx* c : b->ctx) mhar_destroy(c);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
