// mhar_internal.h -- the context layout and the kernel launchers shared by the
// library's translation units.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "../../include/mhar.h"

namespace mhar {

// Tile geometry of the tensor-core path (fixed by the kernel design).
constexpr int kTcM = 128;        // rows of A per MMA tile (TMEM lanes)
constexpr int kTcKChunk = 64;    // FP16 elements per 128-byte swizzled row chunk
constexpr int kTcK = 16;         // K of one kind::f16 MMA

struct DeviceBuffers {
  // Problem (row-major, zero padded to the leading dimensions below).
  double* A64 = nullptr;   // m x n_ld
  double* b64 = nullptr;   // m
  float* A32 = nullptr;    // m x n_ld (FP32 mode)
  float* b32 = nullptr;    // m (FP32 mode: lowered by 3 u |b_i|, see kernels_simt.cu)
  float* kr32 = nullptr;   // 2 m (FP32 mode: the row bounds of chord_simt_kernel)
  double* AE64 = nullptr;  // mE x n_ld
  double* bE64 = nullptr;  // mE
  double* Q64 = nullptr;   // mE x n_ld, orthonormal rows: Q = L^{-1} A_E, P = I - Q^T Q
  float* Q32 = nullptr;    // mE x n_ld, Q in FP32
  float* Q32lo = nullptr;  // mE x n_ld, fl32(Q - Q32): Q32 + Q32lo is Q to about 2^-48
  double* wE64 = nullptr;  // mE, w = L^{-1} b_E (Q x = w on the affine subspace)
  double* Lchol = nullptr; // mE x mE, set-up scratch: Cholesky factors of the Gram matrices
  // Tensor-core operands: A split into FP16 hi/lo after a per-row power-of-two
  // scale; rows padded to m_pad, columns to k_pad.
  __half* Ah = nullptr;    // m_pad x k_pad
  __half* Al = nullptr;    // m_pad x k_pad
  float* row_scale = nullptr; // m_pad: A[i,:] = row_scale[i] * (Ah + Al)[i,:]
  float* bS = nullptr;     // m_pad (FP32 b / row_scale, lowered, 0 beyond m)
  // 4 m_pad: per 32-row block, bS (as above), then Ks (error bound of a_i . x
  // per unit of the walker's point norm), then Kg (of a_i . d per unit of its
  // direction norm), then the block's norm type; tc_common.cuh, row_block.
  float* rows = nullptr;
  float* rowk = nullptr;   // 4 m_pad: Ks_2, Kg_2, Ks_1, Kg_1 of every row (kernels_simt.cu)

  // Walker state.
  double* X64 = nullptr;   // z x n_ld          (FP64 mode)
  float* Xhi = nullptr;    // z x n_ld          (FP32 / mixed: double-float)
  float* Xlo = nullptr;    // z x n_ld
  double* D64 = nullptr;   // z x n_ld          (FP64 mode)
  float* D32 = nullptr;    // z x n_ld          (FP32 mode; mixed: pre-projection scratch)
  __half* Dh = nullptr;    // z x k_pad         (mixed)
  __half* Dl = nullptr;    // z x k_pad         (mixed)
  // Recompute mode: a second pair, so that iteration s reads the directions
  // from pair s % 2 while the next directions go into the other one.
  __half* Dh2 = nullptr;
  __half* Dl2 = nullptr;
  float* S = nullptr;      // m_pad x z_ld      (mixed: tracked slack / row_scale, blocked:
                           //  element (i, k) at ((i / 4) z_ld + k) 4 + i % 4)
  float* corr = nullptr;   // z x mE            (FP32 / mixed with equalities: residual fix, Q d)
  float* corrn = nullptr;  // z                 (the same: ||Q^T corr / sigma||_2 bound)
  __half* Xh = nullptr;    // z_ld x k_pad      (mixed: refresh operand, FP16 hi of scaled X)
  __half* Xl = nullptr;    // z_ld x k_pad      (mixed: FP16 lo)
  float* wscale = nullptr; // z_ld              (mixed: power-of-two scale of each walker)
  // Stored-slack mode: the tracked slack's error since the last refresh.
  float* nx_ref = nullptr;       // z: ||x / sigma||_2 bound at the refresh
  float* theta_acc = nullptr;    // z: sum |theta| ||d_hat||_2 since the refresh
  uint64_t* refresh_step = nullptr;  // iteration counter at the refresh

  // Chord bookkeeping.
  unsigned long long* key_lo = nullptr;  // z: ordered key of lambda_min (atomic max)
  unsigned long long* key_hi = nullptr;  // z: ordered key of lambda_max (atomic min)
  double* lmin = nullptr;  // z
  double* lmax = nullptr;  // z
  double* theta = nullptr; // z
  int* status = nullptr;   // [0] bits, [1] spare
  unsigned long long* counters = nullptr;  // [0] stalls, [1] unbounded
  uint64_t* step = nullptr;  // device iteration counter (graph replays read it)
  double* emit = nullptr;  // z x n staging for host output
  double* check = nullptr; // keys: [0] max violation, [1] eq residual, [2] drift,
                           // [3], [4] running max violation / eq residual of the audits

  // Direction preconditioner d = P (delta .* h + U g) (allocated when set).
  double* pc_delta64 = nullptr;  // n_ld
  double* pc_U64 = nullptr;      // n_ld x 32, row i = U[i, :], zero beyond the rank
  float* pc_delta32 = nullptr;   // n_ld
  float* pc_U32 = nullptr;       // n_ld x 32
  // Power-of-two scale of each coordinate, from the columns of A (every
  // column of A sigma has its largest entry in [0.5, 1) up to one common
  // power of two) and, with a preconditioner, kept within the FP16 range of
  // the scaled directions.  The tensor-core operands hold x_i / sigma_i and
  // d_i / sigma_i and A's columns are multiplied by sigma_i, so A x and A d
  // are unchanged while coordinates of very different size keep their
  // relative precision; every mode bounds its rounding errors in these
  // coordinates (Cauchy-Schwarz on |a_i sigma| . |x / sigma|).
  float* sigma = nullptr;        // n_ld (1 beyond n)
};

}  // namespace mhar

struct mhar_ctx {
  int m = 0, n = 0, mE = 0, z = 0;
  int n_ld = 0;   // walker-major leading dimension for X / D (FP32, FP64)
  int k_pad = 0;  // FP16 operand leading dimension (multiple of 64)
  int m_pad = 0;  // rows of A padded to the tensor-core tile (multiple of 128)
  int kdim = 0;   // MMA reduction length actually used (multiple of 16, >= n)
  mhar_opts opts{};
  cudaStream_t stream = nullptr;
  uint64_t step = 0;
  int64_t since_refresh = 0;
  int device = 0;
  mhar::DeviceBuffers d;
  void* tc = nullptr;  // tensor-core plan (tensor maps, launch shape)
  cudaGraphExec_t g_chunk = nullptr;
  cudaGraphExec_t g_one = nullptr;
  int graph_len = 0;
  int64_t launches = 0;        // kernels launched (graph replays add their nodes)
  int64_t launches_chunk = 0;  // kernel nodes in g_chunk
  int64_t launches_one = 0;    // kernel nodes in g_one
  bool use_ts = false;         // recompute mode: TMEM-operand kernel (n <= 128)
  bool use_sk = false;         // recompute mode: stream-K schedule (kernels_sk.cu)
  void* sk = nullptr;          // its segment table
  int pc_rank = -1;            // -1: isotropic directions; else rank of U (0..32)
  // Recompute mode: the chord kernel itself moves the walkers, re-splits the
  // points and (with no projection / preconditioner) draws the next
  // directions; `operands_fresh` says whether the FP16 operands of the next
  // iteration are in place (false after any change of state from the host).
  bool operands_fresh = false;
  bool unit_sigma = true;      // every sigma_i == 1
  std::vector<float> sigma_A;  // the column scales of A alone (host copy)
  std::vector<float> sigma_host;  // the scales in force (host copy of d.sigma)
  int64_t since_audit = 0;     // iterations since the last audit (opts.audit_every)
  // Typical 2-norm and max-norm of a scaled direction d / sigma, for the
  // choice of bound form per 32-row block (kernels_simt.cu, row_blocks_kernel).
  double dir_norm2 = 1.0, dir_norminf = 1.0;
  int64_t audits = 0;
  double last_drift = 0.0;
  double max_violation = 0.0;
  double eq_residual = 0.0;
  int status_bits = 0;
  char err[512] = {0};
};

namespace mhar {

// MMAs (K = 16) accumulated into one output of the tensor-core products: three
// FP16 products per K step in the recompute mode, four in the stored mode.
inline int mma_per_step(const mhar_ctx* c) {
  return c->opts.precision == MHAR_MIXED_F16X3 ? 4 : 3;
}
inline int mma_chain(const mhar_ctx* c) { return mma_per_step(c) * (c->kdim / kTcK); }

// ---- kernel launchers (kernels_simt.cu) -------------------------------------
// Every launcher enqueues on ctx->stream and returns cudaGetLastError().
// `j` is the iteration offset added to the device counter *d.step.
cudaError_t launch_directions(mhar_ctx* ctx, int j);
// draw: the FP32 / tensor-core projection draws h itself (no preconditioner);
// otherwise it projects the direction kernels' D32 (D64 in FP64 mode).
cudaError_t launch_projection(mhar_ctx* ctx, int j, int draw);
// Opens the projection kernels' dynamic shared memory to mE coefficient
// vectors per block (call once per context before the first launch).
cudaError_t projection_smem_attr(int mE, int n);
cudaError_t launch_chord_simt(mhar_ctx* ctx);
// Small bodies in the FP64 / FP32 modes: one warp per walker does the chord,
// theta and the move (Sections 4.4-4.5) in a single launch.
bool simt_warp_path(const mhar_ctx* ctx);
cudaError_t launch_chord_update_warp(mhar_ctx* ctx, int j);
cudaError_t launch_update_simt(mhar_ctx* ctx, int j);
cudaError_t launch_advance(mhar_ctx* ctx, int steps);
// Recompute mode: flags bit 1 split X, bit 2 draw D (for iteration step + j).
cudaError_t launch_prep_walkers(mhar_ctx* ctx, int j, int flags);
cudaError_t launch_emit(mhar_ctx* ctx, double* out_device, int walkers);  // walkers 0..walkers-1
// FP64 feasibility of walkers 0..walkers-1 into the keys at out_keys[0]
// (max a_i x - b_i) and out_keys[1] (max |A_E x - b_E|).
cudaError_t launch_check(mhar_ctx* ctx, int walkers, unsigned long long* out_keys);
// Stored-slack mode, after a refresh: ||x / sigma|| of every walker, the
// accumulated step sum reset, the refresh's iteration recorded.
cudaError_t launch_stored_reset(mhar_ctx* ctx);
cudaError_t launch_set_points(mhar_ctx* ctx, const double* X_dev);
cudaError_t launch_prepare_tc_operands(mhar_ctx* ctx);
cudaError_t launch_refresh_simt(mhar_ctx* ctx);
cudaError_t launch_reproject(mhar_ctx* ctx);
// d <- delta .* d + U g on the drawn normals (FP64 / FP32 scratch), writing the
// FP16 pair (divided by sigma) when `split`.
cudaError_t launch_precondition(mhar_ctx* ctx, int j, int split);

// ---- preconditioner fit (kernels_fit.cu) --------------------------------------
struct FitScratch {
  double* shift = nullptr;   // n: centre subtracted before the products
  double* s1 = nullptr;      // n: sum of (x - shift)
  double* s2 = nullptr;      // n x n: sum of (x - shift)(x - shift)^T (upper tiles)
  double* sigma = nullptr;   // n x n covariance
  double* Y = nullptr;       // n x 32
  double* Q = nullptr;       // n x 32
  int* flag = nullptr;       // [0] set when a fit kernel met a non-finite value
};
cudaError_t launch_fit_shift(mhar_ctx* ctx, FitScratch* f);   // shift = walker 0's point
cudaError_t launch_fit_accumulate(mhar_ctx* ctx, FitScratch* f);
cudaError_t launch_fit_factor(mhar_ctx* ctx, FitScratch* f, long long samples, int rank,
                              int power_iters);

// ---- errors without a context (mhar_api.cu) -----------------------------------
// The message mhar_last_error(NULL) returns on this host thread: the last
// failed mhar_create / mhar_batch_create, or the last mhar_chord_noalloc
// (cleared when that call succeeds).  NULL clears it.
void set_null_error(const char* msg);

// ---- tensor-core path (kernels_tc.cu) ---------------------------------------
int tc_plan_create(mhar_ctx* ctx);            // 0 or MHAR_E_*
int tc_plan_strips(const mhar_ctx* ctx);      // walker strips of 128
int tc_plan_m_tiles(const mhar_ctx* ctx);     // row tiles of 128
void tc_plan_destroy(mhar_ctx* ctx);
cudaError_t launch_chord_tc(mhar_ctx* ctx, int j);
// X split + S = b - A X (2 launches); check_drift: flag MHAR_ST_DRIFT where the
// tracked slack differs from the recomputed one by more than its error bound.
cudaError_t launch_refresh_tc(mhar_ctx* ctx, bool check_drift);
cudaError_t launch_split_points(mhar_ctx* ctx);     // X -> FP16 pair + per-walker scale

// ---- recompute-slack tensor-core path (kernels_rc.cu) ------------------------
int rc_prepare(mhar_ctx* ctx);                      // 0 or MHAR_E_*
cudaError_t launch_recompute_tc(mhar_ctx* ctx, int j);

// Batches (one launch per iteration for many problems, recompute mode with
// shared-memory operands): a device table of (problem, walker strip) units
// for clusters of C CTAs, largest units first.
int batch_table_build(mhar_ctx* const* ctx, int count, int C, void** table, int* units,
                      char* err, size_t err_len);
cudaError_t launch_recompute_batch(const void* table, int units, int C, int j,
                                   cudaStream_t stream);
// Batched persistent stream-K launch (kernels_sk.cu): one CTA per SM, the
// batch's (problem, strip, row tile) work cut into cost-balanced ranges.
int batch_sk_build(mhar_ctx* const* ctx, int count, void** plan, char* err, size_t err_len);
void batch_sk_destroy(void* plan);
cudaError_t launch_recompute_batch_sk(const void* plan, int j, cudaStream_t stream);
// The batch kernels leave the walker-side work (the moves and the FP16 pairs
// of the moved points, walker_tail.cuh) to one update launch per iteration
// over all the batch's problems (kernels_sk.cu): a device table of
// (problem, walkers) units built from the contexts.
int update_plan_build(mhar_ctx* const* ctx, int count, void** plan, char* err, size_t err_len);
void update_plan_destroy(void* plan);
cudaError_t launch_update_plan(const void* plan, int j, cudaStream_t stream);
cudaError_t launch_advance_many(uint64_t* const* steps, int count, int by, cudaStream_t stream);

// Whether the stream-K schedule beats clusters along the rows for this shape.
bool rc_prefers_stream_k(const mhar_ctx* ctx);

// ---- recompute-slack, stream-K schedule (kernels_sk.cu) ------------------------
int sk_prepare(mhar_ctx* ctx);
void sk_destroy(mhar_ctx* ctx);
cudaError_t launch_recompute_sk(mhar_ctx* ctx, int j);

// ---- recompute-slack, walker operands in tensor memory (kernels_ts.cu) -------
bool ts_eligible(const mhar_ctx* ctx);              // n <= 128
int ts_prepare(mhar_ctx* ctx);
cudaError_t launch_recompute_ts(mhar_ctx* ctx, int j);

}  // namespace mhar
