// kernels_tc.cu -- the fused tensor-core walker step (MHAR_MIXED_F16X3 mode).
//
// One launch performs, for every walker, Sections 4.4 and 4.5 of the paper on
// the stored slack S = b - A X:
//   G = D A^T           tcgen05.mma kind::f16 (FP16 hi/lo split operands,
//                       3 products hi.hi + hi.lo + lo.hi, FP32 accumulation
//                       in tensor memory; TMA-staged 128B-swizzled tiles)
//   lambda_max = min{ s_i / g_i : g_i > 0 },  lambda_min = max{ s_i / g_i : g_i < 0 }
//                       folded in registers straight out of tensor memory --
//                       the m x z ratio matrix never reaches memory
//   theta = lambda_min + u (lambda_max - lambda_min),  u from Philox stream 1
//   S -= G diag(theta),  X += D diag(theta)   (X as FP32 pairs)
//
// Work decomposition.  The MMA's M dimension is the walkers (128 per CTA, one
// walker per tensor-memory lane, so every thread owns one walker and reduces
// its chord sequentially), N is the constraint rows (128 per tile), K is the
// dimension n.  The rows of A are split over the CTAs of a thread-block
// cluster (up to 4 tiles = 512 tensor-memory columns per CTA); the partial
// chords are combined through distributed shared memory, so each CTA can
// update its own slack rows while G is still in tensor memory.
//
// Warp roles (320 threads): warp 0 = TMA producer, warp 1 = MMA issuer and
// tensor-memory owner, warps 2..9 = epilogue (two warps per 32-lane quarter,
// each taking half of every tile's columns).
//
// Every mbarrier wait is bounded (about 2 s of clock); on expiry the kernel
// records a timeout in the error word, stops waiting and still runs
// through every cluster barrier, so no peer is left waiting.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cstdio>
#include <cstring>

#include "mhar_device.cuh"
#include "mhar_internal.h"
#include "tc_common.cuh"
#include "walker_tail.cuh"

namespace mhar {
namespace {

using namespace tc;

constexpr int kStages = 3;
constexpr int kMaxTilesPerCta = 4;                    // 512 TMEM columns
constexpr int kStageBytes = 4 * kOperandBytes;        // A hi, A lo, W hi, W lo
constexpr int kEpiWarps = 16;                         // 4 per TMEM lane quarter
constexpr int kThreadsTc = (2 + kEpiWarps) * 32;

enum : int { kModeChord = 0, kModeRefresh = 1 };

struct TcParams {
  int mode;                 // kModeChord | kModeRefresh
  const float* row_scale;   // m_pad: A[i,:] = row_scale[i] (Ah + Al)[i,:]
  const float* bS;          // m_pad: b[i] / row_scale[i] in FP32 (refresh)
  const float* wscale;      // z_ld: X[k,:] = wscale[k] (Xh + Xl)[k,:] (refresh)
  float* S;                 // slack / row_scale, blocked: [(i/4) z_ld + k] * 4 + i%4
  float* Xhi;               // z x n_ld
  float* Xlo;
  const float* rowk;        // 4 m_pad: Ks_2, Kg_2, Ks_1, Kg_1 of every row (prepare_tc_kernel)
  const __half* Xh;         // z_ld x k_pad: FP16 hi of the points split at the last refresh
  const float* corrn;       // z or null: ||Q^T corr / sigma||_2 (see add_correction)
  // The tracked slack's error since the last refresh, per walker: bounded by
  // Ks_i E_k + k 2^-24 |b_i / scale_i| after k updates, with
  //   E_k = (||x_r / sigma|| + sum_t |theta_t| ||d_hat_t||) (1 + k / (4 T + 4)),
  // x_r the point at the refresh and T the MMAs of one product chain.
  const float* nx_ref;      // z: ||x_r / sigma||_2 bound, set by every refresh
  float* theta_acc;         // z: sum_t |theta_t| ||d_hat_t||_2 since the refresh
  const uint64_t* refresh_step;  // iteration counter at the last refresh
  float growth;             // 1 / (4 T + 4)
  int check_drift;          // refresh: compare the tracked slack with its bound
  const __half* Dh;         // z_ld x k_pad
  const __half* Dl;
  const float* sigma;       // n_ld: coordinate scales (operands hold x / sigma, d / sigma)
  const float* Q32;         // mE x n_ld (orthonormal rows of the equalities) or null
  const float* corr;        // z x mE residual corrections or null
  double* lmin;
  double* lmax;
  double* theta;
  int* status;
  unsigned long long* counters;
  int* err;
  unsigned long long* drift_key;
  const uint64_t* step_ptr;
  uint64_t seed;
  int j;
  uint32_t walker0;
  int m, n, n_ld, z, z_ld, kdim, k_chunks, tiles_per_cta, m_tiles, mE;
};

struct SmemTail {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tfull[kMaxTilesPerCta];
  uint32_t tmem_base;
  int timed_out;
  float part_lo[4][kWalkers];
  float part_hi[4][kWalkers];
  float cta_lo[kWalkers];
  float cta_hi[kWalkers];
  float theta[kWalkers];
  float scale[kMaxTilesPerCta * kRowsTile];
  float brow[kMaxTilesPerCta * kRowsTile];
  float ks[kMaxTilesPerCta * kRowsTile];   // Ks_i of this CTA's rows
  float kg[kMaxTilesPerCta * kRowsTile];   // Kg_i
  float jk[kMaxTilesPerCta * kRowsTile];   // k 2^-24 |b_i / scale_i|, k updates since the refresh
  float nrm[3 * kWalkers];                 // operand_norms
  float nd[kWalkers];                      // ||d_hat||_2 bound of each walker's direction
};

constexpr size_t kSmemBytes = 1024 + static_cast<size_t>(kStages) * kStageBytes + sizeof(SmemTail);
static_assert(kSmemBytes <= 232448, "walker_tc_kernel exceeds the shared memory of a CTA");

// The slack is stored blocked by 4 rows: element (i, k) sits at
// ((i / 4) z_ld + k) 4 + i % 4, so one 16-byte access gives a walker four
// consecutive rows and a warp's 32 consecutive walkers read 512 contiguous
// bytes.  32 rows of one walker = eight such accesses, z_ld * 16 bytes apart.
__device__ __forceinline__ float* s_block(const TcParams& p, int row, int k) {
  return p.S + (static_cast<size_t>(row >> 2) * p.z_ld + k) * 4;
}
__device__ __forceinline__ void load_s32(const TcParams& p, const float* src, float (&v)[32]) {
  const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 t = __ldcg(q + static_cast<size_t>(i) * p.z_ld);
    v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
  }
}
__device__ __forceinline__ void store_s32(const TcParams& p, float* dst, const float (&v)[32]) {
  float4* q = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    __stcg(q + static_cast<size_t>(i) * p.z_ld, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
}

__global__ void __launch_bounds__(kThreadsTc, 1)
walker_tc_kernel(const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
                 const __grid_constant__ CUtensorMap tm_wh, const __grid_constant__ CUtensorMap tm_wl,
                 const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  SmemTail* tail = reinterpret_cast<SmemTail*>(base + kStages * kStageBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = blockIdx.x;       // cluster rank: the cluster spans grid.x
  const uint32_t csize = gridDim.x;
  const int strip = blockIdx.y;
  const int tile0 = static_cast<int>(rank) * p.tiles_per_cta;
  int ntiles = p.m_tiles - tile0;
  ntiles = ntiles < 0 ? 0 : (ntiles > p.tiles_per_cta ? p.tiles_per_cta : ntiles);
  const int row_base = tile0 * kRowsTile;
  const bool refresh = p.mode == kModeRefresh;

  // ---- set-up -------------------------------------------------------------
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&tail->full[s], 1);
      mbar_init(&tail->empty[s], 1);
    }
    for (int t = 0; t < kMaxTilesPerCta; ++t) mbar_init(&tail->tfull[t], 1);
    tail->timed_out = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    const uint32_t cols = p.tiles_per_cta <= 1 ? 128u : (p.tiles_per_cta == 2 ? 256u : 512u);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tail->tmem_base)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // Updates of the tracked slack since the last refresh.
  const float since = static_cast<float>(*p.step_ptr + static_cast<uint64_t>(p.j) -
                                         *p.refresh_step);
  for (int r = threadIdx.x; r < p.tiles_per_cta * kRowsTile; r += blockDim.x) {
    const bool in = r < ntiles * kRowsTile;
    tail->scale[r] = in ? p.row_scale[row_base + r] : 1.0f;
    tail->brow[r] = in ? p.bS[row_base + r] : 0.0f;
    tail->ks[r] = in ? p.rowk[4 * (row_base + r)] : 0.0f;
    tail->kg[r] = in ? p.rowk[4 * (row_base + r) + 1] : 0.0f;
    tail->jk[r] = in ? since * 5.9604645e-8f * fabsf(p.bS[row_base + r]) * 1.0001f : 0.0f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tail->tmem_base;
  volatile int* timed_out = &tail->timed_out;

  if (warp == 0) {
    // ---- TMA producer -------------------------------------------------------
    if (lane == 0) {
      int it = 0;
      for (int nt = 0; nt < ntiles; ++nt) {
        for (int kc = 0; kc < p.k_chunks; ++kc, ++it) {
          const int s = it % kStages;
          if (it >= kStages) mbar_wait(&tail->empty[s], ((it / kStages) - 1) & 1, timed_out, p.err);
          uint8_t* st = base + s * kStageBytes;
          mbar_expect_tx(&tail->full[s], kStageBytes);
          const int x = kc * kTcKChunk;
          const int yr = row_base + nt * kRowsTile;
          const int yw = strip * kWalkers;
          tma_load_2d(st, &tm_ah, &tail->full[s], x, yr);
          tma_load_2d(st + kOperandBytes, &tm_al, &tail->full[s], x, yr);
          tma_load_2d(st + 2 * kOperandBytes, &tm_wh, &tail->full[s], x, yw);
          tma_load_2d(st + 3 * kOperandBytes, &tm_wl, &tail->full[s], x, yw);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer: G = (Wh + Wl)(Ah + Al)^T, four FP16 products ------------
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(kWalkers, kRowsTile);
      int it = 0;
      for (int nt = 0; nt < ntiles; ++nt) {
        const uint32_t d_tmem = tmem + static_cast<uint32_t>(nt * kRowsTile);
        for (int kc = 0; kc < p.k_chunks; ++kc, ++it) {
          const int s = it % kStages;
          mbar_wait(&tail->full[s], (it / kStages) & 1, timed_out, p.err);
          tc_fence_after();
          const uint32_t st = smem_u32(base + s * kStageBytes);
          const uint32_t a_hi = st, a_lo = st + kOperandBytes;
          const uint32_t w_hi = st + 2 * kOperandBytes, w_lo = st + 3 * kOperandBytes;
          int ks_n = (p.kdim - kc * kTcKChunk) / kTcK;
          ks_n = ks_n > kTcKChunk / kTcK ? kTcKChunk / kTcK : ks_n;
          for (int ks = 0; ks < ks_n; ++ks) {
            const uint32_t off = static_cast<uint32_t>(ks * kTcK * 2);  // 32 bytes per K step
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_f16(d_tmem, sw128_desc(w_hi + off), sw128_desc(a_hi + off), idesc, acc);
            mma_f16(d_tmem, sw128_desc(w_hi + off), sw128_desc(a_lo + off), idesc, 1u);
            mma_f16(d_tmem, sw128_desc(w_lo + off), sw128_desc(a_hi + off), idesc, 1u);
            mma_f16(d_tmem, sw128_desc(w_lo + off), sw128_desc(a_lo + off), idesc, 1u);
          }
          mma_commit(&tail->empty[s]);
        }
        mma_commit(&tail->tfull[nt]);
      }
    }
    __syncwarp();
  } else if (refresh) {
    // ---- refresh epilogue: S = b - A X from tensor memory ----------------------
    const int e = warp - 2;
    const int q = warp & 3;
    const int cg = e >> 2;
    const int wl = q * 32 + lane;
    const int k = strip * kWalkers + wl;
    const float ws = p.wscale[k];
    float drift = 0.0f;
    // Bound on |tracked - recomputed| per unit Ks_i: the tracked slack's bound
    // (see TcParams) plus the recomputation's own (ws ||x_hat||_2).
    const float nxw =
        operand_norms<kEpiWarps * 32>(p.Dh, p.Xh, p.k_chunks * kTcKChunk, k, wl, cg, ws, tail->nrm)
            .nxw2;
    const float Eb = (k < p.z && p.check_drift)
                         ? (p.nx_ref[k] + p.theta_acc[k]) *
                                   (1.0f + since * (p.growth + 2.384185791e-7f)) * 1.0001f +
                               nxw
                         : INFINITY;
    bool off = false;
    for (int nt = 0; nt < ntiles; ++nt) {
      const int col = nt * kRowsTile + cg * 32;
      float* Sb = s_block(p, row_base + col, k);
      float sv[32];
      load_s32(p, Sb, sv);
      mbar_wait(&tail->tfull[nt], 0, timed_out, p.err, true);
      tc_fence_after();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float g[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(col + 16 * half), g);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int cc = 16 * half + c;
          const float sn = fmaf(-g[c], ws, tail->brow[col + cc]);
          // drift in the units of the constraint: |change| * row scale
          drift = fmaxf(drift, fabsf(sn - sv[cc]) * tail->scale[col + cc]);
          off = off || fabsf(sn - sv[cc]) > fmaf(tail->ks[col + cc], Eb, tail->jk[col + cc]);
          sv[cc] = sn;
        }
      }
      if (k < p.z) store_s32(p, Sb, sv);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) drift = fmaxf(drift, __shfl_xor_sync(0xffffffffu, drift, off));
    if (lane == 0 && drift > 0.0f) atomicMax(p.drift_key, f64_key(static_cast<double>(drift)));
    if (off && k < p.z) atomicOr(p.status, MHAR_ST_DRIFT);
  } else {
    // ---- chord epilogue, pass 1: partial (lambda_min, lambda_max) ---------------
    const int e = warp - 2;
    const int q = warp & 3;       // TMEM lane quarter this warp may access
    const int cg = e >> 2;        // which 32-column group of each tile
    const int wl = q * 32 + lane; // walker within the strip
    const int k = strip * kWalkers + wl;
    const float nd =
        operand_norms<kEpiWarps * 32>(p.Dh, p.Xh, p.k_chunks * kTcKChunk, k, wl, cg, 1.0f, tail->nrm)
            .nd2 +
        ((p.corrn != nullptr && k < p.z) ? 4194304.0f * p.corrn[k] : 0.0f);
    // Error bound of this walker's tracked slack, in units of Ks_i (see TcParams).
    // (The last factors cover the FP32 sums of theta_acc and E itself.)
    const float E = k < p.z ? (p.nx_ref[k] + p.theta_acc[k]) *
                                  (1.0f + since * (p.growth + 2.384185791e-7f)) * 1.0001f
                            : 0.0f;
    if (cg == 0) tail->nd[wl] = nd;
    ChordAcc acc;
    acc.init();
    float s_cur[32], s_nxt[32];
    if (ntiles > 0) load_s32(p, s_block(p, row_base + cg * 32, k), s_cur);
    for (int nt = 0; nt < ntiles; ++nt) {
      const int col = nt * kRowsTile + cg * 32;
      if (nt + 1 < ntiles) load_s32(p, s_block(p, row_base + col + kRowsTile, k), s_nxt);
      mbar_wait(&tail->tfull[nt], 0, timed_out, p.err, true);
      tc_fence_after();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float g[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(q * 32) << 16) +
                      static_cast<uint32_t>(col + 16 * half), g);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          // Both the slack and G are in units of the row's power-of-two
          // scale, so their ratio is the paper's lambda_i unchanged.  The
          // slack is lowered by its error bound and g pushed away from zero
          // by its own (the margins of tc_common.cuh's slack32 / scan32).
          const int r = col + 16 * half + c;
          const float gg = g[c];
          const float ss = clamp_slack(s_cur[16 * half + c] - fmaf(tail->ks[r], E, tail->jk[r]));
          const float sd = __int_as_float(__float_as_int(nd) | (__float_as_int(gg) & 0x80000000));
          acc.add(ss, fmaf(tail->kg[r], sd, gg));
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) s_cur[c] = s_nxt[c];
    }
    const float lo = acc.lo_all(), hi = acc.hi_all();
    tail->part_lo[cg][wl] = lo;
    tail->part_hi[cg][wl] = hi;
    named_bar<kEpiWarps * 32>();
    if (cg == 0) {
      tail->cta_lo[wl] = fmaxf(fmaxf(lo, tail->part_lo[1][wl]), fmaxf(tail->part_lo[2][wl], tail->part_lo[3][wl]));
      tail->cta_hi[wl] = fminf(fminf(hi, tail->part_hi[1][wl]), fminf(tail->part_hi[2][wl], tail->part_hi[3][wl]));
    }
  }

  // Partials of every CTA of the cluster are now in shared memory.
  cluster_sync_all();

  if (warp >= 2 && !refresh) {
    const int e = warp - 2;
    const int q = warp & 3;
    const int cg = e >> 2;
    const int wl = q * 32 + lane;
    const int k = strip * kWalkers + wl;
    if (cg == 0) {
      float L = -INFINITY, H = INFINITY;
      for (uint32_t r = 0; r < csize; ++r) {
        L = fmaxf(L, ld_dsmem_f32(&tail->cta_lo[wl], r));
        H = fminf(H, ld_dsmem_f32(&tail->cta_hi[wl], r));
      }
      float t = 0.0f;
      int flag = 0;
      if (k < p.z) {
        if (isinf(L) || isinf(H)) {
          flag = MHAR_ST_UNBOUNDED;
        } else if (L > H) {
          flag = MHAR_ST_STALL;
        } else {
          const uint64_t step = *p.step_ptr + static_cast<uint64_t>(p.j);
          const U4 w = philox_block(p.seed, step, p.walker0 + static_cast<uint32_t>(k), 0u,
                                    kStreamChord);
          const double u = open_unit_f64(w.x);
          t = static_cast<float>(static_cast<double>(L) +
                                 u * (static_cast<double>(H) - static_cast<double>(L)));
        }
        if (rank == 0) {
          p.lmin[k] = L;
          p.lmax[k] = H;
          p.theta[k] = t;
          p.theta_acc[k] += fabsf(t) * tail->nd[wl];
          if (flag) {
            atomicOr(p.status, flag);
            atomicAdd(&p.counters[flag == MHAR_ST_STALL ? 0 : 1], 1ull);
          }
        }
      }
      tail->theta[wl] = t;
    }
    named_bar<kEpiWarps * 32>();
    // ---- chord epilogue, pass 2: S -= G diag(theta) -----------------------------
    const float t = tail->theta[wl];
    if (__any_sync(0xffffffffu, t != 0.0f)) {
      float s_cur[32], s_nxt[32];
      if (ntiles > 0) load_s32(p, s_block(p, row_base + cg * 32, k), s_cur);
      for (int nt = 0; nt < ntiles; ++nt) {
        const int col = nt * kRowsTile + cg * 32;
        if (nt + 1 < ntiles) load_s32(p, s_block(p, row_base + col + kRowsTile, k), s_nxt);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float g[16];
          // tcgen05.ld is warp-collective: every lane joins, lanes with theta == 0 skip the update.
          tmem_ld16(tmem + (static_cast<uint32_t>(q * 32) << 16) +
                        static_cast<uint32_t>(col + 16 * half), g);
#pragma unroll
          for (int c = 0; c < 16; ++c) s_cur[16 * half + c] = fmaf(-t, g[c], s_cur[16 * half + c]);
        }
        if (t != 0.0f) store_s32(p, s_block(p, row_base + col, k), s_cur);
#pragma unroll
        for (int c = 0; c < 32; ++c) s_cur[c] = s_nxt[c];
      }
    }
    // ---- X += D diag(theta) on this CTA's slice of coordinates ---------------
    // One flat loop over (walker, coordinate) pairs so every thread keeps
    // several independent loads in flight.
    const int slice = (p.n + static_cast<int>(csize) - 1) / static_cast<int>(csize);
    const int i_begin = static_cast<int>(rank) * slice;
    const int len = max(0, min(p.n, i_begin + slice) - i_begin);
    const int total = kWalkers * len;
    const int k_pad = p.k_chunks * kTcKChunk;
#pragma unroll 4
    for (int idx = e * 32 + lane; idx < total; idx += kEpiWarps * 32) {
      const int w = idx / len;
      const int i = i_begin + (idx - w * len);
      const int kk = strip * kWalkers + w;
      const float tw = tail->theta[w];
      if (kk >= p.z || tw == 0.0f) continue;
      const size_t xr = static_cast<size_t>(kk) * p.n_ld + i;
      const size_t dr = static_cast<size_t>(kk) * k_pad + i;
      const float d = (__half2float(p.Dh[dr]) + __half2float(p.Dl[dr])) * p.sigma[i];
      df_axpy(p.Xhi[xr], p.Xlo[xr], tw, d);
      if (p.corr != nullptr) {
        // Exact null-space correction of the rounded direction (see projection).
        float dlt = 0.0f;
        for (int q2 = 0; q2 < p.mE; ++q2)
          dlt = fmaf(p.Q32[static_cast<size_t>(q2) * p.n_ld + i],
                     p.corr[static_cast<size_t>(kk) * p.mE + q2], dlt);
        p.Xlo[xr] = fmaf(-tw, dlt, p.Xlo[xr]);
      }
    }
  }

  // Peers may still be reading this CTA's partials; all tensor-memory reads
  // are complete once every thread is here.
  tc_fence_before();
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    const uint32_t cols = p.tiles_per_cta <= 1 ? 128u : (p.tiles_per_cta == 2 ? 256u : 512u);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols)
                 : "memory");
  }
}

// Refresh operands: each walker's point x = hi + lo scaled by a power of two
// 2^e (max |x_i| 2^-e in [0.5, 1)) and split into FP16 hi + lo.
__global__ void split_points_kernel(int z, int z_ld, int n, int n_ld, int k_pad, const float* Xhi,
                                    const float* Xlo, __half* Xh, __half* Xl, float* wscale,
                                    const float* sigma) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + warp;
  if (k >= z_ld) return;
  float mx = 0.0f;
  if (k < z)
    for (int i = lane; i < n; i += 32)
      mx = fmaxf(mx, fabsf(Xhi[static_cast<size_t>(k) * n_ld + i]) / sigma[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  int ex = 0;
  if (mx > 0.0f) frexpf(mx, &ex);
  const float inv = ldexpf(1.0f, -ex);
  if (lane == 0) wscale[k] = ldexpf(1.0f, ex);
  for (int i = lane; i < k_pad; i += 32) {
    float v = 0.0f;
    if (k < z && i < n)
      v = (Xhi[static_cast<size_t>(k) * n_ld + i] + Xlo[static_cast<size_t>(k) * n_ld + i]) * inv /
          sigma[i];
    const __half h = __float2half_rn(v);
    Xh[static_cast<size_t>(k) * k_pad + i] = h;
    Xl[static_cast<size_t>(k) * k_pad + i] = __float2half_rn(v - __half2float(h));
  }
}

TcParams make_params(const mhar_ctx* c, const TcPlan* plan, int mode, int j, bool check_drift) {
  TcParams p;
  p.mode = mode;
  p.check_drift = check_drift ? 1 : 0;
  p.row_scale = c->d.row_scale;
  p.bS = c->d.bS;
  p.wscale = c->d.wscale;
  p.S = c->d.S;
  p.Xhi = c->d.Xhi;
  p.Xlo = c->d.Xlo;
  p.rowk = c->d.rowk;
  p.Xh = c->d.Xh;
  p.corrn = c->d.corrn;
  p.nx_ref = c->d.nx_ref;
  p.theta_acc = c->d.theta_acc;
  p.refresh_step = c->d.refresh_step;
  p.growth = 1.0f / static_cast<float>(4 * mma_chain(c) + 4);
  p.Dh = c->d.Dh;
  p.Dl = c->d.Dl;
  p.sigma = c->d.sigma;
  p.Q32 = c->d.Q32;
  p.corr = c->d.corr;
  p.lmin = c->d.lmin;
  p.lmax = c->d.lmax;
  p.theta = c->d.theta;
  p.status = c->d.status;
  p.counters = c->d.counters;
  p.err = c->d.status + 1;
  p.drift_key = reinterpret_cast<unsigned long long*>(c->d.check) + 2;
  p.step_ptr = c->d.step;
  p.seed = c->opts.seed;
  p.j = j;
  p.walker0 = c->opts.walker0;
  p.m = c->m;
  p.n = c->n;
  p.n_ld = c->n_ld;
  p.z = c->z;
  p.z_ld = plan->strips * kWalkers;
  p.kdim = c->kdim;
  p.k_chunks = c->k_pad / kTcKChunk;
  p.tiles_per_cta = plan->tiles_per_cta;
  p.m_tiles = plan->m_tiles;
  p.mE = c->mE;
  return p;
}

cudaError_t launch_walker_tc(mhar_ctx* c, int mode, int j, bool check_drift = false) {
  const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
  const TcParams p = make_params(c, plan, mode, j, check_drift);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan->C, plan->strips, 1);
  cfg.blockDim = dim3(kThreadsTc, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan->C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (mode == kModeRefresh)
    return cudaLaunchKernelEx(&cfg, walker_tc_kernel, plan->ah, plan->al, plan->xh, plan->xl, p);
  return cudaLaunchKernelEx(&cfg, walker_tc_kernel, plan->ah, plan->al, plan->dh, plan->dl, p);
}

}  // namespace

int tc_plan_create(mhar_ctx* c) {
  auto* plan = new TcPlan();
  plan->m_tiles = c->m_pad / kRowsTile;
  plan->tiles_per_cta = plan->m_tiles < kMaxTilesPerCta ? plan->m_tiles : kMaxTilesPerCta;
  plan->C = (plan->m_tiles + plan->tiles_per_cta - 1) / plan->tiles_per_cta;
  const int z_ld = (c->z + kWalkers - 1) / kWalkers * kWalkers;
  plan->strips = z_ld / kWalkers;
  if (plan->C > 16 && c->opts.precision == MHAR_MIXED_F16X3) {
    delete plan;
    snprintf(c->err, sizeof(c->err),
             "tensor-core mode covers m <= 8192 inequality rows (got m=%d)", c->m);
    return MHAR_E_UNSUPPORTED;
  }
  if (!make_map(&plan->ah, c->d.Ah, c->k_pad, c->m_pad) ||
      !make_map(&plan->al, c->d.Al, c->k_pad, c->m_pad) ||
      !make_map(&plan->dh, c->d.Dh, c->k_pad, z_ld) || !make_map(&plan->dl, c->d.Dl, c->k_pad, z_ld) ||
      (c->d.Dh2 && (!make_map(&plan->dh2, c->d.Dh2, c->k_pad, z_ld) ||
                    !make_map(&plan->dl2, c->d.Dl2, c->k_pad, z_ld))) ||
      !make_map(&plan->xh, c->d.Xh, c->k_pad, z_ld) || !make_map(&plan->xl, c->d.Xl, c->k_pad, z_ld)) {
    delete plan;
    snprintf(c->err, sizeof(c->err), "cuTensorMapEncodeTiled failed");
    return MHAR_E_CUDA;
  }
  cudaError_t e = cudaFuncSetAttribute(walker_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmemBytes));
  if (e == cudaSuccess && plan->C > 8)
    e = cudaFuncSetAttribute(walker_tc_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    delete plan;
    snprintf(c->err, sizeof(c->err), "tensor-core kernel attributes: %s", cudaGetErrorString(e));
    return MHAR_E_CUDA;
  }
  c->tc = plan;
  return MHAR_OK;
}

void tc_plan_destroy(mhar_ctx* c) {
  delete static_cast<TcPlan*>(c->tc);
  c->tc = nullptr;
}

cudaError_t launch_chord_tc(mhar_ctx* c, int j) { return launch_walker_tc(c, kModeChord, j); }

cudaError_t launch_split_points(mhar_ctx* c) {
  const int z_ld = (c->z + kWalkers - 1) / kWalkers * kWalkers;
  split_points_kernel<<<(z_ld + 7) / 8, 256, 0, c->stream>>>(c->z, z_ld, c->n, c->n_ld, c->k_pad,
                                                          c->d.Xhi, c->d.Xlo, c->d.Xh, c->d.Xl,
                                                          c->d.wscale, c->d.sigma);
  return cudaGetLastError();
}

cudaError_t launch_refresh_tc(mhar_ctx* c, bool check_drift) {
  cudaError_t e = launch_split_points(c);
  if (e != cudaSuccess) return e;
  return launch_walker_tc(c, kModeRefresh, 0, check_drift);
}

int tc_plan_strips(const mhar_ctx* c) { return static_cast<const TcPlan*>(c->tc)->strips; }
int tc_plan_m_tiles(const mhar_ctx* c) { return static_cast<const TcPlan*>(c->tc)->m_tiles; }

}  // namespace mhar
