// kernels_ts.cu -- the recompute-slack walker step with the walker operands
// resident in tensor memory (MHAR_MIXED_RECOMPUTE mode, n <= 128).
//
// Same arithmetic as kernels_rc.cu (Lemma 4.2 on the tensor cores: P = X A^T
// and G = D A^T from FP16 pairs, three products each, FP32 accumulation;
// s = b - p; the chord; theta), organised for the case where one walker's
// operands fit in tensor memory:
//   * the four walker operands (D hi/lo, X hi/lo: 128 walkers x k_pad FP16,
//     stored interleaved by 8-element chunks so the loads are coalesced)
//     are written once into tensor memory (256 columns) and serve as the A
//     operand of every MMA (tcgen05.mma with A in TMEM), so shared memory
//     only feeds the rows of A -- half the operand bytes per MMA of the
//     shared-memory form, which is what limited that form;
//   * the rows of A stream in 128-row tiles (MMA N = 128) through eight
//     16 KB slots, the hi and lo halves of one K chunk behind one barrier, up
//     to two tiles ahead;
//   * the G and P accumulators of a tile (128 + 128 columns) take the other
//     256 TMEM columns.  A tile's MMAs run as two passes, P first, then G,
//     each with its own full / empty barrier pair: the epilogue copies P to
//     registers while the G pass runs and releases it, so the next tile's P
//     pass follows the G pass without draining the tensor pipe, and likewise
//     for G.  The epilogue's ratio work on a tile overlaps the next tile's
//     MMAs.
// Measured on GB300: an MMA whose operands both come from shared memory needs
// the SM's whole shared-memory bandwidth at full rate, so the loads of the
// other warps and the TMA writes slow it; with A in tensor memory it needs
// half.
//   * the walker-side inputs of each epilogue thread (its item of x hi / lo
//     and the direction pair) are copied into shared memory at kernel start
//     (cp.async), so the move after the chord reads no global memory; the
//     chord's uniform is drawn early, and the moved rows reach global memory
//     as whole lines through the same shared-memory stage.
// The cluster layout (C CTAs along the rows, 128 walkers per CTA), the pushed
// partial chords, the walker-side work (walker_tail.cuh) and the bounded
// waits are those of kernels_rc.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "mhar_device.cuh"
#include "mhar_internal.h"
#include "tc_common.cuh"
#include "walker_tail.cuh"

namespace mhar {
namespace {

using namespace tc;

constexpr int kTile = 128;                           // MMA N: rows of A per tile
constexpr int kSlotBytes = kTile * kTcKChunk * 2;    // 128 x 64 FP16 = 16 KB
constexpr int kSlots = 8;                            // two tiles of A (hi, lo) ahead
constexpr int kPairs = kSlots / 2;                   // hi + lo of one K chunk per barrier
constexpr int kEpiWarps = 16;
constexpr int kThreadsTs = (2 + kEpiWarps) * 32;
constexpr int kMaxCluster = 8;
constexpr uint32_t kOpCol = 256;                     // first TMEM column of the walker operands

struct TsParams {
  const float* rows;        // 3 m_pad: b_i / row_scale_i and the error bounds (row_block)
  const float* wscale;      // z_ld
  const __half* Xh;         // z_ld x k_pad (operands copied into TMEM at start)
  const __half* Xl;
  double* lmin;
  double* lmax;
  double* theta;
  int* status;
  unsigned long long* counters;
  int* err;
  const uint64_t* step_ptr;
  uint64_t seed;
  int j;
  uint32_t walker0;
  int z, z_ld, kdim, k_chunks, k_pad, tiles_per_cta, m_tiles;
  WalkerTail wt;            // walker-side work (walker_tail.cuh)
};

struct alignas(16) TsTail {
  uint64_t a_full[kSlots];
  uint64_t a_empty[kSlots];
  uint64_t p_full, p_empty;    // P accumulator: MMAs done / copied out
  uint64_t g_full, g_empty;    // G accumulator
  uint32_t tmem_base;
  int timed_out;
  float part_lo[4][kWalkers];
  float part_hi[4][kWalkers];
  float recv_lo[kMaxCluster][kWalkers];
  float recv_hi[kMaxCluster][kWalkers];
  float theta_s[kWalkers];
  double theta_u[kWalkers];           // the chord's uniform u (Philox stream 1), drawn early
  unsigned int red[kWalkers];
  float nrm[3][kWalkers];             // each walker's ||d_hat||_2, ||x_hat||_2, max |d_hat|
  float gs[kWalkers * kMaxPcRank];    // low-rank normals of a preconditioned draw
};

// The walker-side items staged at kernel start: one slot per epilogue thread.
constexpr size_t kStageBytes = static_cast<size_t>(kEpiWarps) * 32 * kTailStageBytes;
constexpr size_t kSmemTs =
    1024 + static_cast<size_t>(kSlots) * kSlotBytes + sizeof(TsTail) + kStageBytes;
static_assert(kSmemTs <= 232448, "recompute_ts_kernel exceeds the shared memory of a CTA");

__device__ __forceinline__ void st_dsmem(float* local, uint32_t rank, float v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(remote), "f"(v) : "memory");
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One 64-column K chunk of a tile's P pass (X hi, X lo times A hi; X hi
// times A lo) with KS K steps; pair use pu = p0 + kc holds A hi in half-slot
// 2 (pu % kPairs) and A lo in the next, behind one barrier (every wait, fence
// and commit on the issuing thread's path costs issue time).
template <int KS>
__device__ __forceinline__ void ts_p_chunk(TsTail* tail, uint8_t* base, int p0, int kc,
                                           uint32_t p_tmem, uint32_t op_xh, uint32_t op_xl,
                                           uint32_t idesc, volatile int* timed_out, int* err) {
  const int pu = p0 + kc, ps = pu % kPairs;
  const uint32_t ac0 = static_cast<uint32_t>(kc * 32);   // 2 FP16 per column
  mbar_wait(&tail->a_full[ps], (pu / kPairs) & 1, timed_out, err);
  tc_fence_after();
  // A slot's descriptor is built once; a K step of 16 FP16 adds 2 to it (32 bytes).
  const uint64_t bh = sw128_desc(smem_u32(base + (2 * ps) * kSlotBytes));
  const uint64_t bl = sw128_desc(smem_u32(base + (2 * ps + 1) * kSlotBytes));
  mma_ts_run2<KS>(p_tmem, op_xh + ac0, op_xl + ac0, bh, idesc, kc > 0 ? 1u : 0u);
  mma_ts_run1<KS>(p_tmem, op_xh + ac0, bl, idesc);
}

// The same chunk of the G pass (D hi, D lo times A hi; D hi times A lo); the
// pair was waited for by the P pass and is released here.
template <int KS>
__device__ __forceinline__ void ts_g_chunk(TsTail* tail, uint8_t* base, int p0, int kc,
                                           uint32_t g_tmem, uint32_t op_dh, uint32_t op_dl,
                                           uint32_t idesc) {
  const int pu = p0 + kc, ps = pu % kPairs;
  const uint32_t ac0 = static_cast<uint32_t>(kc * 32);
  const uint64_t bh = sw128_desc(smem_u32(base + (2 * ps) * kSlotBytes));
  const uint64_t bl = sw128_desc(smem_u32(base + (2 * ps + 1) * kSlotBytes));
  mma_ts_run2<KS>(g_tmem, op_dh + ac0, op_dl + ac0, bh, idesc, kc > 0 ? 1u : 0u);
  mma_ts_run1<KS>(g_tmem, op_dh + ac0, bl, idesc);
  mma_commit(&tail->a_empty[ps]);
}

// KCH: 64-column K chunks of A's rows (1 or 2: n <= 128); LAST: K steps (16
// FP16 each) in the last chunk, 1..4, the other chunk having 4.  A
// compile-time K structure makes each pass one straight run of MMAs (the
// issuing thread's stream between MMAs is the limiter).
template <int KCH, int LAST>
__global__ void __launch_bounds__(kThreadsTs, 1)
recompute_ts_kernel(const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
                    const TsParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  TsTail* tail = reinterpret_cast<TsTail*>(base + kSlots * kSlotBytes);
  uint8_t* stage = reinterpret_cast<uint8_t*>(tail + 1);   // 16-byte aligned

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TailItem tail_item;  // the epilogue threads' first tail item
  tail_item.valid = 0;
  const int csz_i = static_cast<int>(gridDim.x);
  const int share = (kWalkers + csz_i - 1) / csz_i;   // walkers of this CTA's walker-side work
  const int w_begin = static_cast<int>(blockIdx.x) * share;
  const int w_count = max(0, min(share, kWalkers - w_begin));
  const uint32_t rank = blockIdx.x;
  const int strip = blockIdx.y;
  const int tile0 = static_cast<int>(rank) * p.tiles_per_cta;
  int ntiles = p.m_tiles - tile0;
  ntiles = ntiles < 0 ? 0 : (ntiles > p.tiles_per_cta ? p.tiles_per_cta : ntiles);
  const int row_base = tile0 * kTile;

  if (threadIdx.x == 32) {
    prefetch_tmap(&tm_ah);
    prefetch_tmap(&tm_al);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) { mbar_init(&tail->a_full[s], 1); mbar_init(&tail->a_empty[s], 1); }
    mbar_init(&tail->p_full, 1);
    mbar_init(&tail->p_empty, kEpiWarps);
    mbar_init(&tail->g_full, 1);
    mbar_init(&tail->g_empty, kEpiWarps);
    tail->timed_out = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tail->tmem_base)), "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tail->tmem_base;
  volatile int* timed_out = &tail->timed_out;
  // Launched as a programmatic dependent of the previous iteration's kernel:
  // the set-up above overlaps its end; nothing it wrote is read before this.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint64_t step = *p.step_ptr + static_cast<uint64_t>(p.j);
  const int cur = static_cast<int>(step & 1ull);  // this iteration's direction pair

  // ---- walker operands into tensor memory: warp (quarter q, operand op) ------
  // writes its 32 walkers' row of operand op, 2 FP16 per 32-bit column.
  if (warp >= 2) {
    const int e = warp - 2;
    const int q = warp & 3;
    const int op = e >> 2;
    const int k = strip * kWalkers + q * 32 + lane;
    const __half* src = op == 0 ? p.wt.Dh[cur] : op == 1 ? p.wt.Dl[cur] : op == 2 ? p.Xh : p.Xl;
    // Operands are interleaved by 8-element chunks: chunk c of walker k is the
    // 16 bytes at (c z_ld + k) 16, so each load below is one contiguous
    // 512-byte line for the warp.
    const uint4* ops = reinterpret_cast<const uint4*>(src);
    const uint32_t col0 = kOpCol + static_cast<uint32_t>(op * 64);
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    uint32_t r0[32], r1[32];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint4 v = __ldg(ops + static_cast<size_t>(i) * p.z_ld + k);
      r0[4 * i] = v.x; r0[4 * i + 1] = v.y; r0[4 * i + 2] = v.z; r0[4 * i + 3] = v.w;
    }
    if (p.k_pad > 64) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint4 v = __ldg(ops + static_cast<size_t>(8 + i) * p.z_ld + k);
        r1[4 * i] = v.x; r1[4 * i + 1] = v.y; r1[4 * i + 2] = v.z; r1[4 * i + 3] = v.w;
      }
    }
    tmem_st32(tmem + lane_off + col0, r0);
    if (p.k_pad > 64) tmem_st32(tmem + lane_off + col0 + 32u, r1);
    tmem_st_wait();
    tc_fence_before();
    // Operands ready: release the MMA warp (the producer never waits on this).
    asm volatile("bar.arrive 2, %0;" ::"n"((kEpiWarps + 1) * 32) : "memory");
    if (op == 0 || op == 2) {
      // The 2-norm bound of the walker's direction (op 0) or scaled point
      // (op 2) from its FP16 hi row, for the chord's error margins.
      // Sums of squares in chunk order: the same bits as operand_norms in the
      // shared-memory-operand kernels.
      float ss = 0.0f, mx = 0.0f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint4 u = make_uint4(r0[4 * i], r0[4 * i + 1], r0[4 * i + 2], r0[4 * i + 3]);
        ss += sumsq8(u);
        mx = fmaxf(mx, absmax8(u));
      }
      if (p.k_pad > 64) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint4 u = make_uint4(r1[4 * i], r1[4 * i + 1], r1[4 * i + 2], r1[4 * i + 3]);
          ss += sumsq8(u);
          mx = fmaxf(mx, absmax8(u));
        }
      }
      tail->nrm[op >> 1][q * 32 + lane] = norm_bound(ss);
      if (op == 0) tail->nrm[2][q * 32 + lane] = mx * 1.00390625f;
    }
  }

  if (warp == 0) {
    // ---- TMA producer: A rows, 64-row tiles, hi and lo in separate slots ------
    if (lane == 0) {
      int pu = 0;
      for (int nt = 0; nt < ntiles; ++nt) {
        const int yr = row_base + nt * kTile;
#pragma unroll
        for (int kc = 0; kc < KCH; ++kc, ++pu) {
          const int s = pu % kPairs;
          if (pu >= kPairs) mbar_wait(&tail->a_empty[s], ((pu / kPairs) - 1) & 1, timed_out, p.err);
          mbar_expect_tx(&tail->a_full[s], 2 * kSlotBytes);
          tma_load_2d(base + (2 * s) * kSlotBytes, &tm_ah, &tail->a_full[s], kc * kTcKChunk, yr);
          tma_load_2d(base + (2 * s + 1) * kSlotBytes, &tm_al, &tail->a_full[s], kc * kTcKChunk, yr);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer ------------------------------------------------------------
    asm volatile("bar.sync 2, %0;" ::"n"((kEpiWarps + 1) * 32) : "memory");
    tc_fence_after();
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(kWalkers, kTile);
      const uint32_t op_dh = tmem + kOpCol, op_dl = op_dh + 64u, op_xh = op_dh + 128u,
                     op_xl = op_dh + 192u;
      const uint32_t g_tmem = tmem;
      const uint32_t p_tmem = tmem + 128u;
      int p0 = 0;    // first pair use of the tile
      for (int nt = 0; nt < ntiles; ++nt, p0 += KCH) {
        // P pass: X hi, X lo times A hi; X hi times A lo.  The accumulator is
        // free once the epilogue has copied the previous tile's P out.
        if (nt >= 1) mbar_wait(&tail->p_empty, (nt - 1) & 1, timed_out, p.err);
        tc_fence_after();
        if constexpr (KCH == 2)
          ts_p_chunk<4>(tail, base, p0, 0, p_tmem, op_xh, op_xl, idesc, timed_out, p.err);
        ts_p_chunk<LAST>(tail, base, p0, KCH - 1, p_tmem, op_xh, op_xl, idesc, timed_out, p.err);
        mma_commit(&tail->p_full);
        // G pass: D hi, D lo times A hi; D hi times A lo.  Each slot is
        // released after its last use here.
        if (nt >= 1) mbar_wait(&tail->g_empty, (nt - 1) & 1, timed_out, p.err);
        tc_fence_after();
        if constexpr (KCH == 2) ts_g_chunk<4>(tail, base, p0, 0, g_tmem, op_dh, op_dl, idesc);
        ts_g_chunk<LAST>(tail, base, p0, KCH - 1, g_tmem, op_dh, op_dl, idesc);
        mma_commit(&tail->g_full);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: s = b - p, ratios, per-walker partial chord ------------------
    // First, while the first row tiles are on their way: iteration s+1's
    // directions into the other pair (walker_tail.cuh, step 0).
    const int e = warp - 2;
    const int q = warp & 3;
    const int cg = e >> 2;              // 32-column group of each 128-column tile
    const int row0 = row_base + cg * 32;
    if (lane < 4 && ntiles > 0) prefetch_l1(row_block(p.rows, row0) + 32 * lane);
    // This thread's walker-side item, copied to shared memory in the background.
    walker_tail_stage<kEpiWarps * 32>(p.wt, cur, strip, p.z, w_begin, w_count,
                                      static_cast<int>(threadIdx.x) - 64,
                                      stage + (threadIdx.x - 64) * kTailStageBytes);
    if (cg == 0) {
      // The chord's uniform does not depend on the chord: draw it now.
      const int kk = strip * kWalkers + q * 32 + lane;
      const U4 w = philox_block(p.seed, step, p.walker0 + static_cast<uint32_t>(kk), 0u,
                                kStreamChord);
      tail->theta_u[q * 32 + lane] = open_unit_f64(w.x);
    }
    if (p.wt.draw)
      walker_draw_next<kEpiWarps * 32>(p.wt, cur, p.seed, step + 1ull, p.walker0, strip, p.z,
                                       w_begin, w_count, static_cast<int>(threadIdx.x) - 64,
                                       tail->gs);
    const int wl = q * 32 + lane;
    const int k = strip * kWalkers + wl;
    const float ws = p.wscale[k];
    // The operand norms of this thread's walker (written by the warps that
    // loaded the operands into tensor memory, before the draw above).
    named_bar<kEpiWarps * 32>();
    WalkerNorms wn;
    wn.nd2 = tail->nrm[0][wl];
    wn.nxw2 = ws * tail->nrm[1][wl];
    wn.ws = ws;
    wn.ndinf = tail->nrm[2][wl];
    if (k < p.z) add_correction(p.wt, k, wn);
    ChordAcc acc;
    acc.init();
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    const uint32_t gcol = tmem + lane_off + static_cast<uint32_t>(cg * 32);
    for (int nt = 0; nt < ntiles; ++nt) {
      // P first (its pass ends first), then G; each accumulator is released
      // as soon as it is in registers.
      if (lane < 4 && nt + 1 < ntiles) prefetch_l1(row_block(p.rows, row0 + (nt + 1) * kTile) + 32 * lane);
      float sv[32], gv[32];
      mbar_wait(&tail->p_full, nt & 1, timed_out, p.err);
      tc_fence_after();
      tmem_ld32(gcol + 128u, sv);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive(&tail->p_empty);
      // The slacks while the G pass finishes.
      float fx, fd;
      wn.pick(p.rows, row0 + nt * kTile, fx, fd);
      slack32(sv, p.rows, row0 + nt * kTile, ws, fx);
      mbar_wait(&tail->g_full, nt & 1, timed_out, p.err);
      tc_fence_after();
      tmem_ld32(gcol, gv);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive(&tail->g_empty);
      scan32(sv, gv, p.rows, row0 + nt * kTile, fd, acc);
    }
    const float lo = acc.lo_all(), hi = acc.hi_all();
    tail->part_lo[cg][wl] = lo;
    tail->part_hi[cg][wl] = hi;
    named_bar<kEpiWarps * 32>();
    if (cg == 0) {
      const float L = fmaxf(fmaxf(lo, tail->part_lo[1][wl]), fmaxf(tail->part_lo[2][wl], tail->part_lo[3][wl]));
      const float H = fminf(fminf(hi, tail->part_hi[1][wl]), fminf(tail->part_hi[2][wl], tail->part_hi[3][wl]));
      // Every CTA of the cluster gets every partial: each then knows the
      // strip's chords and theta without a second barrier.
      for (uint32_t r = 0; r < gridDim.x; ++r) {
        st_dsmem(&tail->recv_lo[rank][wl], r, L);
        st_dsmem(&tail->recv_hi[rank][wl], r, H);
      }
    }
  }

  // Every push is visible after this barrier; no remote access follows it.
  // Between its arrive and its wait the epilogue reads its first tail item
  // back from shared memory (staged at kernel start; it does not depend on
  // theta).
  tc_fence_before();
  cluster_arrive();
  if (warp >= 2)
    walker_tail_unstage<kEpiWarps * 32>(p.wt, strip, p.z, w_begin, w_count,
                                        static_cast<int>(threadIdx.x) - 64,
                                        stage + (threadIdx.x - 64) * kTailStageBytes, tail_item);
  cluster_wait();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }

  if (warp >= 2 && ((warp - 2) >> 2) == 0) {
    const int q = warp & 3;
    const int wl = q * 32 + lane;
    const int k = strip * kWalkers + wl;
    float L = -INFINITY, H = INFINITY;
    for (uint32_t r = 0; r < gridDim.x; ++r) {
      L = fmaxf(L, tail->recv_lo[r][wl]);
      H = fminf(H, tail->recv_hi[r][wl]);
    }
    if (k >= p.z) tail->theta_s[wl] = 0.0f;
    if (k < p.z) {
      float t = 0.0f;
      int flag = 0;
      if (isinf(L) || isinf(H)) {
        flag = MHAR_ST_UNBOUNDED;
      } else if (L > H) {
        flag = MHAR_ST_STALL;
      } else {
        const double u = tail->theta_u[wl];
        t = static_cast<float>(static_cast<double>(L) +
                               u * (static_cast<double>(H) - static_cast<double>(L)));
      }
      tail->theta_s[wl] = t;
      if (rank == 0) {
        p.lmin[k] = L;
        p.lmax[k] = H;
        p.theta[k] = t;
        if (flag) {
          atomicOr(p.status, flag);
          atomicAdd(&p.counters[flag == MHAR_ST_STALL ? 0 : 1], 1ull);
        }
      }
    }
  }
  if (warp >= 2) {
    named_bar<kEpiWarps * 32>();
    // The stage is free again (its items are in registers): route the moved
    // rows through it when they fit.
    const bool rows_fit = static_cast<size_t>(2 * w_count) * tail_row_stride(p.wt.n_ld) *
                              sizeof(float) <= kStageBytes;
    walker_tail<kEpiWarps * 32>(p.wt, cur, strip, p.z, w_begin, w_count, tail->theta_s,
                                tail->red, static_cast<int>(threadIdx.x) - 64, tail_item,
                                rows_fit ? reinterpret_cast<float*>(stage) : nullptr);
  }
}

struct TsShape {
  int C = 1;
  int tiles_per_cta = 1;
  int m_tiles = 1;
};

TsShape ts_shape(const mhar_ctx* c, const TcPlan* plan) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  TsShape s;
  s.m_tiles = c->m_pad / kTile;
  int C = sms / plan->strips;
  C = C < 1 ? 1 : (C > kMaxCluster ? kMaxCluster : C);
  C = C > s.m_tiles ? s.m_tiles : C;
  s.tiles_per_cta = (s.m_tiles + C - 1) / C;
  s.C = (s.m_tiles + s.tiles_per_cta - 1) / s.tiles_per_cta;
  return s;
}

// Instantiations by (chunks, last-chunk K steps): index 4 (KCH - 1) + LAST - 1.
using TsKernel = void (*)(CUtensorMap, CUtensorMap, TsParams);
constexpr TsKernel kTsKernels[8] = {
    recompute_ts_kernel<1, 1>, recompute_ts_kernel<1, 2>, recompute_ts_kernel<1, 3>,
    recompute_ts_kernel<1, 4>, recompute_ts_kernel<2, 1>, recompute_ts_kernel<2, 2>,
    recompute_ts_kernel<2, 3>, recompute_ts_kernel<2, 4>};

}  // namespace

bool ts_eligible(const mhar_ctx* c) { return c->k_pad <= 128; }

int ts_prepare(mhar_ctx* c) {
  auto* plan = static_cast<TcPlan*>(c->tc);
  if (!make_map_rows(&plan->ah64, c->d.Ah, c->k_pad, c->m_pad, kTile) ||
      !make_map_rows(&plan->al64, c->d.Al, c->k_pad, c->m_pad, kTile)) {
    snprintf(c->err, sizeof(c->err), "cuTensorMapEncodeTiled failed (64-row maps)");
    return MHAR_E_CUDA;
  }
  cudaError_t e = cudaSuccess;
  for (TsKernel k : kTsKernels)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(kSmemTs));
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "recompute (TMEM operand) kernel attributes: %s",
             cudaGetErrorString(e));
    cudaGetLastError();
    return MHAR_E_CUDA;
  }
  return MHAR_OK;
}

cudaError_t launch_recompute_ts(mhar_ctx* c, int j) {
  const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
  const TsShape s = ts_shape(c, plan);
  TsParams p;
  p.rows = c->d.rows;
  p.wscale = c->d.wscale;
  p.Xh = c->d.Xh;
  p.Xl = c->d.Xl;
  p.lmin = c->d.lmin;
  p.lmax = c->d.lmax;
  p.theta = c->d.theta;
  p.status = c->d.status;
  p.counters = c->d.counters;
  p.err = c->d.status + 1;
  p.step_ptr = c->d.step;
  p.seed = c->opts.seed;
  p.j = j;
  p.walker0 = c->opts.walker0;
  p.z = c->z;
  p.z_ld = plan->strips * kWalkers;
  p.kdim = c->kdim;
  p.k_chunks = c->k_pad / kTcKChunk;
  p.k_pad = c->k_pad;
  p.tiles_per_cta = s.tiles_per_cta;
  p.m_tiles = s.m_tiles;
  p.wt = make_walker_tail(c, 1, true);

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s.C, plan->strips, 1);
  cfg.blockDim = dim3(kThreadsTs, 1, 1);
  cfg.dynamicSmemBytes = kSmemTs;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = s.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // Programmatic dependent launch: the grid may be scheduled while the
  // previous kernel finishes; it waits (griddepcontrol.wait) before reading.
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const TsKernel k = kTsKernels[4 * (p.k_chunks - 1) + last_chunk_steps(p.kdim, p.k_chunks) - 1];
  return cudaLaunchKernelEx(&cfg, k, plan->ah64, plan->al64, p);
}

}  // namespace mhar
