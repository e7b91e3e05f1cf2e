// kernels_sk.cu -- the recompute-slack walker step (MHAR_MIXED_RECOMPUTE,
// shared-memory walker operands, n > 128) with a stream-K schedule.
//
// Same arithmetic as kernels_rc.cu (Lemma 4.2 on the tensor cores: P = X A^T
// and G = D A^T from FP16 pairs, three products each, FP32 accumulation;
// s = b - p; the chord; theta; the walker-side work of walker_tail.cuh).
// The schedule differs: when the walker strips (128 walkers each) are fewer
// than the SMs, clusters along the rows leave SMs idle (128 strips of 79 row
// tiles on 152 SMs keep 24 idle).  Here every SM runs one CTA, and the
// (strip, row tile) work is cut into equal contiguous ranges, one per CTA, so
// that a strip's rows may be split over several CTAs ("segments").  A CTA
// whose segment covers a whole strip finishes it alone; otherwise each
// segment writes its partial chords (lambda_min, lambda_max of its rows) to
// global memory and bumps the strip's counter, and the CTA that completes
// the strip combines the partials (max / min, exact, so the result does not
// depend on the cut) and draws theta.  The walker-side work (the moves and
// the FP16 pairs of the moved points, walker_tail.cuh) is a second launch,
// walker_update_kernel, over all strips at once: done by the CTA that
// completes a strip it held that CTA's tensor pipe for the whole of a
// latency-bound loop over the strip's points (~0.2 ms for 128 walkers of
// n = 1000, the memory system loaded by the other CTAs' operand streams),
// on the critical path of the launch.  Next iteration's directions are
// drawn early by the strip's segments, each for its share of the walkers.
// The pipelines (TMA producer, two MMA issuers, 16 epilogue warps, double-buffered
// accumulators) run across segment boundaries without re-initialisation.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mhar_device.cuh"
#include "mhar_internal.h"
#include "tc_common.cuh"
#include "walker_tail.cuh"

namespace mhar {
namespace {

using namespace tc;

constexpr int kWSlots = 2;                           // walker-operand slots (Dh, Dl, Xh, Xl chunk)
constexpr int kASlots = 4;                           // A half-slots (hi and lo of two chunks)
constexpr int kAPairs = kASlots / 2;                 // the batched kernel's A slots: hi + lo of a chunk
static_assert(kASlots >= 2 * kWSlots, "the stream-K kernel pairs A half-slots with walker slots");
constexpr int kWBytes = 4 * kOperandBytes;
constexpr int kABytes = kOperandBytes;
constexpr int kEpiWarps = 16;
// Both kernels issue their MMAs from two threads: warp 1 the G products, warp
// kPWarp the P products (a single thread issuing all of them keeps the tensor
// pipe near 80 cycles per 128 x 128 x 16 MMA on GB300, against 64 when two
// threads share the stream).
constexpr int kPWarp = 2 + kEpiWarps;
constexpr int kThreadsSk = (3 + kEpiWarps) * 32;

// One contiguous range of row tiles of one strip, processed by one CTA.
struct SkSeg {
  int strip;     // walker strip (128 walkers)
  int t0, t1;    // row tiles [t0, t1)
  int slot;      // index of this segment among the strip's segments
  int nseg;      // number of segments of the strip
};

struct SkParams {
  const float* rows;        // 3 m_pad: b_i / row_scale_i and the error bounds (row_block)
  const __half* Xh;         // z_ld x k_pad, row-major: FP16 hi of the scaled points
  const float* wscale;
  double* lmin;
  double* lmax;
  double* theta;
  int* status;
  unsigned long long* counters;
  int* err;
  const uint64_t* step_ptr;
  uint64_t seed;
  uint32_t walker0;
  int z, kdim, k_chunks, k_pad;
  const SkSeg* segs;        // all segments, grouped by CTA
  const int* seg_begin;     // CTA b owns segs[seg_begin[b] .. seg_begin[b + 1])
  float* partials;          // [strip][slot][2][128]: lambda_min, lambda_max of a segment
  int* arrivals;            // [strip]: segments done this iteration (reset by the last)
  int max_nseg;
  WalkerTail wt;
};

struct SkTail {
  uint64_t w_full[kWSlots];
  uint64_t w_empty[kWSlots];
  uint64_t a_full[kASlots];
  uint64_t a_empty[kASlots];
  uint64_t t_full[2];
  uint64_t t_empty[2];
  uint32_t tmem_base;
  int timed_out;
  int last;                       // this CTA completes the current strip
  float part_lo[4][kWalkers];
  float part_hi[4][kWalkers];
  float theta_s[kWalkers];
  unsigned int red[kWalkers];
  float nrm[3 * kWalkers];        // operand_norms
};

constexpr size_t kSmemSk = 1024 + static_cast<size_t>(kWSlots) * kWBytes +
                           static_cast<size_t>(kASlots) * kABytes + sizeof(SkTail);
static_assert(kSmemSk <= 232448, "recompute_sk_kernel exceeds the shared memory of a CTA");

__device__ __forceinline__ void mbar_arrive_sk(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// LAST: K steps in the operands' last 64-column chunk (1..4).
template <int LAST>
__global__ void __launch_bounds__(kThreadsSk, 1)
recompute_sk_kernel(const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
                    const __grid_constant__ CUtensorMap tm_dh, const __grid_constant__ CUtensorMap tm_dl,
                    const __grid_constant__ CUtensorMap tm_dh2, const __grid_constant__ CUtensorMap tm_dl2,
                    const __grid_constant__ CUtensorMap tm_xh, const __grid_constant__ CUtensorMap tm_xl,
                    const __grid_constant__ SkParams p, int j) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* wslot = base;
  uint8_t* aslot = base + kWSlots * kWBytes;
  SkTail* tail = reinterpret_cast<SkTail*>(aslot + kASlots * kABytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    // A walker slot is free once both MMA threads have committed it; a tile's
    // accumulators are full once both have.
    for (int s = 0; s < kWSlots; ++s) { mbar_init(&tail->w_full[s], 1); mbar_init(&tail->w_empty[s], 2); }
    for (int s = 0; s < kASlots; ++s) { mbar_init(&tail->a_full[s], 1); mbar_init(&tail->a_empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tail->t_full[b], 2); mbar_init(&tail->t_empty[b], kEpiWarps); }
    tail->timed_out = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&tm_ah);
    prefetch_tmap(&tm_al);
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
  // Programmatic dependent of the previous iteration's kernel: nothing it
  // wrote is read before this.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint64_t step = *p.step_ptr + static_cast<uint64_t>(j);
  const int cur = static_cast<int>(step & 1ull);
  const int sb = p.seg_begin[blockIdx.x], se = p.seg_begin[blockIdx.x + 1];

  if (warp == 0) {
    // ---- TMA producer: per (tile, k chunk) one slot holds the walker operand
    // chunk and A's hi / lo chunk, behind one barrier (every barrier wait,
    // fence and commit on the MMA thread's path costs issue time) ------------
    if (lane == 0) {
      int w_it = 0;
      for (int sg = sb; sg < se; ++sg) {
        const SkSeg seg = p.segs[sg];
        const int yw = seg.strip * kWalkers;
        for (int nt = seg.t0; nt < seg.t1; ++nt) {
          const int yr = nt * kRowsTile;
          for (int kc = 0; kc < p.k_chunks; ++kc, ++w_it) {
            const int x = kc * kTcKChunk;
            const int s = w_it % kWSlots;
            if (w_it >= kWSlots) mbar_wait(&tail->w_empty[s], ((w_it / kWSlots) - 1) & 1, timed_out, p.err);
            uint8_t* dst = wslot + s * kWBytes;
            mbar_expect_tx(&tail->w_full[s], kWBytes + 2 * kABytes);
            tma_load_2d(dst, cur ? &tm_dh2 : &tm_dh, &tail->w_full[s], x, yw);
            tma_load_2d(dst + kOperandBytes, cur ? &tm_dl2 : &tm_dl, &tail->w_full[s], x, yw);
            tma_load_2d(dst + 2 * kOperandBytes, &tm_xh, &tail->w_full[s], x, yw);
            tma_load_2d(dst + 3 * kOperandBytes, &tm_xl, &tail->w_full[s], x, yw);
            tma_load_2d(aslot + (2 * s) * kABytes, &tm_ah, &tail->w_full[s], x, yr);
            tma_load_2d(aslot + (2 * s + 1) * kABytes, &tm_al, &tail->w_full[s], x, yr);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1 || warp == kPWarp) {
    // ---- MMA issuers: warp 1 G = (Dh + Dl) A^T, warp kPWarp P = (Xh + Xl) A^T,
    // three products each, in the same order per accumulator as one issuer --
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(kWalkers, kRowsTile);
      const bool g_side = warp == 1;
      const uint32_t op0 = g_side ? 0u : 2u * kOperandBytes;   // Dh or Xh, then Dl or Xl
      int w_it = 0, gt = 0;
      for (int sg = sb; sg < se; ++sg) {
        const SkSeg seg = p.segs[sg];
        for (int nt = seg.t0; nt < seg.t1; ++nt, ++gt) {
          const int b = gt & 1;
          if (gt >= 2) mbar_wait(&tail->t_empty[b], ((gt >> 1) - 1) & 1, timed_out, p.err);
          tc_fence_after();
          const uint32_t d_tmem = tmem + static_cast<uint32_t>(b * 256) + (g_side ? 0u : 128u);
          // One K chunk: one wait, then the A hi run and the A lo run, then one
          // commit that frees the slot; KS (its K steps) is a compile-time
          // constant so that the MMA runs carry no branches.
          auto chunk = [&](int kc, auto ks_c) {
            constexpr int KS = decltype(ks_c)::value;
            const int ws = w_it % kWSlots;
            mbar_wait(&tail->w_full[ws], (w_it / kWSlots) & 1, timed_out, p.err);
            tc_fence_after();
            const uint32_t w0 = smem_u32(wslot + ws * kWBytes) + op0;
            const uint64_t o_h = sw128_desc(w0), o_l = sw128_desc(w0 + kOperandBytes);
            ss_run2<KS>(d_tmem, o_h, o_l, sw128_desc(smem_u32(aslot + (2 * ws) * kABytes)), idesc,
                        kc > 0 ? 1u : 0u);
            ss_run1<KS>(d_tmem, o_h, sw128_desc(smem_u32(aslot + (2 * ws + 1) * kABytes)), idesc);
            mma_commit(&tail->w_empty[ws]);
            ++w_it;
          };
          for (int kc = 0; kc + 1 < p.k_chunks; ++kc) chunk(kc, std::integral_constant<int, 4>{});
          chunk(p.k_chunks - 1, std::integral_constant<int, LAST>{});
          mma_commit(&tail->t_full[b]);
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: per segment, the partial chord of its rows; the CTA that
    // completes a strip also draws theta and does the walker-side work ----------
    const int tid = static_cast<int>(threadIdx.x) - 64;
    const int e = warp - 2;
    const int q = warp & 3;
    const int cg = e >> 2;
    const int wl = q * 32 + lane;
    int gt = 0;
    for (int sg = sb; sg < se; ++sg) {
      const SkSeg seg = p.segs[sg];
      const int strip = seg.strip;
      const int row0 = cg * 32;
      if (lane < 4 && seg.t1 > seg.t0) prefetch_l1(row_block(p.rows, row0 + seg.t0 * kRowsTile) + 32 * lane);
      // Iteration s+1's directions for this segment's share of the strip's
      // walkers, into the other pair (while the segment's first tile loads).
      if (p.wt.draw) {
        const int share = (kWalkers + seg.nseg - 1) / seg.nseg;
        const int wb = seg.slot * share;
        walker_draw_next<kEpiWarps * 32>(p.wt, cur, p.seed, step + 1ull, p.walker0, strip, p.z,
                                         wb, max(0, min(share, kWalkers - wb)), tid);
      }
      const int k = strip * kWalkers + wl;
      const float ws = p.wscale[k];
      WalkerNorms wn =
          operand_norms<kEpiWarps * 32>(p.wt.Dh[cur], p.Xh, p.k_pad, k, wl, cg, ws, tail->nrm);
      if (k < p.z) add_correction(p.wt, k, wn);
      ChordAcc acc;
      acc.init();
      for (int nt = seg.t0; nt < seg.t1; ++nt, ++gt) {
        const int b = gt & 1;
        if (lane < 4 && nt + 1 < seg.t1) prefetch_l1(row_block(p.rows, row0 + (nt + 1) * kRowsTile) + 32 * lane);
        mbar_wait(&tail->t_full[b], (gt >> 1) & 1, timed_out, p.err, true);
        tc_fence_after();
        const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
        const uint32_t gcol = tmem + lane_off + static_cast<uint32_t>(b * 256 + cg * 32);
        float sv[32], gv[32];
        tmem_ld32(gcol + 128u, sv);
        tmem_ld32(gcol, gv);
        // The accumulators of this buffer are in registers: let the MMA reuse it.
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_sk(&tail->t_empty[b]);
        float fx, fd;
        wn.pick(p.rows, row0 + nt * kRowsTile, fx, fd);
        slack32(sv, p.rows, row0 + nt * kRowsTile, ws, fx);
        scan32(sv, gv, p.rows, row0 + nt * kRowsTile, fd, acc);
      }
      const float lo = acc.lo_all(), hi = acc.hi_all();
      tail->part_lo[cg][wl] = lo;
      tail->part_hi[cg][wl] = hi;
      named_bar<kEpiWarps * 32>();
      float L = -INFINITY, H = INFINITY;
      if (cg == 0) {
        L = fmaxf(fmaxf(lo, tail->part_lo[1][wl]), fmaxf(tail->part_lo[2][wl], tail->part_lo[3][wl]));
        H = fminf(fminf(hi, tail->part_hi[1][wl]), fminf(tail->part_hi[2][wl], tail->part_hi[3][wl]));
      }
      if (seg.nseg > 1) {
        // Publish this segment's partial chords, then count the strip's
        // segments; the last one to arrive finishes the strip.
        float* mine = p.partials + (static_cast<size_t>(strip) * p.max_nseg + seg.slot) * 2 * kWalkers;
        if (cg == 0) {
          mine[wl] = L;
          mine[kWalkers + wl] = H;
          __threadfence();
        }
        named_bar<kEpiWarps * 32>();
        if (tid == 0) {
          const int before = atomicAdd(&p.arrivals[strip], 1);
          const int last = before == seg.nseg - 1;
          if (last) p.arrivals[strip] = 0;  // every segment of the strip has counted
          tail->last = last;
        }
        named_bar<kEpiWarps * 32>();
        if (!tail->last) continue;
        __threadfence();
        if (cg == 0) {
          L = -INFINITY;
          H = INFINITY;
          for (int g = 0; g < seg.nseg; ++g) {
            const float* part = p.partials + (static_cast<size_t>(strip) * p.max_nseg + g) * 2 * kWalkers;
            L = fmaxf(L, __ldcg(part + wl));
            H = fminf(H, __ldcg(part + kWalkers + wl));
          }
        }
      }
      // theta for the strip's walkers (Section 4.5), then the moves.
      if (cg == 0) {
        float t = 0.0f;
        if (k < p.z) {
          int flag = 0;
          if (isinf(L) || isinf(H)) {
            flag = MHAR_ST_UNBOUNDED;
          } else if (L > H) {
            flag = MHAR_ST_STALL;
          } else {
            const U4 w = philox_block(p.seed, step, p.walker0 + static_cast<uint32_t>(k), 0u,
                                      kStreamChord);
            const double u = open_unit_f64(w.x);
            t = static_cast<float>(static_cast<double>(L) +
                                   u * (static_cast<double>(H) - static_cast<double>(L)));
          }
          p.lmin[k] = L;
          p.lmax[k] = H;
          p.theta[k] = t;
          if (flag) {
            atomicOr(p.status, flag);
            atomicAdd(&p.counters[flag == MHAR_ST_STALL ? 0 : 1], 1ull);
          }
        }
      }
      // The moves and the next operands of the strip's walkers follow in
      // walker_update_kernel (one launch over all strips).
      named_bar<kEpiWarps * 32>();
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }
}

// ---- batched persistent launch --------------------------------------------------
// Many polytopes in one persistent launch: one CTA per SM pulls whole
// (problem, walker strip) units from a device queue (an atomic counter over
// the unit table, largest units first) until the table is exhausted, with
// the same pipelines as above carried across units.  The producer fetches
// the next unit as soon as it has issued the current one's loads and hands
// its index to the MMA issuer and the epilogue through a small ring in
// shared memory, so one unit's walker-side work (on the epilogue warps)
// overlaps the next unit's loads and first MMAs, and no CTA is launched or
// torn down between units.  A unit names its problem, whose tensor maps and
// parameters the CTA reads from a table in global memory, and whose K chunk
// count is taken at run time.  Walker operands of a body with n <= 128 (at
// most two K chunks) stay in shared memory for the whole unit; wider bodies
// stream them per tile like the single-body kernel.
struct alignas(128) BskProblem {
  CUtensorMap ah, al, dh, dl, dh2, dl2, xh, xl;
  const float* rows;
  const __half* Xh;
  const float* wscale;
  double* lmin;
  double* lmax;
  double* theta;
  int* status;
  unsigned long long* counters;
  int* err;
  const uint64_t* step_ptr;
  uint64_t seed;
  uint32_t walker0;
  int z, kdim, k_chunks, k_pad, m_tiles;
  WalkerTail wt;
};

struct BskUnit {
  int prob;      // problem
  int strip;     // walker strip within the problem
};

struct BskParams {
  const BskProblem* probs;
  const BskUnit* units;     // largest first
  int n_units;
  int* queue;               // two counters, used by alternate iterations
};

constexpr int kRing = 4;    // unit indices in flight between the producer and the consumers

struct BskRing {
  uint64_t full[kRing];
  uint64_t empty[kRing];    // both MMA threads and every epilogue warp release a slot
  int unit[kRing];
};

constexpr size_t kSmemBsk = kSmemSk + sizeof(BskRing);
static_assert(kSmemBsk <= 232448, "recompute_batch_sk_kernel exceeds the shared memory of a CTA");

__global__ void __launch_bounds__(kThreadsSk, 1)
recompute_batch_sk_kernel(const __grid_constant__ BskParams bp, int j) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* wslot = base;
  uint8_t* aslot = base + kWSlots * kWBytes;
  SkTail* tail = reinterpret_cast<SkTail*>(aslot + kASlots * kABytes);
  BskRing* ring = reinterpret_cast<BskRing*>(tail + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    // Two MMA threads (G and P): slots and accumulators are released, and
    // ring entries consumed, by both.
    for (int s = 0; s < kWSlots; ++s) { mbar_init(&tail->w_full[s], 1); mbar_init(&tail->w_empty[s], 2); }
    for (int s = 0; s < kASlots; ++s) { mbar_init(&tail->a_full[s], 1); mbar_init(&tail->a_empty[s], 2); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tail->t_full[b], 2); mbar_init(&tail->t_empty[b], kEpiWarps); }
    for (int r = 0; r < kRing; ++r) { mbar_init(&ring->full[r], 1); mbar_init(&ring->empty[r], 2 + kEpiWarps); }
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
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // The problems of a batch advance together.  Iteration s (problem 0's
  // count) takes units from counter s % 2 and clears the other for
  // iteration s + 1, which waits for this grid to complete before it reads it.
  int* err0 = bp.probs[0].err;
  const uint64_t bstep = *bp.probs[0].step_ptr + static_cast<uint64_t>(j);
  int* queue = bp.queue + (bstep & 1ull);
  if (blockIdx.x == 0 && threadIdx.x == 0) bp.queue[(bstep + 1ull) & 1ull] = 0;

  if (warp == 0) {
    // ---- TMA producer, and the unit fetch --------------------------------------------
    if (lane == 0) {
      int w_it = 0, a_it = 0;
      for (int r = 0;; ++r) {
        const int rs = r % kRing;
        if (r >= kRing) mbar_wait(&ring->empty[rs], ((r / kRing) - 1) & 1, timed_out, err0);
        int u = *timed_out ? bp.n_units : atomicAdd(queue, 1);
        u = u < bp.n_units ? u : -1;
        ring->unit[rs] = u;
        mbar_arrive_sk(&ring->full[rs]);
        if (u < 0) break;
        const BskUnit un = bp.units[u];
        const BskProblem& P = bp.probs[un.prob];
        const int kch = P.k_chunks;
        const bool resident = kch <= kWSlots;
        const int cur = static_cast<int>((*P.step_ptr + static_cast<uint64_t>(j)) & 1ull);
        const int yw = un.strip * kWalkers;
        auto load_w = [&](int kc) {
          const int s = w_it % kWSlots;
          if (w_it >= kWSlots) mbar_wait(&tail->w_empty[s], ((w_it / kWSlots) - 1) & 1, timed_out, P.err);
          uint8_t* dst = wslot + s * kWBytes;
          const int x = kc * kTcKChunk;
          mbar_expect_tx(&tail->w_full[s], kWBytes);
          tma_load_2d(dst, cur ? &P.dh2 : &P.dh, &tail->w_full[s], x, yw);
          tma_load_2d(dst + kOperandBytes, cur ? &P.dl2 : &P.dl, &tail->w_full[s], x, yw);
          tma_load_2d(dst + 2 * kOperandBytes, &P.xh, &tail->w_full[s], x, yw);
          tma_load_2d(dst + 3 * kOperandBytes, &P.xl, &tail->w_full[s], x, yw);
          ++w_it;
        };
        if (resident)
          for (int kc = 0; kc < kch; ++kc) load_w(kc);
        for (int nt = 0; nt < P.m_tiles; ++nt) {
          for (int kc = 0; kc < kch; ++kc, ++a_it) {
            if (!resident) load_w(kc);
            // A's hi and lo chunk in one pair of half-slots behind one barrier.
            const int s = a_it % kAPairs;
            if (a_it >= kAPairs) mbar_wait(&tail->a_empty[s], ((a_it / kAPairs) - 1) & 1, timed_out, P.err);
            mbar_expect_tx(&tail->a_full[s], 2 * kABytes);
            tma_load_2d(aslot + (2 * s) * kABytes, &P.ah, &tail->a_full[s], kc * kTcKChunk,
                        nt * kRowsTile);
            tma_load_2d(aslot + (2 * s + 1) * kABytes, &P.al, &tail->a_full[s], kc * kTcKChunk,
                        nt * kRowsTile);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1 || warp == kPWarp) {
    // ---- MMA issuers: warp 1 the G products, warp kPWarp the P products ---------------
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(kWalkers, kRowsTile);
      const bool g_side = warp == 1;
      const uint32_t op0 = g_side ? 0u : 2u * kOperandBytes;   // Dh or Xh, then Dl or Xl
      int w_it = 0, a_it = 0, gt = 0;
      for (int r = 0;; ++r) {
        const int rs = r % kRing;
        const bool ok = mbar_wait(&ring->full[rs], (r / kRing) & 1, timed_out, err0);
        const int u = ok ? ring->unit[rs] : -1;
        mbar_arrive_sk(&ring->empty[rs]);
        if (u < 0) break;
        const BskProblem& P = bp.probs[bp.units[u].prob];
        const int kch = P.k_chunks, kdim = P.kdim;
        const bool resident = kch <= kWSlots;
        const int wbase = w_it;
        for (int nt = 0; nt < P.m_tiles; ++nt, ++gt) {
          const int b = gt & 1;
          if (gt >= 2) mbar_wait(&tail->t_empty[b], ((gt >> 1) - 1) & 1, timed_out, P.err);
          tc_fence_after();
          const uint32_t d_tmem = tmem + static_cast<uint32_t>(b * 256) + (g_side ? 0u : 128u);
          for (int kc = 0; kc < kch; ++kc) {
            const int use = resident ? wbase + kc : w_it;
            const int ws = use % kWSlots;
            if (!resident || nt == 0)
              mbar_wait(&tail->w_full[ws], (use / kWSlots) & 1, timed_out, P.err);
            const uint32_t w0 = smem_u32(wslot + ws * kWBytes) + op0;
            const uint64_t o_h = sw128_desc(w0), o_l = sw128_desc(w0 + kOperandBytes);
            const int ks_n = min(kTcKChunk / kTcK, (kdim - kc * kTcKChunk) / kTcK);
            const int as = a_it % kAPairs;
            mbar_wait(&tail->a_full[as], (a_it / kAPairs) & 1, timed_out, P.err);
            tc_fence_after();
            ss_run2_n(ks_n, d_tmem, o_h, o_l, sw128_desc(smem_u32(aslot + (2 * as) * kABytes)), idesc,
                      kc > 0 ? 1u : 0u);
            ss_run1_n(ks_n, d_tmem, o_h, sw128_desc(smem_u32(aslot + (2 * as + 1) * kABytes)), idesc);
            mma_commit(&tail->a_empty[as]);
            ++a_it;
            if (!resident) {
              mma_commit(&tail->w_empty[ws]);
              ++w_it;
            }
          }
          mma_commit(&tail->t_full[b]);
        }
        if (resident) {
          // The unit's operand chunks are free once its last MMAs are done.
          for (int kc = 0; kc < kch; ++kc) mma_commit(&tail->w_empty[(wbase + kc) % kWSlots]);
          w_it = wbase + kch;
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue --------------------------------------------------------------------
    const int tid = static_cast<int>(threadIdx.x) - 64;
    const int e = warp - 2;
    const int q = warp & 3;
    const int cg = e >> 2;
    const int wl = q * 32 + lane;
    int gt = 0;
    for (int r = 0;; ++r) {
      const int rs = r % kRing;
      const bool ok = mbar_wait(&ring->full[rs], (r / kRing) & 1, timed_out, err0, true);
      const int u = ok ? ring->unit[rs] : -1;
      __syncwarp();
      if (lane == 0) mbar_arrive_sk(&ring->empty[rs]);
      if (u < 0) break;
      const BskUnit un = bp.units[u];
      const BskProblem& P = bp.probs[un.prob];
      const uint64_t step = *P.step_ptr + static_cast<uint64_t>(j);
      const int cur = static_cast<int>(step & 1ull);
      const int strip = un.strip;
      const int row0 = cg * 32;
      if (lane < 4) prefetch_l1(row_block(P.rows, row0) + 32 * lane);
      if (P.wt.draw)
        walker_draw_next<kEpiWarps * 32>(P.wt, cur, P.seed, step + 1ull, P.walker0, strip, P.z,
                                         0, kWalkers, tid);
      const int k = strip * kWalkers + wl;
      const float ws = P.wscale[k];
      WalkerNorms wn =
          operand_norms<kEpiWarps * 32>(P.wt.Dh[cur], P.Xh, P.k_pad, k, wl, cg, ws, tail->nrm);
      if (k < P.z) add_correction(P.wt, k, wn);
      ChordAcc acc;
      acc.init();
      for (int nt = 0; nt < P.m_tiles; ++nt, ++gt) {
        const int b = gt & 1;
        if (lane < 4 && nt + 1 < P.m_tiles) prefetch_l1(row_block(P.rows, row0 + (nt + 1) * kRowsTile) + 32 * lane);
        mbar_wait(&tail->t_full[b], (gt >> 1) & 1, timed_out, P.err, true);
        tc_fence_after();
        const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
        const uint32_t gcol = tmem + lane_off + static_cast<uint32_t>(b * 256 + cg * 32);
        float sv[32], gv[32];
        tmem_ld32(gcol + 128u, sv);
        tmem_ld32(gcol, gv);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_sk(&tail->t_empty[b]);
        float fx, fd;
        wn.pick(P.rows, row0 + nt * kRowsTile, fx, fd);
        slack32(sv, P.rows, row0 + nt * kRowsTile, ws, fx);
        scan32(sv, gv, P.rows, row0 + nt * kRowsTile, fd, acc);
      }
      const float lo = acc.lo_all(), hi = acc.hi_all();
      tail->part_lo[cg][wl] = lo;
      tail->part_hi[cg][wl] = hi;
      named_bar<kEpiWarps * 32>();
      if (cg == 0) {
        const float L = fmaxf(fmaxf(lo, tail->part_lo[1][wl]), fmaxf(tail->part_lo[2][wl], tail->part_lo[3][wl]));
        const float H = fminf(fminf(hi, tail->part_hi[1][wl]), fminf(tail->part_hi[2][wl], tail->part_hi[3][wl]));
        float t = 0.0f;
        if (k < P.z) {
          int flag = 0;
          if (isinf(L) || isinf(H)) {
            flag = MHAR_ST_UNBOUNDED;
          } else if (L > H) {
            flag = MHAR_ST_STALL;
          } else {
            const U4 w = philox_block(P.seed, step, P.walker0 + static_cast<uint32_t>(k), 0u,
                                      kStreamChord);
            const double uu = open_unit_f64(w.x);
            t = static_cast<float>(static_cast<double>(L) +
                                   uu * (static_cast<double>(H) - static_cast<double>(L)));
          }
          P.lmin[k] = L;
          P.lmax[k] = H;
          P.theta[k] = t;
          if (flag) {
            atomicOr(P.status, flag);
            atomicAdd(&P.counters[flag == MHAR_ST_STALL ? 0 : 1], 1ull);
          }
        }
      }
      // The moves follow in walker_update_batch_kernel.
      named_bar<kEpiWarps * 32>();
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }
}

}  // namespace

// ---- the walker-side work of the stream-K kernel's iteration -----------------------
// Every item -- a walker's 8-coordinate chunk -- takes the arithmetic of
// walker_tail.cuh, so that the stream-K schedule agrees bit for bit with the
// kernels that do the walker-side work themselves: (1) the move
// x += theta (d - Q^T c') in double-float and the walker's largest scaled
// coordinate, (2) the FP16 pair of the scaled point.
// walker_update_kernel (one context) and walker_update_batch_kernel (a table
// of (problem, first walker, W) units): a CTA of kUpdThreads threads takes W
// consecutive walkers, as many as 12 KB of shared memory holds (at most
// kUpdMaxW): small CTAs, sixteen to an SM, so that one CTA's copies overlap the
// others' arithmetic.  One thread brings the walkers' rows (x hi, x lo: n_ld
// floats each; the direction pair: k_pad halves each) into shared memory with
// bulk copies behind one mbarrier, so that all of a CTA's loads are in flight
// at once; the moved rows and the pair are stored from shared memory with
// coalesced stores (a warp on consecutive chunks of one walker).  Rows too
// long to stage (over kUpdSmemMax a walker) take walker_tail itself,
// kUpdWalkers walkers a CTA.
constexpr int kUpdThreads = 64;
constexpr int kUpdMaxW = 8;
constexpr int kUpdWalkers = 8;
static_assert(kWalkers % kUpdWalkers == 0, "update CTAs tile a walker strip");

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Walkers k0 .. k0 + W - 1 staged in shared memory (W >= 1).
__device__ __forceinline__ void update_staged(const WalkerTail& wt, const double* __restrict__ theta,
                                              const uint64_t* step_ptr, int j, int z, int k0,
                                              int W, int* err) {
  using namespace tail_detail;
  extern __shared__ __align__(128) uint8_t upd_smem[];
  __shared__ uint64_t bar;
  __shared__ float theta_s[kUpdMaxW];
  __shared__ unsigned int red[kUpdMaxW];
  __shared__ int timed_out;
  const int n = wt.n, n_ld = wt.n_ld, k_pad = wt.k_pad;
  float* xs = reinterpret_cast<float*>(upd_smem);                       // [W][hi, lo][n_ld]
  __half* ds = reinterpret_cast<__half*>(xs + static_cast<size_t>(2 * W) * n_ld);  // [W][hi, lo][k_pad]
  const int wn = min(W, z - k0);
  const int tid = static_cast<int>(threadIdx.x);
  const int cur = static_cast<int>((*step_ptr + static_cast<uint64_t>(j)) & 1ull);
  if (tid == 0) {
    timed_out = 0;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < wn) {
    theta_s[tid] = static_cast<float>(theta[k0 + tid]);
    red[tid] = 0u;
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t xb = static_cast<uint32_t>(n_ld) * 4u, db = static_cast<uint32_t>(k_pad) * 2u;
    mbar_expect_tx(&bar, static_cast<uint32_t>(wn) * 2u * (xb + db));
    for (int w = 0; w < wn; ++w) {
      const size_t k = static_cast<size_t>(k0 + w);
      bulk_g2s(xs + static_cast<size_t>(2 * w) * n_ld, wt.Xhi + k * n_ld, xb, &bar);
      bulk_g2s(xs + static_cast<size_t>(2 * w + 1) * n_ld, wt.Xlo + k * n_ld, xb, &bar);
      bulk_g2s(ds + static_cast<size_t>(2 * w) * k_pad, wt.Dh[cur] + k * k_pad, db, &bar);
      bulk_g2s(ds + static_cast<size_t>(2 * w + 1) * k_pad, wt.Dl[cur] + k * k_pad, db, &bar);
    }
  }
  if (!mbar_wait(&bar, 0, &timed_out, err, true)) {
    // The copies are still landing in this CTA's shared memory: wait for
    // them once more (bounded) before leaving.
    timed_out = 0;
    mbar_wait(&bar, 0, &timed_out, err, true);
    return;
  }
  const int chunks = (n + 7) >> 3;
  const int items = wn * chunks;
  // Items it = wo chunks + c, tid + kUpdThreads apart: (wo, c) advanced by a
  // fixed (step_w, step_c) instead of a division per item.
  const int step_w = kUpdThreads / chunks, step_c = kUpdThreads - step_w * chunks;
  const int wo0 = tid / chunks, c0 = tid - wo0 * chunks;
  const bool unit = wt.unit_sigma != 0;
  // (1) the moves, in shared memory, and each walker's largest scaled coordinate.
  for (int it = tid, wo = wo0, c = c0; it < items; it += kUpdThreads) {
    const int k = k0 + wo, i0 = 8 * c;
    const bool last = i0 + 8 > n;   // the one chunk that reaches past n
    float* xh = xs + static_cast<size_t>(2 * wo) * n_ld + i0;
    float* xl = xh + n_ld;
    const float th = theta_s[wo];
    float hi[8], lo[8], sg[8];
    ld8(xh, hi);
    ld8(xl, lo);
    if (!unit) ld8(wt.sigma + i0, sg);
    if (th != 0.0f) {
      float dh[8], dl[8], d[8];
      ld8h(ds + static_cast<size_t>(2 * wo) * k_pad + i0, dh);
      ld8h(ds + static_cast<size_t>(2 * wo + 1) * k_pad + i0, dl);
#pragma unroll
      for (int e = 0; e < 8; ++e) d[e] = unit ? dh[e] + dl[e] : (dh[e] + dl[e]) * sg[e];
      if (last) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (i0 + e >= n) d[e] = 0.0f;
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) df_axpy(hi[e], lo[e], th, d[e]);
      if (wt.corr != nullptr) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int i = i0 + e;
          if (i >= n) continue;
          float dlt = 0.0f;
          for (int q = 0; q < wt.mE; ++q)
            dlt = fmaf(wt.Q32[static_cast<size_t>(q) * n_ld + i],
                       wt.corr[static_cast<size_t>(k) * wt.mE + q], dlt);
          lo[e] = fmaf(-th, dlt, lo[e]);
        }
      }
      st8(xh, hi);
      st8(xl, lo);
    }
    float mx = 0.0f;
    if (unit) {
#pragma unroll
      for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fabsf(hi[e]));   // x = 0 past n
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (!last || i0 + e < n) mx = fmaxf(mx, fabsf(hi[e]) * pow2_recip(sg[e]));
    }
    atomicMax(red + wo, __float_as_uint(mx));  // non-negative floats order as their bits
    c += step_c;
    wo += step_w;
    if (c >= chunks) {
      c -= chunks;
      ++wo;
    }
  }
  __syncthreads();
  // Each walker's power-of-two scale, once.
  __shared__ float inv_s[kUpdMaxW];
  if (tid < wn) {
    const float mx = __uint_as_float(red[tid]);
    int ex = 0;
    if (mx > 0.0f) frexpf(mx, &ex);
    inv_s[tid] = ldexpf(1.0f, -ex);
    wt.wscale[k0 + tid] = ldexpf(1.0f, ex);
  }
  __syncthreads();
  // (2) the moved rows back, and the FP16 pair of the scaled point.
  for (int it = tid, wo = wo0, c = c0; it < items; it += kUpdThreads) {
    const int k = k0 + wo, i0 = 8 * c;
    const float* xh = xs + static_cast<size_t>(2 * wo) * n_ld + i0;
    float hi[8], lo[8], v[8];
    ld8(xh, hi);
    ld8(xh + n_ld, lo);
    const size_t xr = static_cast<size_t>(k) * n_ld + i0;
    st8(wt.Xhi + xr, hi);
    st8(wt.Xlo + xr, lo);
    const float inv = inv_s[wo];
    // x = 0 and sigma = 1 past n: no per-coordinate branch.
    if (unit) {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (hi[e] + lo[e]) * inv;
    } else {
      float sg[8];
      ld8(wt.sigma + i0, sg);
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (hi[e] + lo[e]) * inv * pow2_recip(sg[e]);
    }
    const size_t o = static_cast<size_t>(k) * k_pad + i0;   // row-major operands
    if (split_store8(v, wt.Xh + o, wt.Xl + o)) atomicOr(wt.status, MHAR_ST_NONFINITE);
    c += step_c;
    wo += step_w;
    if (c >= chunks) {
      c -= chunks;
      ++wo;
    }
  }
}

// Walkers k0 .. k0 + kUpdWalkers - 1 (k0 a multiple of kUpdWalkers) by
// walker_tail itself, for rows too long to stage.
__device__ __forceinline__ void update_direct(const WalkerTail& wt, const double* __restrict__ theta,
                                              const uint64_t* step_ptr, int j, int z, int k0) {
  __shared__ float theta_d[kWalkers];
  __shared__ unsigned int red_d[kUpdWalkers];
  const int strip = k0 / kWalkers, w_begin = k0 % kWalkers;
  const int cur = static_cast<int>((*step_ptr + static_cast<uint64_t>(j)) & 1ull);
  if (threadIdx.x < kUpdWalkers) {
    const int k = k0 + static_cast<int>(threadIdx.x);
    theta_d[w_begin + threadIdx.x] = k < z ? static_cast<float>(theta[k]) : 0.0f;
  }
  __syncthreads();
  TailItem none;
  none.valid = 0;
  walker_tail<kUpdThreads>(wt, cur, strip, z, w_begin, kUpdWalkers, theta_d, red_d,
                           static_cast<int>(threadIdx.x), none);
}

// One context: W walkers a CTA (W = 0: the direct form, kUpdWalkers a CTA).
__global__ void __launch_bounds__(kUpdThreads, 16)
walker_update_kernel(const WalkerTail wt, const double* __restrict__ theta,
                     const uint64_t* step_ptr, int j, int z, int W, int* err) {
  // Programmatic dependent of the chord kernel: theta and the points are
  // read after it.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (W > 0)
    update_staged(wt, theta, step_ptr, j, z, static_cast<int>(blockIdx.x) * W, W, err);
  else
    update_direct(wt, theta, step_ptr, j, z, static_cast<int>(blockIdx.x) * kUpdWalkers);
}

// Many contexts (a batch): a table of (problem, first walker, W) units.
struct UpdProblem {
  WalkerTail wt;
  const double* theta;
  const uint64_t* step_ptr;
  int* err;
  int z;
};
struct UpdUnit {
  int prob, k0, w;
};

__global__ void __launch_bounds__(kUpdThreads, 16)
walker_update_batch_kernel(const UpdProblem* __restrict__ probs, const UpdUnit* __restrict__ units,
                           int j) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const UpdUnit u = units[blockIdx.x];
  const UpdProblem& P = probs[u.prob];
  if (u.w > 0)
    update_staged(P.wt, P.theta, P.step_ptr, j, P.z, u.k0, u.w, P.err);
  else
    update_direct(P.wt, P.theta, P.step_ptr, j, P.z, u.k0);
}

// Walkers a walker_update_kernel CTA stages (0: the rows do not fit; the
// direct kernel runs), and its dynamic shared memory.
// The kernels' dynamic shared memory limit is set once to the largest any
// context asks for (kUpdSmemMax): it is a per-function attribute, and
// contexts of different sizes launch the same function.
constexpr int kUpdSmemMax = 200 << 10;
int update_walkers(int n_ld, int k_pad, size_t* smem) {
  const size_t per = 8ull * n_ld + 4ull * k_pad;
  const size_t budget = 12u << 10;
  int w = static_cast<int>(budget / per);
  if (w < 1) w = per <= static_cast<size_t>(kUpdSmemMax) ? 1 : 0;
  if (w > kUpdMaxW) w = kUpdMaxW;
  *smem = static_cast<size_t>(w) * per;
  return w;
}

// ---- host side -------------------------------------------------------------------
struct SkPlan {
  SkSeg* segs = nullptr;
  int* seg_begin = nullptr;
  float* partials = nullptr;
  int* arrivals = nullptr;
  int grid = 0;
  int max_nseg = 1;
  int upd_w = 0;          // walkers per walker_update_kernel CTA (0: direct kernel)
  size_t upd_smem = 0;
};

int sk_prepare(mhar_ctx* c) {
  const int strips = tc_plan_strips(c);
  const int m_tiles = tc_plan_m_tiles(c);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const long long T = static_cast<long long>(strips) * m_tiles;
  const int G = static_cast<int>(std::min<long long>(sms, T));
  std::vector<SkSeg> segs;
  std::vector<int> begin(G + 1, 0);
  std::vector<int> nseg(strips, 0);
  for (int b = 0; b < G; ++b) {
    begin[b] = static_cast<int>(segs.size());
    long long u0 = b * T / G;
    const long long u1 = (b + 1) * T / G;
    while (u0 < u1) {
      SkSeg s;
      s.strip = static_cast<int>(u0 / m_tiles);
      s.t0 = static_cast<int>(u0 % m_tiles);
      s.t1 = static_cast<int>(std::min<long long>(m_tiles, s.t0 + (u1 - u0)));
      s.slot = nseg[s.strip]++;
      s.nseg = 0;
      segs.push_back(s);
      u0 += s.t1 - s.t0;
    }
  }
  begin[G] = static_cast<int>(segs.size());
  int max_nseg = 1;
  for (SkSeg& s : segs) {
    s.nseg = nseg[s.strip];
    max_nseg = std::max(max_nseg, s.nseg);
  }
  SkPlan* plan = new SkPlan();
  plan->grid = G;
  plan->max_nseg = max_nseg;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&plan->segs), sizeof(SkSeg) * segs.size());
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&plan->seg_begin), sizeof(int) * begin.size());
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&plan->partials),
                   sizeof(float) * static_cast<size_t>(strips) * max_nseg * 2 * kWalkers);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&plan->arrivals), sizeof(int) * strips);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->segs, segs.data(), sizeof(SkSeg) * segs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->seg_begin, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(plan->arrivals, 0, sizeof(int) * strips);
  for (auto* k : {recompute_sk_kernel<1>, recompute_sk_kernel<2>, recompute_sk_kernel<3>,
                  recompute_sk_kernel<4>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(kSmemSk));
  plan->upd_w = update_walkers(c->n_ld, c->k_pad, &plan->upd_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(walker_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kUpdSmemMax);
  c->sk = plan;
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "stream-K schedule: %s", cudaGetErrorString(e));
    cudaGetLastError();
    return MHAR_E_CUDA;
  }
  return MHAR_OK;
}

void sk_destroy(mhar_ctx* c) {
  SkPlan* plan = static_cast<SkPlan*>(c->sk);
  if (!plan) return;
  void* ptrs[] = {plan->segs, plan->seg_begin, plan->partials, plan->arrivals};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete plan;
  c->sk = nullptr;
}

cudaError_t launch_recompute_sk(mhar_ctx* c, int j) {
  const TcPlan* tp = static_cast<const TcPlan*>(c->tc);
  const SkPlan* plan = static_cast<const SkPlan*>(c->sk);
  SkParams p;
  p.rows = c->d.rows;
  p.Xh = c->d.Xh;
  p.k_pad = c->k_pad;
  p.wscale = c->d.wscale;
  p.lmin = c->d.lmin;
  p.lmax = c->d.lmax;
  p.theta = c->d.theta;
  p.status = c->d.status;
  p.counters = c->d.counters;
  p.err = c->d.status + 1;
  p.step_ptr = c->d.step;
  p.seed = c->opts.seed;
  p.walker0 = c->opts.walker0;
  p.z = c->z;
  p.kdim = c->kdim;
  p.k_chunks = c->k_pad / kTcKChunk;
  p.segs = plan->segs;
  p.seg_begin = plan->seg_begin;
  p.partials = plan->partials;
  p.arrivals = plan->arrivals;
  p.max_nseg = plan->max_nseg;
  p.wt = make_walker_tail(c, 0);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan->grid, 1, 1);
  cfg.blockDim = dim3(kThreadsSk, 1, 1);
  cfg.dynamicSmemBytes = kSmemSk;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto* kernel = recompute_sk_kernel<4>;
  switch (last_chunk_steps(p.kdim, p.k_chunks)) {
    case 1: kernel = recompute_sk_kernel<1>; break;
    case 2: kernel = recompute_sk_kernel<2>; break;
    case 3: kernel = recompute_sk_kernel<3>; break;
    default: break;
  }
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, tp->ah, tp->al, tp->dh, tp->dl, tp->dh2,
                                     tp->dl2, tp->xh, tp->xl, p, j);
  if (e != cudaSuccess) return e;
  // The walker-side work, a programmatic dependent of the chord kernel.
  cudaLaunchConfig_t ucfg = {};
  ucfg.blockDim = dim3(kUpdThreads, 1, 1);
  ucfg.stream = c->stream;
  ucfg.attrs = attr;
  ucfg.numAttrs = 1;
  const int per = plan->upd_w > 0 ? plan->upd_w : kUpdWalkers;
  ucfg.gridDim = dim3(static_cast<unsigned>((c->z + per - 1) / per), 1, 1);
  ucfg.dynamicSmemBytes = plan->upd_smem;
  return cudaLaunchKernelEx(&ucfg, walker_update_kernel, p.wt, static_cast<const double*>(p.theta),
                            static_cast<const uint64_t*>(p.step_ptr), j, p.z, plan->upd_w, p.err);
}

// ---- the batched walker update: host side -----------------------------------------
struct UpdPlan {
  UpdProblem* probs = nullptr;
  UpdUnit* units = nullptr;
  int n_units = 0;
  size_t smem = 0;
};

int update_plan_build(mhar_ctx* const* ctx, int count, void** plan_out, char* err, size_t err_len) {
  *plan_out = nullptr;
  std::vector<UpdProblem> probs(count);
  std::vector<UpdUnit> units;
  size_t smem = 0;
  for (int q = 0; q < count; ++q) {
    mhar_ctx* c = ctx[q];
    UpdProblem& P = probs[q];
    std::memset(&P, 0, sizeof(P));
    P.wt = make_walker_tail(c, 0);
    P.theta = c->d.theta;
    P.step_ptr = c->d.step;
    P.err = c->d.status + 1;
    P.z = c->z;
    size_t sm = 0;
    const int w = update_walkers(c->n_ld, c->k_pad, &sm);
    smem = std::max(smem, sm);
    const int per = w > 0 ? w : kUpdWalkers;
    for (int k0 = 0; k0 < c->z; k0 += per) units.push_back({q, k0, w});
  }
  UpdPlan* plan = new UpdPlan();
  plan->n_units = static_cast<int>(units.size());
  plan->smem = smem;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&plan->probs), sizeof(UpdProblem) * probs.size());
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&plan->units), sizeof(UpdUnit) * units.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->probs, probs.data(), sizeof(UpdProblem) * probs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->units, units.data(), sizeof(UpdUnit) * units.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(walker_update_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kUpdSmemMax);
  if (e != cudaSuccess) {
    snprintf(err, err_len, "walker update table: %s", cudaGetErrorString(e));
    cudaGetLastError();
    update_plan_destroy(plan);
    return MHAR_E_CUDA;
  }
  *plan_out = plan;
  return MHAR_OK;
}

void update_plan_destroy(void* plan_v) {
  UpdPlan* plan = static_cast<UpdPlan*>(plan_v);
  if (!plan) return;
  if (plan->probs) cudaFree(plan->probs);
  if (plan->units) cudaFree(plan->units);
  delete plan;
}

cudaError_t launch_update_plan(const void* plan_v, int j, cudaStream_t stream) {
  const UpdPlan* plan = static_cast<const UpdPlan*>(plan_v);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(plan->n_units), 1, 1);
  cfg.blockDim = dim3(kUpdThreads, 1, 1);
  cfg.dynamicSmemBytes = plan->smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, walker_update_batch_kernel,
                            static_cast<const UpdProblem*>(plan->probs),
                            static_cast<const UpdUnit*>(plan->units), j);
}

// ---- batched persistent launch: host side ---------------------------------------
struct BatchSkPlan {
  BskProblem* probs = nullptr;
  BskUnit* units = nullptr;
  int* queue = nullptr;
  int n_units = 0;
  int grid = 0;
};

void batch_sk_destroy(void* plan_v) {
  BatchSkPlan* plan = static_cast<BatchSkPlan*>(plan_v);
  if (!plan) return;
  void* ptrs[] = {plan->probs, plan->units, plan->queue};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete plan;
}

int batch_sk_build(mhar_ctx* const* ctx, int count, void** plan_out, char* err, size_t err_len) {
  *plan_out = nullptr;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx[0]->device);
  std::vector<BskProblem> probs(count);
  std::vector<BskUnit> units;
  std::vector<long long> size(count);
  for (int q = 0; q < count; ++q) {
    const mhar_ctx* c = ctx[q];
    const TcPlan* tp = static_cast<const TcPlan*>(c->tc);
    BskProblem& P = probs[q];
    std::memset(&P, 0, sizeof(P));
    P.ah = tp->ah; P.al = tp->al; P.dh = tp->dh; P.dl = tp->dl;
    P.dh2 = tp->dh2; P.dl2 = tp->dl2; P.xh = tp->xh; P.xl = tp->xl;
    P.rows = c->d.rows;
    P.Xh = c->d.Xh;
    P.wscale = c->d.wscale;
    P.lmin = c->d.lmin;
    P.lmax = c->d.lmax;
    P.theta = c->d.theta;
    P.status = c->d.status;
    P.counters = c->d.counters;
    P.err = c->d.status + 1;
    P.step_ptr = c->d.step;
    P.seed = c->opts.seed;
    P.walker0 = c->opts.walker0;
    P.z = c->z;
    P.kdim = c->kdim;
    P.k_chunks = c->k_pad / kTcKChunk;
    P.k_pad = c->k_pad;
    P.m_tiles = tc_plan_m_tiles(c);
    P.wt = make_walker_tail(c, 0);
    size[q] = static_cast<long long>(P.m_tiles) * P.k_chunks;
    for (int st = 0; st < tc_plan_strips(c); ++st) units.push_back({q, st});
  }
  // Largest units first, so that the last units pulled are short ones.
  std::stable_sort(units.begin(), units.end(), [&](const BskUnit& a, const BskUnit& b) {
    return size[a.prob] > size[b.prob];
  });
  BatchSkPlan* plan = new BatchSkPlan();
  plan->n_units = static_cast<int>(units.size());
  plan->grid = std::min(sms, plan->n_units);
  cudaError_t e = cudaFuncSetAttribute(recompute_batch_sk_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmemBsk));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&plan->probs), sizeof(BskProblem) * probs.size());
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&plan->units), sizeof(BskUnit) * units.size());
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&plan->queue), 2 * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->probs, probs.data(), sizeof(BskProblem) * probs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->units, units.data(), sizeof(BskUnit) * units.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(plan->queue, 0, 2 * sizeof(int));
  if (e != cudaSuccess) {
    snprintf(err, err_len, "batched persistent plan: %s", cudaGetErrorString(e));
    cudaGetLastError();
    batch_sk_destroy(plan);
    return MHAR_E_CUDA;
  }
  *plan_out = plan;
  return MHAR_OK;
}

cudaError_t launch_recompute_batch_sk(const void* plan_v, int j, cudaStream_t stream) {
  const BatchSkPlan* plan = static_cast<const BatchSkPlan*>(plan_v);
  BskParams p;
  p.probs = plan->probs;
  p.units = plan->units;
  p.n_units = plan->n_units;
  p.queue = plan->queue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan->grid, 1, 1);
  cfg.blockDim = dim3(kThreadsSk, 1, 1);
  cfg.dynamicSmemBytes = kSmemBsk;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, recompute_batch_sk_kernel, p, j);
}

}  // namespace mhar
