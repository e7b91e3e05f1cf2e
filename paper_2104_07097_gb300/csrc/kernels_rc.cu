// kernels_rc.cu -- the walker step with the slack recomputed on the tensor
// cores every iteration (MHAR_MIXED_RECOMPUTE mode).
//
// This is the paper's own formulation of the line sets (Lemma 4.2: A X, then
// B - A X, then A D, ratios, sign split, column min / max) executed as one
// fused kernel:
//   P = X A^T and G = D A^T   tcgen05.mma kind::f16, each operand an FP16
//                             hi + lo pair, three products per matrix
//                             (hi.hi + hi.lo + lo.hi), FP32 accumulation in
//                             tensor memory
//   s_i = b_i - p_i           (in units of the row's power-of-two scale)
//   lambda_max = min{ s_i / g_i : g_i > 0 },  lambda_min = max{ s_i / g_i : g_i < 0 }
//   theta = lambda_min + u (lambda_max - lambda_min)
// The move X += D diag(theta) is made at the end of the same kernel, which
// also re-splits X; the next directions are drawn early in the kernel into
// the other of two direction pairs (walker_tail.cuh).
// Nothing of size m x z is stored: no slack array, no ratio matrix, no
// drift and no refresh.  Per walker-step the tensor cores do 12 m n flops.
//
// Decomposition: 128 walkers per CTA (MMA M, one walker per TMEM lane), a
// cluster of C CTAs along the constraint rows; each CTA streams its row tiles
// (MMA N = 128) through a pair of double-buffered TMEM accumulators (G and P:
// 4 x 128 columns), so the epilogue of tile t overlaps the MMAs of tile t+1.
// The walker operands (D and X pairs) stay in shared memory for the whole
// launch when n <= 128 and are streamed per tile otherwise; the A pairs stream
// through two pairs of 16 KB half-slots (hi and lo of one K chunk behind one
// barrier) so loads run a K chunk ahead of the MMAs.  Each CTA pushes its
// partial chords into every peer's shared memory before one cluster barrier,
// after which CTAs finish independently.
//
// Warp roles (608 threads): warp 0 TMA producer, warp 1 MMA issuer of the G
// products and TMEM owner, warp 18 MMA issuer of the P products, warps 2..17
// epilogue (four per TMEM lane quarter, each taking 32 of every tile's 128
// columns).  Every mbarrier wait is bounded (~2 s); on expiry
// the kernel flags the error word and still passes every cluster barrier.
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

constexpr int kWSlots = 2;                           // walker-operand slots
constexpr int kASlots = 4;                           // A half-slots (Ah or Al of one chunk)
constexpr int kAPairs = kASlots / 2;                 // A slots: Ah and Al of one chunk
constexpr int kWBytes = 4 * kOperandBytes;           // Dh, Dl, Xh, Xl chunk
constexpr int kABytes = kOperandBytes;               // Ah or Al chunk
constexpr int kEpiWarps = 16;
// The MMAs are issued from two threads: warp 1 the G products, warp kPWarp
// the P products (a single thread issuing all of them keeps the tensor pipe
// near 80 cycles per 128 x 128 x 16 MMA on GB300).
constexpr int kPWarp = 2 + kEpiWarps;
constexpr int kThreadsRc = (3 + kEpiWarps) * 32;
constexpr int kMaxTiles = 32;                        // rows per CTA <= 4096
constexpr int kMaxCluster = 8;

struct RcParams {
  const float* rows;        // 3 m_pad: b_i / row_scale_i and the error bounds (row_block)
  const __half* Xh;         // z_ld x k_pad, row-major: FP16 hi of the scaled points
  const float* wscale;      // z_ld: X[k,:] = wscale[k] (Xh + Xl)[k,:]
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
  int z, kdim, k_chunks, k_pad, tiles_per_cta, m_tiles;
  int ext_tail;             // 1: the walker-side work is a separate launch (batches)
  WalkerTail wt;            // walker-side work (walker_tail.cuh)
};

struct RcTail {
  uint64_t w_full[kWSlots];
  uint64_t w_empty[kWSlots];
  uint64_t a_full[kASlots];
  uint64_t a_empty[kASlots];
  uint64_t t_full[2];
  uint64_t t_empty[2];
  uint32_t tmem_base;
  int timed_out;
  float part_lo[4][kWalkers];
  float part_hi[4][kWalkers];
  float recv_lo[kMaxCluster][kWalkers];   // partial chords pushed by every CTA of the cluster
  float recv_hi[kMaxCluster][kWalkers];
  float theta_s[kWalkers];
  unsigned int red[kWalkers];
  float nrm[3 * kWalkers];                // operand_norms
};

constexpr size_t kSmemRc = 1024 + static_cast<size_t>(kWSlots) * kWBytes +
                           static_cast<size_t>(kASlots) * kABytes + sizeof(RcTail);
static_assert(kSmemRc <= 232448, "recompute_tc_kernel exceeds the shared memory of a CTA");

__device__ __forceinline__ void st_dsmem_f32(float* local, uint32_t rank, float v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(remote), "f"(v) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Tensor maps of one problem: A pair, both direction pairs, point pair.
struct RcMaps {
  CUtensorMap ah, al, dh, dl, dh2, dl2, xh, xl;
};

// One cluster's work for one walker strip of one problem (`strip`), iteration
// step + j.  The maps may live in kernel parameters or in global memory.
// LAST: K steps in the operands' last 64-column chunk (1..4), a compile-time
// constant so that the MMA runs carry no branches; 0: taken at run time (the
// batched kernel, whose units differ in n).
template <int LAST>
__device__ __forceinline__ void rc_body(const RcMaps& mp, const RcParams& p, int strip, int j) {
  const CUtensorMap& tm_ah = mp.ah;
  const CUtensorMap& tm_al = mp.al;
  const CUtensorMap& tm_dh = mp.dh;
  const CUtensorMap& tm_dl = mp.dl;
  const CUtensorMap& tm_dh2 = mp.dh2;
  const CUtensorMap& tm_dl2 = mp.dl2;
  const CUtensorMap& tm_xh = mp.xh;
  const CUtensorMap& tm_xl = mp.xl;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* wslot = base;                                   // kWSlots x 64 KB
  uint8_t* aslot = base + kWSlots * kWBytes;               // kASlots x 16 KB
  RcTail* tail = reinterpret_cast<RcTail*>(aslot + kASlots * kABytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TailItem tail_item;  // the epilogue threads' first tail item
  tail_item.valid = 0;
  const int csz_i = static_cast<int>(gridDim.x);
  const int share = (kWalkers + csz_i - 1) / csz_i;   // walkers of this CTA's walker-side work
  const int w_begin = static_cast<int>(blockIdx.x) * share;
  const int w_count = max(0, min(share, kWalkers - w_begin));
  const uint32_t rank = blockIdx.x;
  const uint32_t csize = gridDim.x;
  const int tile0 = static_cast<int>(rank) * p.tiles_per_cta;
  int ntiles = p.m_tiles - tile0;
  ntiles = ntiles < 0 ? 0 : (ntiles > p.tiles_per_cta ? p.tiles_per_cta : ntiles);
  const int row_base = tile0 * kRowsTile;
  const bool resident = p.k_chunks <= kWSlots;

  if (threadIdx.x == 0) {
    // Slots are free, and a tile's accumulators full, once both MMA threads
    // have committed them.
    for (int s = 0; s < kWSlots; ++s) { mbar_init(&tail->w_full[s], 1); mbar_init(&tail->w_empty[s], 2); }
    for (int s = 0; s < kASlots; ++s) { mbar_init(&tail->a_full[s], 1); mbar_init(&tail->a_empty[s], 2); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tail->t_full[b], 2); mbar_init(&tail->t_empty[b], kEpiWarps); }
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
  const uint64_t step = *p.step_ptr + static_cast<uint64_t>(j);
  const int cur = static_cast<int>(step & 1ull);  // this iteration's direction pair

  if (warp == 0) {
    // ---- TMA producer --------------------------------------------------------
    if (lane == 0) {
      int w_it = 0, a_it = 0;
      const int yw = strip * kWalkers;
      for (int nt = 0; nt < ntiles; ++nt) {
        for (int kc = 0; kc < p.k_chunks; ++kc) {
          const int x = kc * kTcKChunk;
          if (!resident || nt == 0) {
            const int s = w_it % kWSlots;
            if (w_it >= kWSlots) mbar_wait(&tail->w_empty[s], ((w_it / kWSlots) - 1) & 1, timed_out, p.err);
            uint8_t* dst = wslot + s * kWBytes;
            mbar_expect_tx(&tail->w_full[s], kWBytes);
            tma_load_2d(dst, cur ? &tm_dh2 : &tm_dh, &tail->w_full[s], x, yw);
            tma_load_2d(dst + kOperandBytes, cur ? &tm_dl2 : &tm_dl, &tail->w_full[s], x, yw);
            tma_load_2d(dst + 2 * kOperandBytes, &tm_xh, &tail->w_full[s], x, yw);
            tma_load_2d(dst + 3 * kOperandBytes, &tm_xl, &tail->w_full[s], x, yw);
            ++w_it;
          }
          // A's hi and lo chunk in one pair of half-slots behind one barrier
          // (every wait, fence and commit on the MMA thread's path costs issue
          // time).
          const int yr = row_base + nt * kRowsTile;
          const int s = a_it % kAPairs;
          if (a_it >= kAPairs) mbar_wait(&tail->a_empty[s], ((a_it / kAPairs) - 1) & 1, timed_out, p.err);
          mbar_expect_tx(&tail->a_full[s], 2 * kABytes);
          tma_load_2d(aslot + (2 * s) * kABytes, &tm_ah, &tail->a_full[s], x, yr);
          tma_load_2d(aslot + (2 * s + 1) * kABytes, &tm_al, &tail->a_full[s], x, yr);
          ++a_it;
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
      int w_it = 0, a_it = 0;
      for (int nt = 0; nt < ntiles; ++nt) {
        const int b = nt & 1;
        if (nt >= 2) mbar_wait(&tail->t_empty[b], ((nt >> 1) - 1) & 1, timed_out, p.err);
        tc_fence_after();
        const uint32_t d_tmem = tmem + static_cast<uint32_t>(b * 256) + (g_side ? 0u : 128u);
        auto chunk = [&](int kc, auto ks_c) {
          constexpr int KS = decltype(ks_c)::value;
          int ws;
          if (resident) {
            ws = kc;
            if (nt == 0) mbar_wait(&tail->w_full[ws], 0, timed_out, p.err);
          } else {
            ws = w_it % kWSlots;
            mbar_wait(&tail->w_full[ws], (w_it / kWSlots) & 1, timed_out, p.err);
          }
          // Descriptors are built once per slot; one K step of 16 FP16 moves the
          // start address by 32 bytes, i.e. adds 2 to the descriptor.
          const uint32_t w0 = smem_u32(wslot + ws * kWBytes) + op0;
          const uint64_t o_h = sw128_desc(w0), o_l = sw128_desc(w0 + kOperandBytes);
          // A hi: the two products that read it; A lo: the hi part of the
          // walker operand times it; then release the pair of half-slots.
          const int as = a_it % kAPairs;
          mbar_wait(&tail->a_full[as], (a_it / kAPairs) & 1, timed_out, p.err);
          tc_fence_after();
          const uint64_t ah = sw128_desc(smem_u32(aslot + (2 * as) * kABytes));
          const uint64_t al = sw128_desc(smem_u32(aslot + (2 * as + 1) * kABytes));
          if constexpr (KS > 0) {
            ss_run2<KS>(d_tmem, o_h, o_l, ah, idesc, kc > 0 ? 1u : 0u);
            ss_run1<KS>(d_tmem, o_h, al, idesc);
          } else {
            const int ks_n = min(kTcKChunk / kTcK, (p.kdim - kc * kTcKChunk) / kTcK);
            ss_run2_n(ks_n, d_tmem, o_h, o_l, ah, idesc, kc > 0 ? 1u : 0u);
            ss_run1_n(ks_n, d_tmem, o_h, al, idesc);
          }
          mma_commit(&tail->a_empty[as]);
          ++a_it;
          if (!resident) {
            mma_commit(&tail->w_empty[ws]);
            ++w_it;
          }
        };
        if constexpr (LAST > 0) {
          for (int kc = 0; kc + 1 < p.k_chunks; ++kc) chunk(kc, std::integral_constant<int, 4>{});
          chunk(p.k_chunks - 1, std::integral_constant<int, LAST>{});
        } else {
          for (int kc = 0; kc < p.k_chunks; ++kc) chunk(kc, std::integral_constant<int, 0>{});
        }
        mma_commit(&tail->t_full[b]);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: s = b - p, ratios, per-walker partial chord ------------------
    // First, while the first row tiles are on their way: iteration s+1's
    // directions into the other pair (walker_tail.cuh, step 0).
    const int e = warp - 2;
    const int q = warp & 3;
    const int cg = e >> 2;
    const int row0 = row_base + cg * 32;
    if (lane < 4 && ntiles > 0) prefetch_l1(row_block(p.rows, row0) + 32 * lane);
    if (p.wt.draw)
      walker_draw_next<kEpiWarps * 32>(p.wt, cur, p.seed, step + 1ull, p.walker0, strip, p.z,
                                       w_begin, w_count, static_cast<int>(threadIdx.x) - 64);
    const int wl = q * 32 + lane;
    const int k = strip * kWalkers + wl;
    const float ws = p.wscale[k];
    WalkerNorms wn =
        operand_norms<kEpiWarps * 32>(p.wt.Dh[cur], p.Xh, p.k_pad, k, wl, cg, ws, tail->nrm);
    if (k < p.z) add_correction(p.wt, k, wn);
    ChordAcc acc;
    acc.init();
    for (int nt = 0; nt < ntiles; ++nt) {
      const int b = nt & 1;
      if (lane < 4 && nt + 1 < ntiles) prefetch_l1(row_block(p.rows, row0 + (nt + 1) * kRowsTile) + 32 * lane);
      mbar_wait(&tail->t_full[b], (nt >> 1) & 1, timed_out, p.err, true);
      tc_fence_after();
      const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
      const uint32_t gcol = tmem + lane_off + static_cast<uint32_t>(b * 256 + cg * 32);
      float sv[32], gv[32];
      tmem_ld32(gcol + 128u, sv);
      tmem_ld32(gcol, gv);
      // The accumulators of this buffer are in registers: let the MMA reuse it.
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tail->t_empty[b]);
      float fx, fd;
      wn.pick(p.rows, row0 + nt * kRowsTile, fx, fd);
      slack32(sv, p.rows, row0 + nt * kRowsTile, ws, fx);
      scan32(sv, gv, p.rows, row0 + nt * kRowsTile, fd, acc);
    }
    const float lo = acc.lo_all(), hi = acc.hi_all();
    tail->part_lo[cg][wl] = lo;
    tail->part_hi[cg][wl] = hi;
    named_bar<kEpiWarps * 32>();
    if (cg == 0) {
      const float L = fmaxf(fmaxf(lo, tail->part_lo[1][wl]), fmaxf(tail->part_lo[2][wl], tail->part_lo[3][wl]));
      const float H = fminf(fminf(hi, tail->part_hi[1][wl]), fminf(tail->part_hi[2][wl], tail->part_hi[3][wl]));
      // Push this CTA's partial chord into slot `rank` of every CTA of the
      // cluster: each then knows the strip's chords without a second barrier.
      for (uint32_t r = 0; r < csize; ++r) {
        st_dsmem_f32(&tail->recv_lo[rank][wl], r, L);
        st_dsmem_f32(&tail->recv_hi[rank][wl], r, H);
      }
    }
  }

  // Every push is visible after this barrier; no remote access follows it.
  // Between its arrive and its wait the epilogue loads its first tail item
  // (the loads do not depend on theta), so their latency overlaps the barrier.
  tc_fence_before();
  cluster_arrive();
  if (warp >= 2 && warp < kPWarp && !p.ext_tail)
    walker_tail_prefetch<kEpiWarps * 32>(p.wt, cur, strip, p.z, w_begin, w_count,
                                         static_cast<int>(threadIdx.x) - 64, tail_item);
  cluster_wait();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }

  if (warp >= 2 && warp < kPWarp && ((warp - 2) >> 2) == 0) {
    const int q = warp & 3;
    const int wl = q * 32 + lane;
    const int k = strip * kWalkers + wl;
    float L = -INFINITY, H = INFINITY;
    for (uint32_t r = 0; r < csize; ++r) {
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
        const U4 w = philox_block(p.seed, step, p.walker0 + static_cast<uint32_t>(k), 0u,
                                  kStreamChord);
        const double u = open_unit_f64(w.x);
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
  if (warp >= 2 && warp < kPWarp && !p.ext_tail) {
    named_bar<kEpiWarps * 32>();
    walker_tail<kEpiWarps * 32>(p.wt, cur, strip, p.z, w_begin, w_count, tail->theta_s,
                                tail->red, static_cast<int>(threadIdx.x) - 64, tail_item);
  }
}


template <int LAST>
__global__ void __launch_bounds__(kThreadsRc, 1)
recompute_tc_kernel(const __grid_constant__ RcMaps maps, const __grid_constant__ RcParams p) {
  rc_body<LAST>(maps, p, static_cast<int>(blockIdx.y), p.j);
}

// Batched form: one launch for many problems.  blockIdx.y indexes a unit, a
// (problem, walker strip) pair, whose maps and parameters are in global
// memory; every unit's cluster is gridDim.x CTAs along its rows.
struct alignas(128) BatchUnit {
  RcMaps maps;
  RcParams p;
  int strip;
};

__global__ void __launch_bounds__(kThreadsRc, 1)
recompute_batch_kernel(const BatchUnit* __restrict__ units, int j) {
  const BatchUnit& u = units[blockIdx.y];
  rc_body<0>(u.maps, u.p, u.strip, j);
}

struct RcShape {
  int C = 1;
  int tiles_per_cta = 1;
};

RcShape rc_shape(const mhar_ctx* c, const TcPlan* plan) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  RcShape s;
  // Fill the SMs with (row groups x walker strips) CTAs, one per SM.
  int C = sms / plan->strips;
  C = C < 1 ? 1 : (C > 8 ? 8 : C);
  C = C > plan->m_tiles ? plan->m_tiles : C;
  s.tiles_per_cta = (plan->m_tiles + C - 1) / C;
  while (s.tiles_per_cta > kMaxTiles && C < kMaxCluster) {
    ++C;
    s.tiles_per_cta = (plan->m_tiles + C - 1) / C;
  }
  s.C = (plan->m_tiles + s.tiles_per_cta - 1) / s.tiles_per_cta;
  return s;
}

}  // namespace

bool rc_prefers_stream_k(const mhar_ctx* c) {
  const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const RcShape s = rc_shape(c, plan);
  // Row tiles on the busiest SM: clusters run in waves of `sms` CTAs; the
  // stream-K cut gives every SM an equal share plus about one tile of
  // per-segment overhead.
  // A body too tall for clusters of at most 8 CTAs goes to stream-K.
  if (s.C > kMaxCluster || s.tiles_per_cta > kMaxTiles) return true;
  const long long ctas = static_cast<long long>(plan->strips) * s.C;
  const long long waves = (ctas + sms - 1) / sms;
  const long long cluster_cost = waves * s.tiles_per_cta;
  const long long total = static_cast<long long>(plan->strips) * plan->m_tiles;
  const long long sk_cost = (total + sms - 1) / sms + 1;
  return sk_cost * 100 < cluster_cost * 93;
}

int rc_prepare(mhar_ctx* c) {
  const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
  const RcShape s = rc_shape(c, plan);
  if (s.C > kMaxCluster || s.tiles_per_cta > kMaxTiles) {
    snprintf(c->err, sizeof(c->err),
             "recompute mode covers m <= %d inequality rows (got %d row tiles)",
             kMaxCluster * kMaxTiles * kRowsTile, plan->m_tiles);
    return MHAR_E_UNSUPPORTED;
  }
  cudaError_t e = cudaSuccess;
  for (auto* k : {recompute_tc_kernel<1>, recompute_tc_kernel<2>, recompute_tc_kernel<3>,
                  recompute_tc_kernel<4>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(kSmemRc));
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "recompute kernel attributes: %s", cudaGetErrorString(e));
    cudaGetLastError();
    return MHAR_E_CUDA;
  }
  return MHAR_OK;
}

namespace {

RcParams rc_params(const mhar_ctx* c, int j, int tiles_per_cta) {
  const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
  RcParams p;
  p.rows = c->d.rows;
  p.Xh = c->d.Xh;
  p.k_pad = c->k_pad;
  p.ext_tail = 0;
  p.wscale = c->d.wscale;
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
  p.kdim = c->kdim;
  p.k_chunks = c->k_pad / kTcKChunk;
  p.tiles_per_cta = tiles_per_cta;
  p.m_tiles = plan->m_tiles;
  p.wt = make_walker_tail(c, 0);
  return p;
}

RcMaps rc_maps(const TcPlan* plan) {
  RcMaps maps;
  maps.ah = plan->ah;
  maps.al = plan->al;
  maps.dh = plan->dh;
  maps.dl = plan->dl;
  maps.dh2 = plan->dh2;
  maps.dl2 = plan->dl2;
  maps.xh = plan->xh;
  maps.xl = plan->xl;
  return maps;
}

cudaLaunchConfig_t rc_config(int C, int rows, cudaStream_t stream, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, rows, 1);
  cfg.blockDim = dim3(kThreadsRc, 1, 1);
  cfg.dynamicSmemBytes = kSmemRc;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // Programmatic dependent launch: the grid may be scheduled while the
  // previous kernel finishes; it waits (griddepcontrol.wait) before reading.
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cfg;
}

}  // namespace

cudaError_t launch_recompute_tc(mhar_ctx* c, int j) {
  const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
  const RcShape s = rc_shape(c, plan);
  const RcParams p = rc_params(c, j, s.tiles_per_cta);
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = rc_config(s.C, plan->strips, c->stream, attr);
  switch (last_chunk_steps(p.kdim, p.k_chunks)) {
    case 1: return cudaLaunchKernelEx(&cfg, recompute_tc_kernel<1>, rc_maps(plan), p);
    case 2: return cudaLaunchKernelEx(&cfg, recompute_tc_kernel<2>, rc_maps(plan), p);
    case 3: return cudaLaunchKernelEx(&cfg, recompute_tc_kernel<3>, rc_maps(plan), p);
    default: return cudaLaunchKernelEx(&cfg, recompute_tc_kernel<4>, rc_maps(plan), p);
  }
}

// ---- batches ------------------------------------------------------------------
int batch_table_build(mhar_ctx* const* ctx, int count, int C, void** table, int* units,
                      char* err, size_t err_len) {
  *table = nullptr;
  *units = 0;
  cudaError_t e = cudaFuncSetAttribute(recompute_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmemRc));
  if (e != cudaSuccess) {
    snprintf(err, err_len, "batch kernel attributes: %s", cudaGetErrorString(e));
    cudaGetLastError();
    return MHAR_E_CUDA;
  }
  std::vector<BatchUnit> host;
  for (int q = 0; q < count; ++q) {
    const mhar_ctx* c = ctx[q];
    const TcPlan* plan = static_cast<const TcPlan*>(c->tc);
    const int tpc = (plan->m_tiles + C - 1) / C;
    for (int st = 0; st < plan->strips; ++st) {
      BatchUnit u;
      std::memset(&u, 0, sizeof(u));
      u.maps = rc_maps(plan);
      u.p = rc_params(c, 0, tpc);
      u.p.ext_tail = 1;   // walker_update_batch_kernel follows
      u.strip = st;
      host.push_back(u);
    }
  }
  // Largest units first: CTAs start in grid order, so the long ones do not
  // end up alone at the end of the launch.
  std::stable_sort(host.begin(), host.end(), [](const BatchUnit& a, const BatchUnit& b) {
    return static_cast<long long>(a.p.m_tiles) * a.p.k_chunks >
           static_cast<long long>(b.p.m_tiles) * b.p.k_chunks;
  });
  void* d = nullptr;
  e = cudaMalloc(&d, sizeof(BatchUnit) * host.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(d, host.data(), sizeof(BatchUnit) * host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    snprintf(err, err_len, "batch table: %s", cudaGetErrorString(e));
    cudaGetLastError();
    return MHAR_E_CUDA;
  }
  *table = d;
  *units = static_cast<int>(host.size());
  return MHAR_OK;
}

cudaError_t launch_recompute_batch(const void* table, int units, int C, int j,
                                   cudaStream_t stream) {
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = rc_config(C, units, stream, attr);
  return cudaLaunchKernelEx(&cfg, recompute_batch_kernel,
                            static_cast<const BatchUnit*>(table), j);
}

}  // namespace mhar
