// walker_tail.cuh -- the walker-side work of a recompute-mode iteration, run
// inside the chord kernel of iteration s (the TMEM-operand and cluster
// kernels), or after it, item for item the same, by the walker update kernels
// of the stream-K and batched launches (kernels_sk.cu).
//
// Every CTA of a walker strip's cluster takes a contiguous share of the
// strip's 128 walkers.
// Early, while the first row tiles are still on their way, when neither a
// projection nor a preconditioner follows the draw:
//  (0) draw iteration s+1's directions (Section 4.3, Philox stream 0) into
//      FP16 pair (s+1) % 2 -- the kernel reads pair s % 2, so no one reads
//      the pair being written.
// After the cluster barrier, when every CTA holds the strip's 128 chords and
// theta (computed identically in each CTA):
//  (1) move the point, x += theta (d - Q^T c')  (Section 4.5; c' is the
//      exact row-space part of the rounded direction, Q the orthonormal rows
//      of A_E, when m_E > 0),
//      in double-float arithmetic;
//  (2) split the moved point into the FP16 operand pair of the next
//      iteration: x_i / (sigma_i 2^e), 2^e the per-walker power of two with
//      max_i |x_i| / sigma_i 2^-e in [0.5, 1).
// The arithmetic is element for element that of prep_walkers_kernel.
// Threads take (walker, 8-coordinate chunk) items with the walker fastest, so
// a warp moves whole chunks of 32 consecutive walkers.
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "mhar_device.cuh"
#include "mhar_internal.h"
#include "tc_common.cuh"

namespace mhar {

struct WalkerTail {
  float* Xhi;            // z x n_ld
  float* Xlo;
  __half* Dh[2];         // direction pairs s % 2 (operand layout, op_off)
  __half* Dl[2];
  __half* Xh;
  __half* Xl;
  float* wscale;         // z_ld
  const float* sigma;    // n_ld
  const float* Q32;      // mE x n_ld or null: orthonormal rows Q = L^{-1} A_E
  const float* corr;     // z x mE or null
  const float* corrn;    // z or null: ||Q^T corr / sigma||_2 of each walker's direction
  int mE, n, n_ld, k_pad, z_ld, inter, draw;
  int unit_sigma;        // 1: every sigma_i is 1, skip them
  // Preconditioned draw d = delta .* h + U g (pc_rank >= 0; only kernels that
  // pass shared scratch for g to walker_draw_next draw it themselves).
  const float* pc_delta; // n_ld
  const float* pc_U;     // n_ld x 32, zero beyond the rank
  int pc_rank;
  int* status;           // MHAR_ST_NONFINITE if a split value leaves the FP16 range
};

// The tail's arguments for a context (`inter`: interleaved operand layout;
// `pc_draw`: the kernel can draw preconditioned directions itself).
inline WalkerTail make_walker_tail(const mhar_ctx* c, int inter, bool pc_draw = false) {
  WalkerTail t;
  t.Xhi = c->d.Xhi;
  t.Xlo = c->d.Xlo;
  t.Dh[0] = c->d.Dh;
  t.Dl[0] = c->d.Dl;
  t.Dh[1] = c->d.Dh2 ? c->d.Dh2 : c->d.Dh;
  t.Dl[1] = c->d.Dl2 ? c->d.Dl2 : c->d.Dl;
  t.Xh = c->d.Xh;
  t.Xl = c->d.Xl;
  t.wscale = c->d.wscale;
  t.sigma = c->d.sigma;
  t.Q32 = c->d.Q32;
  t.corr = c->d.corr;
  t.corrn = c->d.corrn;
  t.mE = c->mE;
  t.n = c->n;
  t.n_ld = c->n_ld;
  t.k_pad = c->k_pad;
  t.z_ld = (c->z + tc::kWalkers - 1) / tc::kWalkers * tc::kWalkers;
  t.inter = inter;
  t.draw = (c->mE == 0 && (c->pc_rank < 0 || pc_draw)) ? 1 : 0;
  t.unit_sigma = c->unit_sigma ? 1 : 0;
  t.pc_delta = c->d.pc_delta32;
  t.pc_U = c->d.pc_U32;
  t.pc_rank = c->pc_rank;
  t.status = c->d.status;
  return t;
}

namespace tail_detail {

__device__ __forceinline__ void ld8(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void st8(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<float4*>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void ld8h(const __half* p, float* v) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    v[2 * e] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[e] & 0xffffu)));
    v[2 * e + 1] = __half2float(__ushort_as_half(static_cast<unsigned short>(w[e] >> 16)));
  }
}
// Splits 8 values into FP16 hi / lo halves and stores both 16-byte chunks;
// true if a value is non-finite or beyond the FP16 range.
__device__ __forceinline__ bool split_store8(const float* v, __half* hi_dst, __half* lo_dst) {
  uint32_t h[4], l[4];
  bool bad = false;
#pragma unroll
  for (int e = 0; e < 8; ++e) bad |= !(fabsf(v[e]) <= kHalfMax);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __half h0 = __float2half_rn(v[2 * e]);
    const __half h1 = __float2half_rn(v[2 * e + 1]);
    const __half l0 = __float2half_rn(v[2 * e] - __half2float(h0));
    const __half l1 = __float2half_rn(v[2 * e + 1] - __half2float(h1));
    h[e] = static_cast<uint32_t>(__half_as_ushort(h0)) | (static_cast<uint32_t>(__half_as_ushort(h1)) << 16);
    l[e] = static_cast<uint32_t>(__half_as_ushort(l0)) | (static_cast<uint32_t>(__half_as_ushort(l1)) << 16);
  }
  *reinterpret_cast<uint4*>(hi_dst) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_dst) = make_uint4(l[0], l[1], l[2], l[3]);
  return bad;
}

}  // namespace tail_detail

// Norm bounds of one walker's direction and scaled point (the chord's error
// margins, tc_common.cuh) from the FP16 hi rows of the row-major operands
// (walker k at k * k_pad): thread part == 0 of the walker sums the squares of
// its 8-element chunks in chunk order (the same order as the tensor-memory
// kernel) and takes the largest |d|, and shares them through `scr` (3 x 128
// floats of shared memory).  Run by all kThreads threads (named barrier 1).
// Returns (ws ||x_hat||_2, ||d_hat||_2, ws, max |d_hat|) for the walker with
// point scale ws.
template <int kThreads>
__device__ __forceinline__ tc::WalkerNorms operand_norms(const __half* Dh, const __half* Xh,
                                                         int k_pad, int k, int wl, int part,
                                                         float ws, float* scr) {
  constexpr int W = tc::kWalkers;
  if (part == 0) {
    const uint4* d4 = reinterpret_cast<const uint4*>(Dh + static_cast<size_t>(k) * k_pad);
    const uint4* x4 = reinterpret_cast<const uint4*>(Xh + static_cast<size_t>(k) * k_pad);
    float sd = 0.0f, sx = 0.0f, md = 0.0f;
    for (int c = 0; c < (k_pad >> 3); ++c) {
      const uint4 dv = __ldg(d4 + c);
      sd += tc::sumsq8(dv);
      md = fmaxf(md, tc::absmax8(dv));
      sx += tc::sumsq8(__ldg(x4 + c));
    }
    scr[wl] = sd;
    scr[W + wl] = sx;
    scr[2 * W + wl] = md;
  }
  tc::named_bar<kThreads>();
  tc::WalkerNorms r;
  r.nxw2 = ws * tc::norm_bound(scr[W + wl]);
  r.nd2 = tc::norm_bound(scr[wl]);
  r.ws = ws;
  r.ndinf = scr[2 * W + wl] * 1.00390625f;
  return r;
}

// With equalities the point moves along d - Q^T c' (walker_tail (1)) while
// the chord is found along d: |a_i . Q^T c'| <= |a_hat_i|_p ||Q^T c' /
// sigma||_2 and Kg_p >= 2^-22 |a_hat_i|_p, so 2^22 ||Q^T c' / sigma||_2 added
// to both direction norms covers it in the margin of a_i . d.
__device__ __forceinline__ void add_correction(const WalkerTail& t, int k, tc::WalkerNorms& wn) {
  if (t.corrn == nullptr) return;
  const float cc = 4194304.0f * __ldg(t.corrn + k);
  wn.nd2 += cc;
  wn.ndinf += cc;
}

// A thread's first item, loaded before theta is known (the loads do not
// depend on it), so that their latency hides behind the cluster barrier.
struct TailItem {
  float hi[8], lo[8], d[8];
  int valid;
};

// Item `tid` of the strip's share: x hi / lo and d = sigma (d_hi + d_lo).
template <int kThreads>
__device__ __forceinline__ void walker_tail_prefetch(const WalkerTail& t, int cur, int strip,
                                                     int z, int w_begin, int w_count, int tid,
                                                     TailItem& r) {
  using namespace tail_detail;
  const int chunks = (t.n + 7) >> 3;
  r.valid = 0;
  if (w_count <= 0 || tid >= w_count * chunks) return;
  const int c = tid / w_count, wo = tid - c * w_count;
  const int k = strip * tc::kWalkers + w_begin + wo;
  if (k >= z) return;
  const int i0 = 8 * c;
  const size_t xr = static_cast<size_t>(k) * t.n_ld + i0;
  const size_t o = op_off(k, i0, t.k_pad, t.z_ld, t.inter);
  float dh[8], dl[8];
  ld8(t.Xhi + xr, r.hi);
  ld8(t.Xlo + xr, r.lo);
  ld8h(t.Dh[cur] + o, dh);
  ld8h(t.Dl[cur] + o, dl);
#pragma unroll
  for (int e = 0; e < 8; ++e)
    r.d[e] = i0 + e < t.n ? (t.unit_sigma ? dh[e] + dl[e] : (dh[e] + dl[e]) * t.sigma[i0 + e]) : 0.0f;
  r.valid = 1;
}

// The same item staged in shared memory instead: at kernel start each thread
// copies its first item's x hi, x lo (8 floats each) and direction pair (8
// FP16 each) with asynchronous 16-byte copies (cp.async, no registers held),
// into its own kTailStageBytes slot; after the chord it reads them back with
// no global-memory latency on the walker-side path.  112-byte slots keep the
// 16-byte accesses of 8 consecutive threads on distinct banks.
constexpr int kTailStageBytes = 112;

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

template <int kThreads>
__device__ __forceinline__ void walker_tail_stage(const WalkerTail& t, int cur, int strip, int z,
                                                  int w_begin, int w_count, int tid,
                                                  uint8_t* slot) {
  using namespace tail_detail;
  const int chunks = (t.n + 7) >> 3;
  if (w_count <= 0 || tid >= w_count * chunks) return;
  const int c = tid / w_count, wo = tid - c * w_count;
  const int k = strip * tc::kWalkers + w_begin + wo;
  if (k >= z) return;
  const int i0 = 8 * c;
  const size_t xr = static_cast<size_t>(k) * t.n_ld + i0;
  const size_t o = op_off(k, i0, t.k_pad, t.z_ld, t.inter);
  cp_async16(slot, t.Xhi + xr);
  cp_async16(slot + 16, t.Xhi + xr + 4);
  cp_async16(slot + 32, t.Xlo + xr);
  cp_async16(slot + 48, t.Xlo + xr + 4);
  cp_async16(slot + 64, t.Dh[cur] + o);
  cp_async16(slot + 80, t.Dl[cur] + o);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int kThreads>
__device__ __forceinline__ void walker_tail_unstage(const WalkerTail& t, int strip, int z,
                                                    int w_begin, int w_count, int tid,
                                                    const uint8_t* slot, TailItem& r) {
  using namespace tail_detail;
  const int chunks = (t.n + 7) >> 3;
  r.valid = 0;
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (w_count <= 0 || tid >= w_count * chunks) return;
  const int c = tid / w_count, wo = tid - c * w_count;
  const int k = strip * tc::kWalkers + w_begin + wo;
  if (k >= z) return;
  const int i0 = 8 * c;
  float dh[8], dl[8];
  ld8(reinterpret_cast<const float*>(slot), r.hi);
  ld8(reinterpret_cast<const float*>(slot + 32), r.lo);
  ld8h(reinterpret_cast<const __half*>(slot + 64), dh);
  ld8h(reinterpret_cast<const __half*>(slot + 80), dl);
#pragma unroll
  for (int e = 0; e < 8; ++e)
    r.d[e] = i0 + e < t.n ? (t.unit_sigma ? dh[e] + dl[e] : (dh[e] + dl[e]) * t.sigma[i0 + e]) : 0.0f;
  r.valid = 1;
}

// (0): run by kThreads threads (tid = 0..kThreads-1, sharing named barrier 1
// when preconditioned); `next_step` = s + 1.  With a preconditioner the
// direction is d = delta .* h + U g, g the walker's rank-r normals (Philox
// stream 2), kept in `gs` (w_count x 32 floats of shared memory); the
// arithmetic is that of precondition_kernel (FP32, terms in column order,
// then d / sigma split into the FP16 pair).
template <int kThreads>
__device__ void walker_draw_next(const WalkerTail& t, int cur, uint64_t seed, uint64_t next_step,
                                 uint32_t walker0, int strip, int z, int w_begin, int w_count,
                                 int tid, float* gs = nullptr) {
  using namespace tail_detail;
  const int chunks = (t.n + 7) >> 3;
  const int items = w_count * chunks;
  __half* Dh = t.Dh[cur ^ 1];
  __half* Dl = t.Dl[cur ^ 1];
  const bool pre = t.pc_rank >= 0 && gs != nullptr;
  if (pre) {
    const int quads = (t.pc_rank + 3) >> 2;
    for (int idx = tid; idx < w_count * (kMaxPcRank / 4); idx += kThreads) {
      const int w = idx / (kMaxPcRank / 4), q = idx - w * (kMaxPcRank / 4);
      const int k = strip * tc::kWalkers + w_begin + w;
      float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (q < quads && k < z) {
        const U4 r = philox_block(seed, next_step, walker0 + static_cast<uint32_t>(k),
                                  static_cast<uint32_t>(q), kStreamLowRank);
        box_muller_f32(r.x, r.y, v[0], v[1]);
        box_muller_f32(r.z, r.w, v[2], v[3]);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) gs[w * kMaxPcRank + 4 * q + e] = 4 * q + e < t.pc_rank ? v[e] : 0.0f;
    }
    tc::named_bar<kThreads>();
  }
  for (int it = tid; it < items; it += kThreads) {
    const int c = it / w_count, wo = it - c * w_count;
    const int k = strip * tc::kWalkers + w_begin + wo;
    if (k >= z) continue;
    const int i0 = 8 * c;
    const size_t o = op_off(k, i0, t.k_pad, t.z_ld, t.inter);
    float v[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (i0 + 4 * h < t.n) {
        const U4 w = philox_block(seed, next_step, walker0 + static_cast<uint32_t>(k),
                                  static_cast<uint32_t>(2 * c + h), kStreamDirection);
        box_muller_f32(w.x, w.y, v[4 * h], v[4 * h + 1]);
        box_muller_f32(w.z, w.w, v[4 * h + 2], v[4 * h + 3]);
      } else {
        v[4 * h] = v[4 * h + 1] = v[4 * h + 2] = v[4 * h + 3] = 0.0f;
      }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (i0 + e >= t.n) v[e] = 0.0f;
    if (!pre && !t.unit_sigma) {
      // The FP16 pair holds d_i / sigma_i (sigma a power of two: exact).
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] *= pow2_recip(t.sigma[i0 + e]);
    }
    if (pre) {
      const float* g = gs + wo * kMaxPcRank;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = i0 + e;
        if (i >= t.n) continue;
        const float* u = t.pc_U + static_cast<size_t>(i) * kMaxPcRank;
        float acc = t.pc_delta[i] * v[e];
#pragma unroll 8
        for (int c2 = 0; c2 < kMaxPcRank; ++c2) acc = fmaf(u[c2], g[c2], acc);
        v[e] = acc * pow2_recip(t.sigma[i]);
      }
    }
    if (split_store8(v, Dh + o, Dl + o)) atomicOr(t.status, MHAR_ST_NONFINITE);
  }
}

// Shared scratch that walker_tail can route the moved points through, so
// that their rows go to global memory as whole coalesced lines (an item's 32
// bytes per thread, one row per walker, would otherwise be a separate
// transaction per thread): 2 w_count rows of tail_row_stride(n_ld) floats.
__host__ __device__ constexpr int tail_row_stride(int n_ld) { return n_ld + 4; }

// (1) and (2): run by kThreads threads (tid = 0..kThreads-1) that share named
// barrier 1.  theta_s: the strip's 128 theta values (shared memory); red:
// w_count words of shared scratch; `cur` = s % 2.  `first`: item tid,
// prefetched; items tid + kThreads, ... are loaded here.  `xrows`: null, or
// the scratch above when every item is a first item (items <= kThreads).
template <int kThreads>
__device__ void walker_tail(const WalkerTail& t, int cur, int strip, int z, int w_begin,
                            int w_count, const float* theta_s, unsigned int* red, int tid,
                            TailItem& first, float* xrows = nullptr) {
  using namespace tail_detail;
  const int chunks = (t.n + 7) >> 3;
  const int items = w_count * chunks;
  const int rs = tail_row_stride(t.n_ld);
  if (items > kThreads || chunks > 16) xrows = nullptr;
  for (int w = tid; w < w_count; w += kThreads) red[w] = 0u;
  tc::named_bar<kThreads>();

  // (1) move, and the walker's largest scaled coordinate.
  for (int it = tid; it < items; it += kThreads) {
    const int c = it / w_count, wo = it - c * w_count;
    const int k = strip * tc::kWalkers + w_begin + wo;
    if (k >= z) continue;
    const int i0 = 8 * c;
    const size_t xr = static_cast<size_t>(k) * t.n_ld + i0;
    const float th = theta_s[w_begin + wo];
    const bool cached = it == tid && first.valid;
    float hi[8], lo[8], d[8];
    if (cached) {
#pragma unroll
      for (int e = 0; e < 8; ++e) { hi[e] = first.hi[e]; lo[e] = first.lo[e]; d[e] = first.d[e]; }
    } else {
      ld8(t.Xhi + xr, hi);
      ld8(t.Xlo + xr, lo);
      if (th != 0.0f) {
        float dh[8], dl[8];
        const size_t o = op_off(k, i0, t.k_pad, t.z_ld, t.inter);
        ld8h(t.Dh[cur] + o, dh);
        ld8h(t.Dl[cur] + o, dl);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          d[e] = i0 + e < t.n ? (t.unit_sigma ? dh[e] + dl[e] : (dh[e] + dl[e]) * t.sigma[i0 + e]) : 0.0f;
      }
    }
    if (th != 0.0f) {
      // Coordinates past n have x = 0 and d = 0, for which the update is a
      // no-op: no per-coordinate branch.
#pragma unroll
      for (int e = 0; e < 8; ++e) df_axpy(hi[e], lo[e], th, d[e]);
      if (t.corr != nullptr) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int i = i0 + e;
          if (i >= t.n) continue;
          float dlt = 0.0f;
          for (int q = 0; q < t.mE; ++q)
            dlt = fmaf(t.Q32[static_cast<size_t>(q) * t.n_ld + i],
                       t.corr[static_cast<size_t>(k) * t.mE + q], dlt);
          lo[e] = fmaf(-th, dlt, lo[e]);
        }
      }
      if (xrows != nullptr) {
        // Into the walker's row in shared memory; stored below, coalesced.
        st8(xrows + wo * rs + i0, hi);
        st8(xrows + (w_count + wo) * rs + i0, lo);
      } else {
        st8(t.Xhi + xr, hi);
        st8(t.Xlo + xr, lo);
      }
    } else if (xrows != nullptr) {
      st8(xrows + wo * rs + i0, hi);
      st8(xrows + (w_count + wo) * rs + i0, lo);
    }
    if (cached) {
#pragma unroll
      for (int e = 0; e < 8; ++e) { first.hi[e] = hi[e]; first.lo[e] = lo[e]; }
    }
    float mx = 0.0f;
    if (t.unit_sigma) {
#pragma unroll
      for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fabsf(hi[e]));   // x = 0 past n
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (i0 + e < t.n) mx = fmaxf(mx, fabsf(hi[e]) * pow2_recip(t.sigma[i0 + e]));
    }
    atomicMax(red + wo, __float_as_uint(mx));  // non-negative floats order as their bits
  }
  tc::named_bar<kThreads>();
  if (xrows != nullptr) {
    // The moved rows: a warp per row, 16 bytes per lane along it (xrows is
    // only used when a row is at most 32 float4s: n <= 128).
    const int q4 = 2 * chunks;   // float4s of a row that items cover
    const int lane = tid & 31;
    for (int row = tid >> 5; row < 2 * w_count; row += kThreads / 32) {
      const int wo = row < w_count ? row : row - w_count;
      const int k = strip * tc::kWalkers + w_begin + wo;
      if (k >= z || lane >= q4) continue;
      const float4 v = *reinterpret_cast<const float4*>(xrows + row * rs + 4 * lane);
      float* dst = (row < w_count ? t.Xhi : t.Xlo) + static_cast<size_t>(k) * t.n_ld + 4 * lane;
      *reinterpret_cast<float4*>(dst) = v;
    }
  }

  // (2) FP16 pair of the scaled point.
  for (int it = tid; it < items; it += kThreads) {
    const int c = it / w_count, wo = it - c * w_count;
    const int k = strip * tc::kWalkers + w_begin + wo;
    if (k >= z) continue;
    const int i0 = 8 * c;
    const size_t xr = static_cast<size_t>(k) * t.n_ld + i0;
    const size_t o = op_off(k, i0, t.k_pad, t.z_ld, t.inter);
    const float mx = __uint_as_float(red[wo]);
    int ex = 0;
    if (mx > 0.0f) frexpf(mx, &ex);
    const float inv = ldexpf(1.0f, -ex);
    if (c == 0) t.wscale[k] = ldexpf(1.0f, ex);
    float hi[8], lo[8], v[8];
    if (it == tid && first.valid) {
#pragma unroll
      for (int e = 0; e < 8; ++e) { hi[e] = first.hi[e]; lo[e] = first.lo[e]; }
    } else {
      ld8(t.Xhi + xr, hi);
      ld8(t.Xlo + xr, lo);
    }
    // x = 0 and sigma = 1 past n: no per-coordinate branch.
    if (t.unit_sigma) {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (hi[e] + lo[e]) * inv;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (hi[e] + lo[e]) * inv * pow2_recip(t.sigma[i0 + e]);
    }
    if (split_store8(v, t.Xh + o, t.Xl + o)) atomicOr(t.status, MHAR_ST_NONFINITE);
  }
}

}  // namespace mhar
