// tc_common.cuh -- PTX building blocks shared by the tensor-core kernels:
// mbarriers with bounded waits, TMA tile loads, tcgen05 shared-memory and
// instruction descriptors, MMA issue / commit, tensor-memory loads, cluster
// barriers and distributed shared memory, plus the tensor-map plan.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "mhar_internal.h"

namespace mhar {
namespace tc {

constexpr int kWalkers = 128;                         // MMA M: walkers per CTA
constexpr int kRowsTile = 128;                        // MMA N: constraint rows per tile
constexpr int kOperandBytes = 128 * kTcKChunk * 2;    // one 128 x 64 FP16 tile = 16 KB
constexpr long long kTimeoutCycles = 4000000000ll;    // ~2 s at 2 GHz
constexpr int kErrTimeout = 1;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// One test of the phase with parity `parity` (no suspension: the producer and
// MMA threads are on the critical path and must resume the moment it completes).
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false (and flags the CTA) once ~2 s have passed or
// an earlier wait of this CTA already expired.  `sleepy` waiters (the
// epilogue warps, whose wait is long and not on the issue path) back off with
// __nanosleep so they do not take issue slots from the producer / MMA threads.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* timed_out,
                                          int* err, bool sleepy = false) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try_wait(a, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 16; ++i) {
      if (mbar_try_wait(a, parity)) return true;
      if (sleepy) __nanosleep(64);
    }
    if (*timed_out) return false;
    if (clock64() - t0 > kTimeoutCycles) {
      *timed_out = 1;
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor for a K-major operand stored as 128-byte
// rows with the 128B swizzle (8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);   // start address
  d |= static_cast<uint64_t>(1) << 16;                    // leading byte offset (unused)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;            // stride byte offset: 8 rows
  d |= static_cast<uint64_t>(1) << 46;                    // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                    // 128B swizzle
  return d;
}

// Instruction descriptor: kind::f16, A = B = FP16, D = FP32, both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Same MMA with the A operand read from tensor memory (lane = row of A, each
// 32-bit column two consecutive K elements) instead of shared memory.
__device__ __forceinline__ void mma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// A run of TMEM-operand MMAs over ks = 0..KS-1 K steps of one shared-memory
// slot, unrolled at compile time (a runtime trip count puts branches and
// address arithmetic between the single issuing thread's MMAs, which
// measurably starves the tensor pipe):
//   two operands:  D += A0[ks] B[ks]; D += A1[ks] B[ks]   (ks = 0..KS-1)
//   one operand:   D += A0[ks] B[ks]
// A operands in tensor memory at a + 8 ks (2 FP16 per 32-bit column), B
// descriptors at b + 2 ks (32 bytes per K step).  The very first MMA
// overwrites D when acc_first == 0; every other one accumulates.
template <int KS>
__device__ __forceinline__ void mma_ts_run2(uint32_t d, uint32_t a0, uint32_t a1, uint64_t b,
                                            uint32_t idesc, uint32_t acc_first) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint32_t ac = static_cast<uint32_t>(ks * 8);
    mma_f16_ts(d, a0 + ac, b + static_cast<uint64_t>(2 * ks), idesc, ks > 0 ? 1u : acc_first);
    mma_f16_ts(d, a1 + ac, b + static_cast<uint64_t>(2 * ks), idesc, 1u);
  }
}
template <int KS>
__device__ __forceinline__ void mma_ts_run1(uint32_t d, uint32_t a0, uint64_t b, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
    mma_f16_ts(d, a0 + static_cast<uint32_t>(ks * 8), b + static_cast<uint64_t>(2 * ks), idesc, 1u);
}

// The same for the shared-memory-operand kernels: one K chunk's MMAs against
// the A hi slot (G += Dh A, G += Dl A, P += Xh A, P += Xl A per K step) and
// against the A lo slot (G += Dh A, P += Xh A); descriptors advance by 2 per
// K step.  The first G and P MMAs of the hi run overwrite when acc_first == 0.
template <int KS>
__device__ __forceinline__ void mma_ss_hi(uint32_t g, uint32_t p, uint64_t dh, uint64_t dl,
                                          uint64_t xh, uint64_t xl, uint64_t ad, uint32_t idesc,
                                          uint32_t acc_first) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint64_t o = static_cast<uint64_t>(2 * ks);
    const uint32_t acc = ks > 0 ? 1u : acc_first;
    mma_f16(g, dh + o, ad + o, idesc, acc);
    mma_f16(g, dl + o, ad + o, idesc, 1u);
    mma_f16(p, xh + o, ad + o, idesc, acc);
    mma_f16(p, xl + o, ad + o, idesc, 1u);
  }
}
template <int KS>
__device__ __forceinline__ void mma_ss_lo(uint32_t g, uint32_t p, uint64_t dh, uint64_t xh,
                                          uint64_t ad, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint64_t o = static_cast<uint64_t>(2 * ks);
    mma_f16(g, dh + o, ad + o, idesc, 1u);
    mma_f16(p, xh + o, ad + o, idesc, 1u);
  }
}

// One accumulator's share of those runs, for kernels that issue the G and the
// P products from two threads: D += A0[ks] B[ks], D += A1[ks] B[ks] per K step
// (B = the A hi slot), and D += A0[ks] B[ks] (B = the A lo slot), shared-memory
// descriptors advancing by 2 per K step; the first MMA overwrites when
// acc_first == 0.
template <int KS>
__device__ __forceinline__ void ss_run2(uint32_t d, uint64_t a0, uint64_t a1, uint64_t b,
                                        uint32_t idesc, uint32_t acc_first) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint64_t o = static_cast<uint64_t>(2 * ks);
    mma_f16(d, a0 + o, b + o, idesc, ks > 0 ? 1u : acc_first);
    mma_f16(d, a1 + o, b + o, idesc, 1u);
  }
}
template <int KS>
__device__ __forceinline__ void ss_run1(uint32_t d, uint64_t a0, uint64_t b, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const uint64_t o = static_cast<uint64_t>(2 * ks);
    mma_f16(d, a0 + o, b + o, idesc, 1u);
  }
}

// Runtime K-step count (1..4) to ss_run2 / ss_run1.
__device__ __forceinline__ void ss_run2_n(int ks_n, uint32_t d, uint64_t a0, uint64_t a1, uint64_t b,
                                          uint32_t idesc, uint32_t acc_first) {
  switch (ks_n) {
    case 4: ss_run2<4>(d, a0, a1, b, idesc, acc_first); break;
    case 3: ss_run2<3>(d, a0, a1, b, idesc, acc_first); break;
    case 2: ss_run2<2>(d, a0, a1, b, idesc, acc_first); break;
    default: ss_run2<1>(d, a0, a1, b, idesc, acc_first); break;
  }
}
__device__ __forceinline__ void ss_run1_n(int ks_n, uint32_t d, uint64_t a0, uint64_t b,
                                          uint32_t idesc) {
  switch (ks_n) {
    case 4: ss_run1<4>(d, a0, b, idesc); break;
    case 3: ss_run1<3>(d, a0, b, idesc); break;
    case 2: ss_run1<2>(d, a0, b, idesc); break;
    default: ss_run1<1>(d, a0, b, idesc); break;
  }
}

// Runtime K-step count (1..4) to the runs above, for kernels that serve
// bodies of different n in one launch.
__device__ __forceinline__ void mma_ss_hi_n(int ks_n, uint32_t g, uint32_t p, uint64_t dh,
                                            uint64_t dl, uint64_t xh, uint64_t xl, uint64_t ad,
                                            uint32_t idesc, uint32_t acc_first) {
  switch (ks_n) {
    case 4: mma_ss_hi<4>(g, p, dh, dl, xh, xl, ad, idesc, acc_first); break;
    case 3: mma_ss_hi<3>(g, p, dh, dl, xh, xl, ad, idesc, acc_first); break;
    case 2: mma_ss_hi<2>(g, p, dh, dl, xh, xl, ad, idesc, acc_first); break;
    default: mma_ss_hi<1>(g, p, dh, dl, xh, xl, ad, idesc, acc_first); break;
  }
}
__device__ __forceinline__ void mma_ss_lo_n(int ks_n, uint32_t g, uint32_t p, uint64_t dh,
                                            uint64_t xh, uint64_t ad, uint32_t idesc) {
  switch (ks_n) {
    case 4: mma_ss_lo<4>(g, p, dh, xh, ad, idesc); break;
    case 3: mma_ss_lo<3>(g, p, dh, xh, ad, idesc); break;
    case 2: mma_ss_lo<2>(g, p, dh, xh, ad, idesc); break;
    default: mma_ss_lo<1>(g, p, dh, xh, ad, idesc); break;
  }
}

// K steps (16 FP16 each) in the last 64-column chunk of the operands: 1..4.
__host__ __device__ inline int last_chunk_steps(int kdim, int k_chunks) {
  return (kdim - (k_chunks - 1) * kTcKChunk) / kTcK;
}

// 32 consecutive 32-bit columns of this warp's 32 TMEM lanes from registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
      "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]),
      "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]),
      "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// The two halves of cluster_sync_all, for work that fits between them.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

__device__ __forceinline__ float ld_dsmem_f32(const float* local, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
  return v;
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes, one load.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// One walker's running chord over a scan of rows (Algorithm 2's lambda_min /
// lambda_max from the ratios r_i = s_i / g_i, s_i >= 0).  Branch-free and
// select-free: r_i = s_i * rcp(g_i) is formed for every row and folded in by
// integer min over its bit pattern --
//   lambda_max = min over r >= 0 (g > 0): the unsigned min of the bits, where
//     every negative float (sign bit set) and NaN ranks above +Inf;
//   lambda_min = max over r <= 0 (g < 0): the signed min of the bits, where
//     every non-negative float ranks above -Inf and, among negative floats,
//     a smaller magnitude gives a smaller signed integer (-0 is the least).
// g = 0 gives r = +-Inf or NaN, which never wins; s = +0 (clamp_slack) gives
// r = +0 (g > 0) or -0 (g < 0), a chord end at the point itself.  The result is the exact
// min (max) of the rounded ratios whatever the order or split of the scan,
// so different launch shapes give the same bits.
struct ChordAcc {
  unsigned int hib;   // bits of lambda_max (starts at +Inf)
  int lob;            // bits of lambda_min (starts at -Inf)

  __device__ __forceinline__ void init() {
    hib = 0x7f800000u;
    lob = static_cast<int>(0xff800000u);
  }
  __device__ __forceinline__ void add(float ss, float gg) {
    float rg;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rg) : "f"(gg));
    const float r = ss * rg;
    hib = min(hib, __float_as_uint(r));
    lob = min(lob, __float_as_int(r));
  }
  __device__ __forceinline__ float lo_all() const { return __int_as_float(lob); }
  __device__ __forceinline__ float hi_all() const { return __uint_as_float(hib); }
};

// Brings one 128-byte line into L1 ahead of its use.  The chord epilogue
// prefetches the four lines of a 32-row block (row_block below: b_i, Ks, Kg,
// the form flag), one per lane of lanes 0..3: L1 does not keep them from one
// launch to the next, and each line missed costs the epilogue -- which sets
// the pace of a tile when the MMAs are short -- an L2 round trip.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Slack clamped at +0: an integer max over the bit pattern sends every
// negative value, -0 included, to +0 (the chord scan's sign rule needs s to
// be +0, never -0: s = -0 over g > 0 would read as a lambda_min).
__device__ __forceinline__ float clamp_slack(float s) {
  return __int_as_float(max(__float_as_int(s), 0));
}

// Per-row data of the chord epilogue, in blocks of 32 rows: block g (rows
// 32 g .. 32 g + 31) is 128 floats -- b_i / scale_i, then Ks_i, then Kg_i,
// then the block's bound form (0: 2-norms, 1: max-norms) -- so one pointer
// serves all of it (rows in the units of the row's power-of-two scale):
//   b_i / scale_i, lowered by 2^-21 |b_i / scale_i| (the relative rounding of
//       this value, the slack FMA, the ratio and theta)
//   Ks: bound on |computed - exact| of p_i = a_i . x per unit of the walker's
//       ws |x_hat| (2-norm form: ws ||x_hat||_2; max-norm form: ws, since
//       max |x_hat| < 1)
//   Kg: bound on |computed - exact| of g_i = a_i . d per unit of |d_hat|
//       (||d_hat||_2 or max |d_hat_i|)
// Both cover the representation error of the FP16 pair of row i (exact,
// from the split), the dropped lo.lo product, the point's own split and the
// FP32 accumulation of the MMA chain in tensor memory.  See prepare_tc_kernel
// in kernels_simt.cu.  `row0` below is always a multiple of 32.
__device__ __forceinline__ const float* row_block(const float* rows, int row0) {
  return rows + (row0 >> 5) * 128;
}

// The walker factors of a 32-row block: (ws ||x_hat||_2, ||d_hat||_2) or
// (ws, max |d_hat|) by the block's form.
struct WalkerNorms {
  float nxw2, nd2, ws, ndinf;
  __device__ __forceinline__ void pick(const float* rows, int row0, float& fx, float& fd) const {
    const bool inf = __ldg(row_block(rows, row0) + 96) != 0.0f;
    fx = inf ? ws : nxw2;
    fd = inf ? ndinf : nd2;
  }
};

// Slack of one walker at 32 rows from its P = X A^T columns (in place):
// s_i = b_i - p_i ws - Ks_i nxw, clamped at 0 -- Lemma 4.2's s = b - A x,
// lowered by the bound on its rounding error so that a chord end computed
// from it never lies outside the facet (nxw = ws ||x_hat||_2 of the walker).
__device__ __forceinline__ void slack32(float (&v)[32], const float* rows, int row0, float ws,
                                        float nxw) {
  const float4* b4 = reinterpret_cast<const float4*>(row_block(rows, row0));
  const float4* k4 = b4 + 8;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 b = __ldg(b4 + i);
    const float4 kk = __ldg(k4 + i);
    const float bb[4] = {b.x, b.y, b.z, b.w};
    const float ks[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float sv = fmaf(-v[4 * i + j], ws, bb[j]);
      sv = fmaf(-ks[j], nxw, sv);
      v[4 * i + j] = clamp_slack(sv);
    }
  }
}

// The chord scan over 32 rows: slacks s (from slack32) against G = D A^T,
// each g_i pushed away from zero by its error bound Kg_i nd (nd = ||d_hat||_2
// of the walker), so that s / g never exceeds the exact ratio of the lowered
// slack.  G and the slacks are finite: the FP16 operands are (the splits of
// the points and directions flag any value beyond the FP16 range) and so is
// every sum of their products.
__device__ __forceinline__ void scan32(const float (&s)[32], const float (&g)[32],
                                       const float* rows, int row0, float nd, ChordAcc& acc) {
  const float4* k4 = reinterpret_cast<const float4*>(row_block(rows, row0)) + 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 kk = __ldg(k4 + i);
    const float kg[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float gg = g[4 * i + j];
      const float sd = __int_as_float(__float_as_int(nd) | (__float_as_int(gg) & 0x80000000));
      acc.add(s[4 * i + j], fmaf(kg[j], sd, gg));
    }
  }
}

// Bound on the 2-norm of one walker's scaled operand from its FP16 hi part
// (sum of squares in FP32): ||v|| <= ||v_hi|| (1 + 2^-11) for the FP16 pair,
// and the FP32 sum of at most 1024 squares and the square root stay well
// inside the (1 + 2^-8) factor.  The same factor bounds max |v| from max |v_hi|.
__device__ __forceinline__ float norm_bound(float sumsq) {
  return sqrtf(sumsq) * 1.00390625f;
}

// Largest |value| of 8 FP16 values packed in a uint4.
__device__ __forceinline__ float absmax8(uint4 u) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
  float mx = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[e]));
    mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
  }
  return mx;
}

// Sum of squares of 8 FP16 values packed in a uint4.
__device__ __forceinline__ float sumsq8(uint4 u) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
  float acc = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[e]));
    acc = fmaf(f.x, f.x, acc);
    acc = fmaf(f.y, f.y, acc);
  }
  return acc;
}

template <int kThreads>
__device__ __forceinline__ void named_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

// Tensor maps and launch shape of one context, shared by both modes.
struct TcPlan {
  CUtensorMap ah, al, dh, dl, xh, xl;
  CUtensorMap dh2, dl2;  // recompute mode: the second direction pair
  CUtensorMap ah64, al64;   // A pair with 64-row boxes (TMEM-operand kernel)
  int C = 1;
  int tiles_per_cta = 1;
  int m_tiles = 1;
  int strips = 1;
};

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 2D FP16 map over a (rows x cols) row-major array with 128 x 64 boxes and
// the 128-byte swizzle the MMA descriptors expect.
inline bool make_map_rows(CUtensorMap* map, const void* ptr, int cols, int rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcKChunk), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

inline bool make_map(CUtensorMap* map, const void* ptr, int cols, int rows) {
  return make_map_rows(map, ptr, cols, rows, 128);
}

}  // namespace tc
}  // namespace mhar
