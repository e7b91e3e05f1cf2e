// mhar_device.cuh -- device helpers shared by the MHAR kernels.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the
// counter-based generator both the kernels and the test oracle implement
// independently from its published definition.  Counter layout of one block:
//   ctr = (q, walker, step_lo32, (step_hi24 << 8) | stream),  key = (seed_lo, seed_hi)
// stream 0 draws direction entries (quad q covers coordinates 4q..4q+3),
// stream 1 draws the chord uniform (q = 0, word 0), stream 2 the r low-rank
// normals g of a preconditioned direction, stream 3 the starting block of the
// preconditioner fit (column c drawn as walker c at step 0).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mhar {

constexpr uint32_t kStreamDirection = 0u;
constexpr uint32_t kStreamChord = 1u;
constexpr uint32_t kStreamLowRank = 2u;
constexpr uint32_t kStreamFit = 3u;
constexpr int kMaxPcRank = 32;  // columns of the low-rank factor U
// Largest finite FP16 value: a value split into an FP16 pair must stay within
// it (beyond it the pair would be infinite and so would the products).
constexpr float kHalfMax = 65504.0f;

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ U4 philox_block(uint64_t seed, uint64_t step, uint32_t walker,
                                           uint32_t q, uint32_t stream) {
  U4 c{q, walker, static_cast<uint32_t>(step),
       (static_cast<uint32_t>((step >> 32) & 0xffffffu) << 8) | (stream & 0xffu)};
  return philox4x32_10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// (w + 1/2) 2^-32: exact in FP64, strictly inside (0,1).
__device__ __forceinline__ double open_unit_f64(uint32_t w) {
  return (static_cast<double>(w) + 0.5) * 2.3283064365386963e-10;
}

// Box-Muller pair from two open uniforms.
__device__ __forceinline__ void box_muller_f64(double ua, double ub, double& z0, double& z1) {
  const double r = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// (w + 1/2) 2^-32 rounded once to FP32, without FP64 arithmetic: the high 24
// bits times 256 are exact in FP32 and the low byte plus 1/2 is exact, so
// their FP32 sum is the correctly rounded w + 1/2 (and scaling by 2^-32 is
// exact).  Equals (float)open_unit_f64(w).
__device__ __forceinline__ float open_unit_f32(uint32_t w) {
  const float hi = __uint2float_rn(w >> 8) * 256.0f;
  const float lo = __uint2float_rn(w & 0xffu) + 0.5f;
  return (hi + lo) * 2.3283064365386963e-10f;
}

// FP32 variant: the same uniforms as the FP64 path, rounded once; log and
// sincospi in FP32.
__device__ __forceinline__ void box_muller_f32(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float ua = open_unit_f32(wa);
  const float ub = open_unit_f32(wb);
  // ua rounds to 1.0f only for wa >= 2^32 - 128; log then gives 0 (radius 0),
  // a valid draw.
  const float r = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Offset of element (walker k, coordinate i) of a tensor-core walker operand
// (FP16 pair of D or X): row-major k * k_pad + i, or interleaved by 8-element
// chunks, ((i / 8) z_ld + k) 8 + i % 8, so that the same chunk of consecutive
// walkers is contiguous (one 512-byte line for a warp's 32 walkers).
__device__ __forceinline__ size_t op_off(int k, int i, int k_pad, int z_ld, int inter) {
  return inter ? ((static_cast<size_t>(i >> 3) * z_ld + k) << 3) + (i & 7)
               : static_cast<size_t>(k) * k_pad + i;
}

// ---- ordered keys for floating-point atomic min / max ---------------------
// Monotone map: a < b  <=>  key(a) < key(b) (as unsigned), for non-NaN values.
__device__ __forceinline__ unsigned long long f64_key(double f) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(f));
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double f64_unkey(unsigned long long k) {
  const unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(static_cast<long long>(u));
}

// 1 / sigma for a coordinate scale sigma = 2^e, -126 <= e <= 126 (every
// scale is a power of two in that range, 1 past n; set_sigma checks it): the
// exponent negated, exactly, so x * pow2_recip(sigma) has the bits of
// x / sigma.
__device__ __forceinline__ float pow2_recip(float sigma) {
  return __int_as_float(0x7f000000 - __float_as_int(sigma));
}

// ---- double-float (pairs of FP32) arithmetic --------------------------------
// Knuth's TwoSum and Dekker's FastTwoSum; TwoProd via FMA.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (hi, lo) += t * d  with the product and the sum carried exactly to ~2^-46.
__device__ __forceinline__ void df_axpy(float& hi, float& lo, float t, float d) {
  const float p = t * d;
  const float pe = fmaf(t, d, -p);
  float s, e;
  two_sum(hi, p, s, e);
  e += lo + pe;
  fast_two_sum(s, e, hi, lo);
}

}  // namespace mhar
