// noalloc.cu -- mhar_chord_noalloc: the chord computation (lambda_min,
// lambda_max per walker) for callers that must not allocate device memory.
//
// Who needs this: code that owns a fixed device-memory budget (a serving
// process that reserves its pool up front, an allocator-managed framework)
// cannot let a library call cudaMalloc behind its back, and latency-critical
// loops cannot afford the device-wide synchronisation that cudaMalloc and
// cudaFree may imply.  This entry point therefore takes only caller-owned
// inputs and outputs and keeps its one piece of working memory -- the
// per-walker ordered keys the blocks fold their partial chords into -- in a
// fixed array compiled into the library.
//
// The array is a file-scope static __device__ buffer: every GPU that loads the
// library holds it (1 MiB) until the process exits.  Host code cannot use the
// symbol itself as a device address; the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it, so that first call should come before any stream capture.  All calls
// share the array and it keeps the last call's contents: each call clears the
// keys it uses before the kernel runs, and calls whose work overlaps on the GPU
// (different streams, or host threads racing) corrupt each other's results.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mhar_device.cuh"
#include "mhar_internal.h"

namespace {

constexpr int kNoAllocMaxWalkers = 65536;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;
constexpr unsigned long long kBadKey = ~0ull;   // a walker that met a non-finite value

// Keys [0, max) fold lambda_min (atomic max), keys [max, 2 max) lambda_max
// (atomic min).
static __device__ __align__(256) unsigned long long g_chord_scratch[2 * kNoAllocMaxWalkers];

std::mutex g_setup_mu;
unsigned long long* g_scratch_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double ninf() { return -__longlong_as_double(0x7ff0000000000000ll); }
__device__ __forceinline__ double pinf() { return __longlong_as_double(0x7ff0000000000000ll); }

__global__ void noalloc_clear_kernel(int z, unsigned long long* keys) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < z) {
    keys[k] = mhar::f64_key(ninf());
    keys[kNoAllocMaxWalkers + k] = mhar::f64_key(pinf());
  }
}

// The chord of every walker on caller buffers: A (m x n), X and D (z x n),
// all FP64 row-major with no padding.  For each row, the slack b_i - a_i . x
// (counted as 0 when rounding makes it negative) over a_i . d gives one end
// of the walker's chord; rows with a_i . d == 0 give none.  Tiles of 64 rows
// x 64 walkers; every block folds its rows into the per-walker keys.  A
// non-finite slack or product marks the walker (its lambda_min key becomes
// kBadKey) and both of its chord ends come out NaN.
__global__ void __launch_bounds__(kThreads)
noalloc_chord_kernel(const double* __restrict__ A, const double* __restrict__ b,
                     const double* __restrict__ X, const double* __restrict__ D, int m, int n,
                     int z, unsigned long long* keys) {
  constexpr int BK = 8;
  __shared__ double As[BK][64];
  __shared__ double Xs[BK][64];
  __shared__ double Ds[BK][64];
  __shared__ double red_lo[16][64];
  __shared__ double red_hi[16][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * 64, w0 = blockIdx.y * 64;
  double accS[4][4], accG[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) { accS[r][c] = 0.0; accG[r][c] = 0.0; }
  for (int k0 = 0; k0 < n; k0 += BK) {
    for (int e = tid; e < 64 * BK; e += kThreads) {
      const int r = e / BK, c = e - r * BK;
      const int gi = i0 + r, gw = w0 + r, kc = k0 + c;
      const bool kin = kc < n;
      As[c][r] = (gi < m && kin) ? A[static_cast<size_t>(gi) * n + kc] : 0.0;
      Xs[c][r] = (gw < z && kin) ? X[static_cast<size_t>(gw) * n + kc] : 0.0;
      Ds[c][r] = (gw < z && kin) ? D[static_cast<size_t>(gw) * n + kc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], xv[4], dv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) { xv[c] = Xs[kk][tx + 16 * c]; dv[c] = Ds[kk][tx + 16 * c]; }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          accS[r][c] += a[r] * xv[c];
          accG[r][c] += a[r] * dv[c];
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double lo = ninf(), hi = pinf();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gi = i0 + ty * 4 + r;
      if (gi >= m) continue;
      double s = b[gi] - accS[r][c];
      const double g = accG[r][c];
      if (!isfinite(s) || !isfinite(g)) {
        lo = __longlong_as_double(0x7ff8000000000000ll);   // NaN: the walker is marked
        hi = lo;
        break;
      }
      if (s < 0.0) s = 0.0;
      if (g > 0.0) {
        const double lam = s / g;
        hi = lam < hi ? lam : hi;
      } else if (g < 0.0) {
        const double lam = s / g;
        lo = lam > lo ? lam : lo;
      }
    }
    red_lo[ty][tx + 16 * c] = lo;
    red_hi[ty][tx + 16 * c] = hi;
  }
  __syncthreads();
  if (tid < 64) {
    double lo = red_lo[0][tid], hi = red_hi[0][tid];
    bool bad = isnan(lo);
#pragma unroll
    for (int t = 1; t < 16; ++t) {
      bad = bad || isnan(red_lo[t][tid]);
      lo = red_lo[t][tid] > lo ? red_lo[t][tid] : lo;
      hi = red_hi[t][tid] < hi ? red_hi[t][tid] : hi;
    }
    const int gw = w0 + tid;
    if (gw < z) {
      if (bad) {
        // The all-ones key is the largest, so no later atomicMax undoes it.
        atomicMax(&keys[gw], kBadKey);
      } else {
        if (!isinf(lo)) atomicMax(&keys[gw], mhar::f64_key(lo));
        if (!isinf(hi)) atomicMin(&keys[kNoAllocMaxWalkers + gw], mhar::f64_key(hi));
      }
    }
  }
}

__global__ void noalloc_finish_kernel(int z, const unsigned long long* keys, double* lmin,
                                      double* lmax) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < z) {
    const unsigned long long klo = keys[k], khi = keys[kNoAllocMaxWalkers + k];
    const bool bad = klo == kBadKey;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    lmin[k] = bad ? nan : mhar::f64_unkey(klo);
    lmax[k] = bad ? nan : mhar::f64_unkey(khi);
  }
}

int fail(int code, const char* msg) {
  char buf[320];
  snprintf(buf, sizeof(buf), "mhar_chord_noalloc: %s", msg);
  mhar::set_null_error(buf);
  return code;
}

// Device address of the scratch array for the current device (looked up once
// per device, with that device current).
int scratch_for_current_device(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MHAR_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MHAR_E_UNSUPPORTED, "device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_chord_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MHAR_E_CUDA, cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MHAR_OK;
}

}  // namespace

extern "C" int mhar_chord_noalloc(const double* A, const double* b, int m, int n, const double* X,
                                  const double* D, int z, double* lmin, double* lmax,
                                  void* stream) {
  if (!A || !b || !X || !D || !lmin || !lmax || m < 1 || n < 1 || z < 1)
    return fail(MHAR_E_ARG, "null pointer or non-positive size");
  if (z > kNoAllocMaxWalkers) {
    char msg[160];
    snprintf(msg, sizeof(msg), "z = %d exceeds the fixed scratch capacity of %d walkers", z,
             kNoAllocMaxWalkers);
    return fail(MHAR_E_ARG, msg);
  }
  // An error left pending by earlier, unrelated work is not this call's: report
  // it as such and launch nothing (it stays pending for its owner).
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "a CUDA error was already pending before the call (%s); nothing launched",
             cudaGetErrorString(e));
    return fail(MHAR_E_CUDA, msg);
  }
  unsigned long long* keys = nullptr;
  int rc = scratch_for_current_device(&keys);
  if (rc != MHAR_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  noalloc_clear_kernel<<<(z + kThreads - 1) / kThreads, kThreads, 0, s>>>(z, keys);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(MHAR_E_CUDA, cudaGetErrorString(e));
  dim3 grid((m + 63) / 64, (z + 63) / 64);
  noalloc_chord_kernel<<<grid, kThreads, 0, s>>>(A, b, X, D, m, n, z, keys);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(MHAR_E_CUDA, cudaGetErrorString(e));
  noalloc_finish_kernel<<<(z + kThreads - 1) / kThreads, kThreads, 0, s>>>(z, keys, lmin, lmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(MHAR_E_CUDA, cudaGetErrorString(e));
  mhar::set_null_error(nullptr);
  return MHAR_OK;
}
