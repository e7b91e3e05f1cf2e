"""The oracle's Philox4x32-10 against a library implementation on the GPU.

The oracle's block function (Salmon et al. 2011) is pinned on the CPU by the
published known-answer vectors; here it is also compared, word for word, with
cuRAND's device Philox4x32-10 (curand_Philox4x32_10 from curand_kernel.h) over
random counters and keys and over the counter layout the sampler uses
(q, walker, step_lo, step_hi << 8 | stream).  The library kernels draw their
directions from the same block function: their FP64 walks match the oracle's
to 1e-10 only with bit-equal words (tests/test_gpu_parity.py), so this closes
the chain oracle == cuRAND == library.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include <curand_kernel.h>

__global__ void blocks(const uint4* ctr, const uint2* key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "rb");
  int n = 0;
  if (!f || std::fread(&n, sizeof(int), 1, f) != 1) return 2;
  std::vector<uint4> c(n);
  std::vector<uint2> k(n);
  std::vector<uint4> o(n);
  if (std::fread(c.data(), sizeof(uint4), n, f) != static_cast<size_t>(n)) return 3;
  if (std::fread(k.data(), sizeof(uint2), n, f) != static_cast<size_t>(n)) return 4;
  std::fclose(f);
  uint4 *dc, *dout;
  uint2* dk;
  if (cudaMalloc(&dc, n * sizeof(uint4)) || cudaMalloc(&dk, n * sizeof(uint2)) ||
      cudaMalloc(&dout, n * sizeof(uint4)))
    return 5;
  cudaMemcpy(dc, c.data(), n * sizeof(uint4), cudaMemcpyHostToDevice);
  cudaMemcpy(dk, k.data(), n * sizeof(uint2), cudaMemcpyHostToDevice);
  blocks<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
  if (cudaMemcpy(o.data(), dout, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 6;
  f = std::fopen(argv[2], "wb");
  std::fwrite(o.data(), sizeof(uint4), n, f);
  std::fclose(f);
  return 0;
}
"""


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_oracle_philox_matches_curand(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "philox_curand.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "philox_curand"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    rng = np.random.default_rng(2104)
    n_rand = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n_rand, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n_rand, 2), dtype=np.uint64).astype(np.uint32)
    # The sampler's own layouts: direction blocks q of walker k at step s,
    # streams 0..3, seeds 0 and 2^40 + 7 (both key words in use).
    lay_c, lay_k = [], []
    for seed in (0, (1 << 40) + 7):
        for step in (0, 1, 63, (1 << 32) + 5):
            for walker in (0, 1, 4095, 70000):
                for stream in range(4):
                    for q in (0, 1, 24):
                        lay_c.append([q, walker, step & 0xFFFFFFFF, ((step >> 32) << 8) | stream])
                        lay_k.append([seed & 0xFFFFFFFF, seed >> 32])
    ctr = np.vstack([ctr, np.array(lay_c, dtype=np.uint32)])
    key = np.vstack([key, np.array(lay_k, dtype=np.uint32)])
    n = ctr.shape[0]
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.int32(n).tobytes())
        f.write(np.ascontiguousarray(ctr).tobytes())
        f.write(np.ascontiguousarray(key).tobytes())
    out = tmp_path / "out.bin"
    subprocess.run([str(exe), str(inp), str(out)], check=True, timeout=120)
    got = np.fromfile(out, dtype=np.uint32).reshape(n, 4)
    want = np.array([oracle.philox(ctr[i], key[i]) for i in range(n)], dtype=np.uint32)
    np.testing.assert_array_equal(got, want)
