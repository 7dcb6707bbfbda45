// Test helper: raw Philox4x32-10 words from cuRAND's documented device API,
// an implementation independent of this repository, for pinning the oracle.
// curand_init(seed, subsequence, 0) keys the generator with the 64-bit seed
// and starts the 128-bit counter at subsequence * 2^64; skipahead(4 a) moves
// it on by a (in steps below 2^60, since the offset counts 32-bit outputs);
// curand4() returns the four words of the current counter.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_words(uint64_t seed, const uint64_t *lo64, const uint64_t *hi64, int n, uint4 *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, hi64[i], 0ull, &st);  // counter = hi64 * 2^64
  unsigned long long left = lo64[i];
  while (left > 0) {  // at most 16 steps
    const unsigned long long a = left < (1ull << 60) ? left : (1ull << 60);
    skipahead(4ull * a, &st);
    left -= a;
  }
  out[i] = curand4(&st);
}

extern "C" int curand_philox_words(uint64_t seed, const uint64_t *lo64, const uint64_t *hi64, int n,
                                   uint32_t *out_host) {
  uint64_t *dlo = nullptr, *dhi = nullptr;
  uint4 *dout = nullptr;
  if (cudaMalloc(&dlo, n * sizeof(uint64_t)) != cudaSuccess) return 1;
  if (cudaMalloc(&dhi, n * sizeof(uint64_t)) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, n * sizeof(uint4)) != cudaSuccess) return 1;
  cudaMemcpy(dlo, lo64, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
  cudaMemcpy(dhi, hi64, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
  k_words<<<(n + 127) / 128, 128>>>(seed, dlo, dhi, n, dout);
  cudaError_t e = cudaMemcpy(out_host, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost);
  cudaFree(dlo);
  cudaFree(dhi);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 2;
}
