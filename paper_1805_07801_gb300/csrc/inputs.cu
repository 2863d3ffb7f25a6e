// Counter-based pseudo-random fields for synthetic workloads.
//
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a counter-based
// generator: output c of the stream started at state 0 is
// mix64((c + 1) * 0x9E3779B97F4A7C15).  Written from the published
// description; the tests check it against an independent numpy copy.
#include <cuda_runtime.h>

#include "internal.h"

namespace fftk {

fftk_status from_cuda(cudaError_t e);

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long splitmix_at(unsigned long long c) {
  return mix64((c + 1ull) * 0x9E3779B97F4A7C15ull);
}

__global__ void k_fill_normal(float* __restrict__ out, long long count, unsigned long long base) {
  const double two_pi = 6.283185307179586476925286766559;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long c = base + 2ull * (unsigned long long)i;
    const unsigned long long x1 = splitmix_at(c), x2 = splitmix_at(c + 1ull);
    const double u1 = ((double)(x1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(x2 >> 11) * 0x1.0p-53;
    out[i] = (float)(sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
  }
}

__global__ void k_fill_uniform(float* __restrict__ out, long long count, unsigned long long base) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long x = splitmix_at(base + (unsigned long long)i);
    const double u = (double)(x >> 40) * 0x1.0p-24;
    out[i] = (float)(2.0 * u - 1.0);
  }
}

static fftk_status fill_check(float* dev, long long count, int seed, int field, bool pairs) {
  if (!dev || count < 0 || seed < 0 || seed >= (1 << 24) || field < 0 || field >= 16)
    return FFTK_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(dev) & 3u) != 0) return FFTK_ERR_INVALID_ARG;
  const long long lim = 1LL << 36;
  if ((pairs ? 2 * count : count) > lim) return FFTK_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return FFTK_ERR_NO_DEVICE;
  }
  return FFTK_OK;
}

}  // namespace fftk

using namespace fftk;

extern "C" fftk_status fftk_fill_normal(float* dev, long long count, int seed, int field,
                                        void* cuda_stream) {
  fftk_status s = fill_check(dev, count, seed, field, true);
  if (s != FFTK_OK || count == 0) return s;
  const unsigned long long base = ((unsigned long long)seed << 40) | ((unsigned long long)field << 36);
  k_fill_normal<<<152 * 8, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(dev, count, base);
  return from_cuda(cudaGetLastError());
}

extern "C" fftk_status fftk_fill_uniform(float* dev, long long count, int seed, int field,
                                         void* cuda_stream) {
  fftk_status s = fill_check(dev, count, seed, field, false);
  if (s != FFTK_OK || count == 0) return s;
  const unsigned long long base = ((unsigned long long)seed << 40) | ((unsigned long long)field << 36);
  k_fill_uniform<<<152 * 8, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(dev, count, base);
  return from_cuda(cudaGetLastError());
}
