// Strided passes of an n^3 transform restricted to the 2/3-rule set (the
// dealiasing of Sec. 2.2: modes with 3|k| >= n on any axis are zero), for
// the convection solver (its z pass is fused with the products, rbc.cu).
//
// Inverse (spectrum -> real): the x pass reads only the kept k_x rows of the
// kept (k_y, k_z) columns and writes whole x lines; the y pass reads the kept
// k_y rows of the kept k_z columns for every x and writes whole y lines; the
// z pass then reads k_z < kc.  Each pass reads exactly what the previous one
// wrote.  Forward: after a z pass that writes k_z < kc, the y pass reads
// whole y lines of those columns and writes the kept k_y rows, the x pass
// writes the kept k_x rows of the kept columns; entries outside the kept set
// are left undefined.
#include <mutex>

#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {

__device__ __forceinline__ bool pr_kept(int a, int n, int kd) { return a <= kd || a >= n - kd; }

// index of the d-th kept x/y row (d in [0, 2kd]): 0..kd, then n-kd..n-1
__device__ __forceinline__ int pr_dense(int d, int n, int kd) { return d <= kd ? d : n - (2 * kd + 1 - d); }

template <int N>
struct PCfg {
  static constexpr int G = elems_per_thread(N);
  static constexpr int S = N / G;
  static constexpr int T = S <= 16 ? 256 / S : (S <= 64 ? 16 : 1024 / S);
  static constexpr int THREADS = T * S;
  static constexpr int MINB = THREADS <= 512 ? 2 : 1;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)N * T;
};

// XPASS: lines along x (row stride n h1), columns (dense k_y, k_z < kc);
// otherwise lines along y (row stride h1), columns (x, k_z < kc).
template <int N, int SIGN, bool XPASS>
__global__ void __launch_bounds__(PCfg<N>::THREADS, PCfg<N>::MINB)
    k_pcpass(const float2* in, float2* out, int ktiles, int outer, const float2* __restrict__ tw, float scale) {
  using C = PCfg<N>;
  constexpr int G = C::G, S = C::S, T = C::T;
  constexpr long long H1 = N / 2 + 1, M = (long long)N * N * H1;
  constexpr int KD = (N - 1) / 3, KC = KD + 1;
  extern __shared__ float2 smp[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const long long blk = blockIdx.x;
  const long long bo = blk / ktiles;  // batch * outer + o
  const int kt = (int)(blk - bo * ktiles);
  const long long b = bo / outer;
  const int o = (int)(bo - b * outer);
  const int kz = kt * T + c;
  const bool valid = kz < KC;
  const long long rs = XPASS ? (long long)N * H1 : H1;
  const long long base = b * M + (XPASS ? (long long)pr_dense(o, N, KD) * H1 : (long long)o * N * H1) + kz;
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int row = j + m * S;
    const bool rd = valid && (SIGN < 0 || pr_kept(row, N, KD));
    v[m] = rd ? in[base + row * rs] : make_float2(0.f, 0.f);
  }
  fft_line<N, G, SIGN>(v, j, ColX<T>{smp, c}, tw);
  if (valid) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int row = j + m * S;
      if (SIGN > 0 || pr_kept(row, N, KD)) out[base + row * rs] = cscale(v[m], scale);
    }
  }
}

template <int N, int SIGN, bool XPASS>
static cudaError_t pcpass_n(fftk_plan p, const float2* in, float2* out, long long B, float scale, cudaStream_t st) {
  using C = PCfg<N>;
  static PerDevice once;
  const cudaError_t attr_err = once.run([](int) {
    return cudaFuncSetAttribute(k_pcpass<N, SIGN, XPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  constexpr int KD = (N - 1) / 3, KC = KD + 1;
  const int ktiles = (KC + C::T - 1) / C::T;
  const int outer = XPASS ? 2 * KD + 1 : N;
  const long long blocks = B * outer * ktiles;
  LaunchScope ls(p, XPASS ? (SIGN < 0 ? KK_X_FWD : KK_X_INV) : (SIGN < 0 ? KK_Y_FWD : KK_Y_INV), st);
  k_pcpass<N, SIGN, XPASS><<<(unsigned)blocks, C::THREADS, C::SMEM, st>>>(in, out, ktiles, outer, twiddles(p, N),
                                                                         scale);
  return cudaGetLastError();
}

#define FFTK_PRUNED_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

cudaError_t launch_pruned_x(fftk_plan p, int sign, const float2* in, float2* out, long long B, float scale,
                            cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
#define CASE(n)                                                                          \
  case n:                                                                                \
    return sign < 0 ? pcpass_n<n, -1, true>(p, in, out, B, scale, st)                   \
                    : pcpass_n<n, +1, true>(p, in, out, B, scale, st);
  switch (p->nx) { FFTK_PRUNED_SIZES(CASE) }
#undef CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_pruned_y(fftk_plan p, int sign, const float2* in, float2* out, long long B, float scale,
                            cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
#define CASE(n)                                                                          \
  case n:                                                                                \
    return sign < 0 ? pcpass_n<n, -1, false>(p, in, out, B, scale, st)                  \
                    : pcpass_n<n, +1, false>(p, in, out, B, scale, st);
  switch (p->ny) { FFTK_PRUNED_SIZES(CASE) }
#undef CASE
  return cudaErrorInvalidValue;
}

}  // namespace fftk
