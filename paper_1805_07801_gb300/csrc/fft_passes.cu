// The three 1D pass kinds of the 3D transform (paper Sec. 3): the z pass
// (real <-> half complex, contiguous lines) and the strided complex pass used
// for y and x.  The paper's MPI_Alltoall exchanges between passes are absent:
// every pass reads its lines in place, batched across the contiguous index
// (the transpose-free layout of Appendix A), so no reorder pass exists.
#include <mutex>

// these passes are bound by their 8-byte global accesses; scalar FP32 sums
// measured faster here than the paired ones (see fft_engine.cuh)
#define FFTK_PAIRED_FP32 0
#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {

// ------------------------------------------------------------------ z pass --
template <int N>
struct ZCfg {
  static constexpr int H = N / 2;                  // complex length of the packed line
  static constexpr int G = elems_per_thread(H);
  static constexpr int S = H / G;                  // threads per line
  static constexpr int LPC = S >= 256 ? 1 : 256 / S;  // lines per CTA
  static constexpr int THREADS = LPC * S;
  static constexpr bool WARP = S <= 32;
  static constexpr int MINB = 4;  // 32 warps per SM at <= 64 registers
};

// Real-to-complex along z.  The N reals of a line are packed as H = N/2
// complex values z[n] = x[2n] + i x[2n+1]; after the H-point transform Z,
//   X[k] = (Z[k] + conj Z[H-k])/2 + exp(-2 pi i k/N) (Z[k] - conj Z[H-k])/(2i),
// k = 0..H (Z[H] = Z[0]).
template <int N>
__global__ void __launch_bounds__(ZCfg<N>::THREADS, ZCfg<N>::MINB)
    k_z_r2c(const float* __restrict__ in, float2* __restrict__ out, long long nlines,
            const float2* __restrict__ tw, float scale) {  // tw: size-N table
  using C = ZCfg<N>;
  constexpr int H = C::H, G = C::G, S = C::S;
  constexpr int LOGN = Log2<N>::value;
  __shared__ float2 sm[C::LPC * H];
  const int li = threadIdx.x / S, j = threadIdx.x % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < nlines;
  const LineX<C::WARP> xc{sm + li * H};
  float2 v[G];
  const float2* src = reinterpret_cast<const float2*>(in + line * N);
#pragma unroll
  for (int m = 0; m < G; ++m) v[m] = valid ? src[j + m * S] : make_float2(0.f, 0.f);
  fft_line<H, G, -1, LOGN>(v, j, xc, tw);
#pragma unroll
  for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
  xc.sync();
  if (valid) {
    float2* dst = out + line * (H + 1);
    const float2 Wj = __ldg(&tw[j]);  // exp(-2 pi i k / N) = W_j exp(-2 pi i m / 2G), k = j + m S
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 A = v[m];
      const float2 Bc = cconj(xc.ld((H - k) & (H - 1)));
      const float2 E = cscale(cadd(A, Bc), 0.5f);
      const float2 D = csub(A, Bc);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // D / (2i)
      dst[k] = cscale(cadd(E, cmul(mul_root32(Wj, m * (16 / G)), O)), scale);
    }
    if (j == 0) dst[H] = make_float2((v[0].x - v[0].y) * scale, 0.f);
  }
}

// Complex-to-real along z: the inverse of the packing above.  With
// E = X[k] + conj X[H-k] and O = (X[k] - conj X[H-k]) exp(+2 pi i k/N),
// Z[k] = E + i O, and the unnormalised H-point inverse of Z gives
// x[2n] + i x[2n+1].  Im X[0] and Im X[H] are ignored (line-wise c2r).
template <int N>
__global__ void __launch_bounds__(ZCfg<N>::THREADS, ZCfg<N>::MINB)
    k_z_c2r(const float2* __restrict__ in, float* __restrict__ out, long long nlines,
            const float2* __restrict__ tw) {  // tw: size-N table
  using C = ZCfg<N>;
  constexpr int H = C::H, G = C::G, S = C::S;
  constexpr int LOGN = Log2<N>::value;
  __shared__ float2 sm[C::LPC * H];
  const int li = threadIdx.x / S, j = threadIdx.x % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < nlines;
  const LineX<C::WARP> xc{sm + li * H};
  const float2* src = in + line * (H + 1);
  // X[0..H-1] of the line pass through the exchange buffer once, so the
  // mirror X[H - k] is read from there instead of a second global load
  // (X[H] itself, the k = 0 mirror, is one broadcast load)
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    v[m] = valid ? src[j + m * S] : make_float2(0.f, 0.f);
    xc.st(j + m * S, v[m]);
  }
  const float2 XH = valid ? src[H] : make_float2(0.f, 0.f);
  const float2 Wj = __ldg(&tw[j]);  // exp(-2 pi i k / N) = W_j exp(-2 pi i m / 2G), k = j + m S
  xc.sync();
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int k = j + m * S;
    float2 A = v[m];
    float2 B = k == 0 ? XH : xc.ld(H - k);
    if (k == 0) {
      A.y = 0.f;
      B.y = 0.f;
    }
    const float2 Bc = cconj(B);
    const float2 E = cadd(A, Bc);
    const float2 O = cmulc(csub(A, Bc), mul_root32(Wj, m * (16 / G)));
    v[m] = make_float2(E.x - O.y, E.y + O.x);
  }
  xc.sync();  // every mirror has been read before the transform's exchanges
  fft_line<H, G, +1, LOGN>(v, j, xc, tw);
  if (valid) {
    float2* dst = reinterpret_cast<float2*>(out + line * N);
#pragma unroll
    for (int m = 0; m < G; ++m) dst[j + m * S] = v[m];
  }
}

// ------------------------------------------------------- strided c2c pass --
// Tile = T adjacent columns (contiguous index q) x the full line (L rows of
// stride Q).  Loads and stores are T-wide row segments, coalesced along q.
// Tile width T per line length: 32 warps per SM at <= 64 registers per
// thread (2 CTAs of 512 threads up to L = 512, one of 1024 beyond), and row
// segments of 128 bytes (T = 16) where the 227 KB of shared memory allows.
template <int L>
struct CCfg {
  static constexpr int G = elems_per_thread(L);
  static constexpr int S = L / G;
  static constexpr int T = S <= 16 ? 256 / S : (S <= 64 ? 16 : 1024 / S);
  static constexpr int THREADS = T * S;
  static constexpr int MINB = THREADS <= 512 ? 2 : 1;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)L * T;
};

template <int L, int SIGN>
__global__ void __launch_bounds__(CCfg<L>::THREADS, CCfg<L>::MINB)
    k_cpass(const float2* in, float2* out, long long Q, long long qtiles,
            const float2* __restrict__ tw, float scale) {  // tw: size-L table
  using C = CCfg<L>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smc[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const long long tile = blockIdx.x;
  const long long p = tile / qtiles;
  const long long q = (tile - p * qtiles) * T + c;
  const bool valid = q < Q;
  const long long base = p * (long long)L * Q + q;
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m)
    v[m] = valid ? in[base + (long long)(j + m * S) * Q] : make_float2(0.f, 0.f);
  fft_line<L, G, SIGN>(v, j, ColX<T>{smc, c}, tw);
  if (valid) {
#pragma unroll
    for (int m = 0; m < G; ++m) out[base + (long long)(j + m * S) * Q] = cscale(v[m], scale);
  }
}

// ----------------------------------------------------------- launchers -----
template <int N>
static cudaError_t z_r2c_n(fftk_plan p, const float* in, float2* out, long long nl, float scale,
                           cudaStream_t st) {
  using C = ZCfg<N>;
  const long long blocks = (nl + C::LPC - 1) / C::LPC;
  LaunchScope ls(p, KK_Z_R2C, st);
  k_z_r2c<N><<<(unsigned)blocks, C::THREADS, 0, st>>>(in, out, nl, twiddles(p, N), scale);
  return cudaGetLastError();
}

template <int N>
static cudaError_t z_c2r_n(fftk_plan p, const float2* in, float* out, long long nl,
                           cudaStream_t st) {
  using C = ZCfg<N>;
  const long long blocks = (nl + C::LPC - 1) / C::LPC;
  LaunchScope ls(p, KK_Z_C2R, st);
  k_z_c2r<N><<<(unsigned)blocks, C::THREADS, 0, st>>>(in, out, nl, twiddles(p, N));
  return cudaGetLastError();
}

template <int L, int SIGN>
static cudaError_t cpass_l(fftk_plan p, const float2* in, float2* out, long long P, long long Q,
                           float scale, int kind, cudaStream_t st) {
  using C = CCfg<L>;
  static PerDevice once;
  const cudaError_t attr_err = once.run([](int) {
    return cudaFuncSetAttribute(k_cpass<L, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const long long qtiles = (Q + C::T - 1) / C::T;
  const long long blocks = P * qtiles;
  LaunchScope ls(p, kind, st);
  k_cpass<L, SIGN><<<(unsigned)blocks, C::THREADS, C::SMEM, st>>>(in, out, Q, qtiles, twiddles(p, L), scale);
  return cudaGetLastError();
}

#define FFTK_SIZES(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t launch_z_r2c(fftk_plan p, const float* in, float2* out, long long nlines, float scale,
                         cudaStream_t st) {
  if (nlines <= 0) return cudaSuccess;
  if (!is_pow2(p->nz)) return launch_z3(p, true, in, out, nlines, scale, st);
  switch (p->nz) {
#define CASE(n) \
  case n:       \
    return z_r2c_n<n>(p, in, out, nlines, scale, st);
    FFTK_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_z_c2r(fftk_plan p, const float2* in, float* out, long long nlines,
                         cudaStream_t st) {
  if (nlines <= 0) return cudaSuccess;
  if (!is_pow2(p->nz)) return launch_z3(p, false, in, out, nlines, 1.f, st);
  switch (p->nz) {
#define CASE(n) \
  case n:       \
    return z_c2r_n<n>(p, in, out, nlines, st);
    FFTK_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cpass(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P,
                         long long Q, float scale, int kind, cudaStream_t st) {
  if (P <= 0 || Q <= 0) return cudaSuccess;
  if (sign < 0) {
    switch (L) {
#define CASE(n) \
  case n:       \
    return cpass_l<n, -1>(p, in, out, P, Q, scale, kind, st);
      FFTK_SIZES(CASE)
#undef CASE
    }
  } else {
    switch (L) {
#define CASE(n) \
  case n:       \
    return cpass_l<n, +1>(p, in, out, P, Q, scale, kind, st);
      FFTK_SIZES(CASE)
#undef CASE
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftk
