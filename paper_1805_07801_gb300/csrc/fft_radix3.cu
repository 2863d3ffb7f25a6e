// Lines of length 3 * 2^m (the paper's 768^3, 1536^3, 3072^3 grids of the
// Cray XC40 runs, Sec. 5): one radix-3 step of Cooley and Tukey's
// decimation in time on top of the power-of-two engine.  With L = 3P,
//   Y_r = DFT_P(x[3j + r]),  r = 0, 1, 2,
//   X[k1 + P k2] = sum_r W_L^(r k1) W_3^(r k2) Y_r[k1],   k1 < P, k2 < 3
// (W_n = exp(-+2 pi i / n) with the transform's sign).  The three sub-lines
// run through the same register/shared-memory engine, each in its own
// exchange region; the radix-3 butterfly reads the three results of one k1
// from shared memory.
#include <mutex>

#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {

// exp(SIGN 2 pi i / 3) applied r times to a value: the radix-3 butterfly
// of (a, b, c) for output k2, b and c already twiddled by W_L^(k1), W_L^(2 k1)
template <int SIGN>
__device__ __forceinline__ float2 radix3_out(float2 a, float2 b, float2 c, int k2) {
  constexpr float h = 0.8660254037844386f;  // sin(pi / 3)
  if (k2 == 0) return make_float2(a.x + b.x + c.x, a.y + b.y + c.y);
  // W_3^k2 b + W_3^(2 k2) c with W_3 = -1/2 + SIGN i sqrt(3)/2
  const float sx = b.x + c.x, sy = b.y + c.y;   // b + c
  const float dx = b.x - c.x, dy = b.y - c.y;   // b - c
  const float s = (k2 == 1 ? 1.f : -1.f) * (float)SIGN * h;
  // a - (b + c)/2 + s i (b - c)
  return make_float2(a.x - 0.5f * sx - s * dy, a.y - 0.5f * sy + s * dx);
}

// twiddle exp(SIGN 2 pi i e / L) from the size-L table exp(-2 pi i m / L)
template <int SIGN>
__device__ __forceinline__ float2 tw3(const float2* __restrict__ t, int e) {
  const float2 w = __ldg(&t[e]);
  return SIGN < 0 ? w : make_float2(w.x, -w.y);
}

// ------------------------------------------------------ strided pass -----
template <int P>
struct C3Cfg {
  static constexpr int L = 3 * P;
  static constexpr int G = elems_per_thread(P);
  static constexpr int S = P / G;                        // threads per sub-line
  static constexpr int T = 3 * S <= 48 ? 16 : (3 * S <= 96 ? 8 : 4);  // columns per tile
  static constexpr int THREADS = T * 3 * S;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)L * T;
};

// One tile = T adjacent columns (contiguous index q) x the whole line of
// L = 3P rows of stride Q.  Thread (r, j, c): sub-line r of column c.
// tw: size-P table; t3: size-L table.
template <int P, int SIGN>
__global__ void __launch_bounds__(C3Cfg<P>::THREADS)
    k_cpass3(const float2* in, float2* out, long long Q, long long qtiles, const float2* __restrict__ tw,
             const float2* __restrict__ t3, float scale) {
  using C = C3Cfg<P>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 sm3[];
  const int c = threadIdx.x % T, q3 = threadIdx.x / T;
  const int r = q3 / S, j = q3 % S;
  const long long tile = blockIdx.x;
  const long long p = tile / qtiles;
  const long long q = (tile - p * qtiles) * T + c;
  const bool valid = q < Q;
  const long long base = p * (long long)C::L * Q + q;
  const ColX<T> xc{sm3 + r * P * T, c};
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m)
    v[m] = valid ? in[base + (long long)(3 * (j + m * S) + r) * Q] : make_float2(0.f, 0.f);
  fft_line<P, G, SIGN>(v, j, xc, tw);
#pragma unroll
  for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
  __syncthreads();
  const ColX<T> x0{sm3, c}, x1{sm3 + P * T, c}, x2{sm3 + 2 * P * T, c};
  if (valid) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k1 = j + m * S;
      const float2 a = x0.ld(k1);
      const float2 b = cmul(x1.ld(k1), tw3<SIGN>(t3, k1));
      const float2 d = cmul(x2.ld(k1), tw3<SIGN>(t3, 2 * k1));
      out[base + (long long)(k1 + P * r) * Q] = cscale(radix3_out<SIGN>(a, b, d, r), scale);
    }
  }
}

// --------------------------------------------------------- z passes -----
template <int N>
struct Z3Cfg {
  static constexpr int H = N / 2;  // packed complex length, 3 P
  static constexpr int P = H / 3;
  static constexpr int G = elems_per_thread(P);
  static constexpr int S = P / G;
  static constexpr int LT = 3 * S;                                  // threads per line
  static constexpr int LPC = LT >= 192 ? 1 : (LT >= 96 ? 2 : (LT >= 48 ? 4 : 8));  // lines per CTA
  static constexpr int THREADS = LPC * LT;
};

// Real-to-complex along z for N = 6P: the N reals of a line packed as
// H = 3P complex values, the H-point transform by the radix-3 step, then the
// split X[k] = (Z[k] + conj Z[H-k])/2 + exp(-2 pi i k/N) (Z[k] - conj Z[H-k])/(2i).
// tw: size-P table; t3: size-N table (exp(-2 pi i m / N)), whose even
// entries are the size-H table.
template <int N>
__global__ void __launch_bounds__(Z3Cfg<N>::THREADS)
    k_z_r2c3(const float* __restrict__ in, float2* __restrict__ out, long long nlines,
             const float2* __restrict__ tw, const float2* __restrict__ t3, float scale) {
  using C = Z3Cfg<N>;
  constexpr int H = C::H, P = C::P, G = C::G, S = C::S;
  __shared__ float2 sm[C::LPC * H];
  const int li = threadIdx.x / C::LT, t = threadIdx.x % C::LT;
  const int r = t / S, j = t % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < nlines;
  float2* buf = sm + li * H;
  const LineX<false> xc{buf + r * P};
  const float2* src = reinterpret_cast<const float2*>(in + line * N);
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m) v[m] = valid ? src[3 * (j + m * S) + r] : make_float2(0.f, 0.f);
  fft_line<P, G, -1>(v, j, xc, tw);
#pragma unroll
  for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
  __syncthreads();
  const LineX<false> x0{buf}, x1{buf + P}, x2{buf + 2 * P};
  float2 z[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int k1 = j + m * S;
    const float2 b = cmul(x1.ld(k1), tw3<-1>(t3, 2 * k1));  // W_H^k1 = W_N^(2 k1)
    const float2 d = cmul(x2.ld(k1), tw3<-1>(t3, 4 * k1));
    z[m] = radix3_out<-1>(x0.ld(k1), b, d, r);
  }
  __syncthreads();
  // Z in natural order, plain indexing
#pragma unroll
  for (int m = 0; m < G; ++m) buf[j + m * S + P * r] = z[m];
  __syncthreads();
  if (valid) {
    float2* dst = out + line * (H + 1);
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S + P * r;
      const float2 A = z[m];
      const float2 Bc = cconj(buf[k == 0 ? 0 : H - k]);
      const float2 E = cscale(cadd(A, Bc), 0.5f);
      const float2 D = csub(A, Bc);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // D / (2i)
      dst[k] = cscale(cadd(E, cmul(__ldg(&t3[k]), O)), scale);
    }
    if (t == 0) dst[H] = make_float2((buf[0].x - buf[0].y) * scale, 0.f);
  }
}

// Complex-to-real along z for N = 6P: Z[k] = E + i O from X[k], X[H-k]
// (Im X[0], Im X[H] ignored), then the inverse H-point transform by the
// radix-3 step over the sub-sequences Z[3k' + r].
template <int N>
__global__ void __launch_bounds__(Z3Cfg<N>::THREADS)
    k_z_c2r3(const float2* __restrict__ in, float* __restrict__ out, long long nlines,
             const float2* __restrict__ tw, const float2* __restrict__ t3) {
  using C = Z3Cfg<N>;
  constexpr int H = C::H, P = C::P, G = C::G, S = C::S;
  __shared__ float2 sm[C::LPC * H];
  const int li = threadIdx.x / C::LT, t = threadIdx.x % C::LT;
  const int r = t / S, j = t % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < nlines;
  float2* buf = sm + li * H;
  const LineX<false> xc{buf + r * P};
  const float2* src = in + line * (H + 1);
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int k = 3 * (j + m * S) + r;
    float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
    if (valid) {
      A = src[k];
      B = src[H - k];
    }
    if (k == 0) {
      A.y = 0.f;
      B.y = 0.f;
    }
    const float2 Bc = cconj(B);
    const float2 E = cadd(A, Bc);
    const float2 O = cmulc(csub(A, Bc), __ldg(&t3[k]));  // (X[k] - conj X[H-k]) exp(+2 pi i k/N)
    v[m] = make_float2(E.x - O.y, E.y + O.x);
  }
  fft_line<P, G, +1>(v, j, xc, tw);
#pragma unroll
  for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
  __syncthreads();
  const LineX<false> x0{buf}, x1{buf + P}, x2{buf + 2 * P};
  if (valid) {
    float2* dst = reinterpret_cast<float2*>(out + line * N);
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k1 = j + m * S;
      const float2 b = cmul(x1.ld(k1), tw3<+1>(t3, 2 * k1));
      const float2 d = cmul(x2.ld(k1), tw3<+1>(t3, 4 * k1));
      dst[k1 + P * r] = radix3_out<+1>(x0.ld(k1), b, d, r);
    }
  }
}

// ------------------------------------------------------------ launchers --
template <int P, int SIGN>
static cudaError_t cpass3_p(fftk_plan p, const float2* in, float2* out, long long B, long long Q, float scale,
                            int kind, cudaStream_t st) {
  using C = C3Cfg<P>;
  static PerDevice once;
  const cudaError_t attr_err = once.run([](int) {
    return cudaFuncSetAttribute(k_cpass3<P, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const long long qtiles = (Q + C::T - 1) / C::T;
  LaunchScope ls(p, kind, st);
  k_cpass3<P, SIGN><<<(unsigned)(B * qtiles), C::THREADS, C::SMEM, st>>>(in, out, Q, qtiles, twiddles(p, P),
                                                                        twiddles3(p, 3 * P), scale);
  return cudaGetLastError();
}

template <int N>
static cudaError_t z3_n(fftk_plan p, bool fwd, const void* in, void* out, long long nl, float scale,
                        cudaStream_t st) {
  using C = Z3Cfg<N>;
  const unsigned blocks = (unsigned)((nl + C::LPC - 1) / C::LPC);
  if (fwd) {
    LaunchScope ls(p, KK_Z_R2C, st);
    k_z_r2c3<N><<<blocks, C::THREADS, 0, st>>>(static_cast<const float*>(in), static_cast<float2*>(out), nl,
                                              twiddles(p, C::P), twiddles3(p, N), scale);
  } else {
    LaunchScope ls(p, KK_Z_C2R, st);
    k_z_c2r3<N><<<blocks, C::THREADS, 0, st>>>(static_cast<const float2*>(in), static_cast<float*>(out), nl,
                                              twiddles(p, C::P), twiddles3(p, N));
  }
  return cudaGetLastError();
}

#define FFTK_SIZES3(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

cudaError_t launch_cpass3(fftk_plan p, int L, int sign, const float2* in, float2* out, long long B, long long Q,
                          float scale, int kind, cudaStream_t st) {
  if (B <= 0 || Q <= 0) return cudaSuccess;
#define CASE(n)                                                                                   \
  case 3 * n:                                                                                     \
    return sign < 0 ? cpass3_p<n, -1>(p, in, out, B, Q, scale, kind, st)                          \
                    : cpass3_p<n, +1>(p, in, out, B, Q, scale, kind, st);
  switch (L) { FFTK_SIZES3(CASE) }
#undef CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_z3(fftk_plan p, bool fwd, const void* in, void* out, long long nlines, float scale,
                      cudaStream_t st) {
  if (nlines <= 0) return cudaSuccess;
#define CASE(n) \
  case 6 * n:   \
    return z3_n<6 * n>(p, fwd, in, out, nlines, scale, st);
  switch (p->nz) { FFTK_SIZES3(CASE) }
#undef CASE
  return cudaErrorInvalidValue;
}

}  // namespace fftk
