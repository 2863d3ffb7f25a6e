// Sine and cosine transforms along one axis (the free-slip bases of paper
// Sec. 2.1, Eq. (2b, 2c)), on the same line engine as the Fourier passes.
//
// A line of L points s_j = (j + 1/2) pi / L of [0, pi]; the inverse is
//   f_j = sum_k fhat_k 2 cos(k s_j), k = 0..L-1   (cosine, fhat_k at k), or
//   f_j = sum_k fhat_k 2 sin(k s_j), k = 1..L     (sine, fhat_k at k - 1),
// the forward its inverse (fhat_k = C_k / L, halved for the cosine k = 0 and
// the sine k = L).  Both reduce to one complex FFT of length L (Makhoul, "A
// fast cosine transform in one and two dimensions", IEEE Trans. ASSP 28,
// 1980):
//   C_k = sum_j x_j cos(k s_j):  v_r = x_{2r}, v_{L-1-r} = x_{2r+1} (r < L/2),
//   V = DFT(v),  C_k = (W_k V_k + conj(W_k) V_{L-k}) / 2,  W_k = exp(-i pi k / 2L),
// which holds for complex x (complex-linear; for real x it is Re(W_k V_k)).
// Inverse: V_k = conj(W_k) (C_k - i C_{L-k}) with C_L = 0, v = IDFT(V).
// The sine transform is the cosine transform of (-1)^j x_j read backwards:
// sin((L - k) s_j) = (-1)^j cos(k s_j).
//
// Kernels: a strided pass over float2 columns (x or y lines of a spectrum, or
// of a real field read as pairs of adjacent z values) and a contiguous pass
// over real z lines that transforms two lines at once as re + i im.
#include <mutex>

#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {

__device__ __forceinline__ int mk_perm(int r, int L) { return r < L / 2 ? 2 * r : 2 * (L - 1 - r) + 1; }
// position r of element i in the permuted line
__device__ __forceinline__ int mk_unperm(int i, int L) { return (i & 1) ? L - 1 - (i >> 1) : (i >> 1); }

// C_k from V_k, V_{L-k} and W_k
__device__ __forceinline__ float2 mk_post(float2 vk, float2 vn, float2 w) {
  const float2 a = cmul(w, vk), b = cmulc(vn, w);  // W V_k, conj(W) V_{L-k}
  return make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
}

// V_k = conj(W_k) (C_k - i C_{L-k})
__device__ __forceinline__ float2 mk_pre(float2 ck, float2 cn, float2 w) {
  const float2 d = make_float2(ck.x + cn.y, ck.y - cn.x);  // C_k - i C_{L-k}
  return cmulc(d, w);
}

// --------------------------------------------------------- strided pass --
template <int L>
struct SCfg {
  static constexpr int G = elems_per_thread(L);
  static constexpr int S = L / G;
  static constexpr int T = S <= 16 ? 256 / S : (S <= 64 ? 16 : 1024 / S);
  static constexpr int THREADS = T * S;
  static constexpr int MINB = THREADS <= 512 ? 2 : 1;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)L * T;
};

// One tile = T adjacent columns x the whole line (rows of stride Q), as the
// Fourier strided pass.  SINE selects the basis, DIR -1 forward, +1 inverse.
// tw: the size-L table, tq: the size-4L table (W_k = tq[k]).
template <int L, bool SINE, int DIR>
__global__ void __launch_bounds__(SCfg<L>::THREADS, SCfg<L>::MINB)
    k_scpass(const float2* in, float2* out, long long Q, long long qtiles, const float2* __restrict__ tw,
             const float2* __restrict__ tq, float scale) {
  using C = SCfg<L>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smc[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const long long tile = blockIdx.x;
  const long long p = tile / qtiles;
  const long long q = (tile - p * qtiles) * T + c;
  const bool valid = q < Q;
  const long long base = p * (long long)L * Q + q;
  const ColX<T> xc{smc, c};
  float2 v[G];
  if (DIR < 0) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int r = j + m * S;
      float2 x = valid ? in[base + (long long)mk_perm(r, L) * Q] : make_float2(0.f, 0.f);
      if (SINE && r >= L / 2) x = make_float2(-x.x, -x.y);  // (-1)^j at odd j
      v[m] = x;
    }
    fft_line<L, G, -1>(v, j, xc, tw);
#pragma unroll
    for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
    xc.sync();
    if (valid) {
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const int k = j + m * S;
        const float2 ck = mk_post(v[m], xc.ld((L - k) & (L - 1)), __ldg(&tq[k]));
        const float f = (k == 0 ? 0.5f : 1.f) * scale;
        const int row = SINE ? L - 1 - k : k;
        out[base + (long long)row * Q] = cscale(ck, f);
      }
    }
  } else {
    // coefficient rows in natural order, doubled at k = 0, through shared memory
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const int row = SINE ? L - 1 - k : k;
      float2 x = valid ? in[base + (long long)row * Q] : make_float2(0.f, 0.f);
      if (k == 0) x = cscale(x, 2.f);
      v[m] = x;
      xc.st(k, x);
    }
    xc.sync();
    float2 w[G];
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 cn = k == 0 ? make_float2(0.f, 0.f) : xc.ld(L - k);
      w[m] = mk_pre(v[m], cn, __ldg(&tq[k]));
    }
    xc.sync();
    fft_line<L, G, +1>(w, j, xc, tw);
    if (valid) {
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const int r = j + m * S;
        float2 x = w[m];
        if (SINE && r >= L / 2) x = make_float2(-x.x, -x.y);
        out[base + (long long)mk_perm(r, L) * Q] = cscale(x, scale);
      }
    }
  }
}

// The strided pass restricted to the 2/3-rule set of an n^3 spectrum
// (L = n along x): columns are the kept (k_y, k_z) only (k_y rows 0..kd and
// n-kd..n-1, k_z < kd + 1), the inverse reads only coefficient rows with
// 3 k_x < 2n (sine row s is k_x = s + 1, cosine row s is k_x = s) and the
// forward writes only those; B batch elements of [n][n][n/2+1].
template <int L, bool SINE, int DIR>
__global__ void __launch_bounds__(SCfg<L>::THREADS, SCfg<L>::MINB)
    k_scpass_pr(const float2* in, float2* out, int ktiles, const float2* __restrict__ tw,
                const float2* __restrict__ tq, float scale) {
  using C = SCfg<L>;
  constexpr int G = C::G, S = C::S, T = C::T;
  constexpr long long H1 = L / 2 + 1, M = (long long)L * L * H1, Q = (long long)L * H1;
  constexpr int KD = (L - 1) / 3, KC = KD + 1, NK = 2 * KD + 1;
  extern __shared__ float2 smc[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const long long blk = blockIdx.x;
  const long long bo = blk / ktiles;
  const int kt = (int)(blk - bo * ktiles);
  const long long b = bo / NK;
  const int o = (int)(bo - b * NK);
  const int ay = o <= KD ? o : L - (NK - o);
  const int kz = kt * T + c;
  const bool valid = kz < KC;
  const long long base = b * M + (long long)ay * H1 + kz;
  const ColX<T> xc{smc, c};
  auto kept_row = [](int row) { return 3 * (SINE ? row + 1 : row) < 2 * L; };
  float2 v[G];
  if (DIR < 0) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int r = j + m * S;
      float2 x = valid ? in[base + (long long)mk_perm(r, L) * Q] : make_float2(0.f, 0.f);
      if (SINE && r >= L / 2) x = make_float2(-x.x, -x.y);
      v[m] = x;
    }
    fft_line<L, G, -1>(v, j, xc, tw);
#pragma unroll
    for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
    xc.sync();
    if (valid) {
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const int k = j + m * S;
        const int row = SINE ? L - 1 - k : k;
        if (!kept_row(row)) continue;
        const float2 ck = mk_post(v[m], xc.ld((L - k) & (L - 1)), __ldg(&tq[k]));
        out[base + (long long)row * Q] = cscale(ck, (k == 0 ? 0.5f : 1.f) * scale);
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const int row = SINE ? L - 1 - k : k;
      float2 x = (valid && kept_row(row)) ? in[base + (long long)row * Q] : make_float2(0.f, 0.f);
      if (k == 0) x = cscale(x, 2.f);
      v[m] = x;
      xc.st(k, x);
    }
    xc.sync();
    float2 w[G];
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 cn = k == 0 ? make_float2(0.f, 0.f) : xc.ld(L - k);
      w[m] = mk_pre(v[m], cn, __ldg(&tq[k]));
    }
    xc.sync();
    fft_line<L, G, +1>(w, j, xc, tw);
    if (valid) {
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const int r = j + m * S;
        float2 x = w[m];
        if (SINE && r >= L / 2) x = make_float2(-x.x, -x.y);
        out[base + (long long)mk_perm(r, L) * Q] = cscale(x, scale);
      }
    }
  }
}

// ------------------------------------------------- contiguous real pass --
template <int N>
struct SZCfg {
  static constexpr int G = elems_per_thread(N);
  static constexpr int S = N / G;                    // threads per line pair
  static constexpr int LPC = S >= 256 ? 1 : 256 / S;  // line pairs per CTA
  static constexpr int THREADS = LPC * S;
  static constexpr bool WARP = S <= 32;
};

// Two real lines a, b of length N (z fastest) as one complex line a + i b.
// Pair `pr` holds lines 2 pr and 2 pr + 1; an odd last line pairs with zeros.
template <int N, bool SINE, int DIR>
__global__ void __launch_bounds__(SZCfg<N>::THREADS)
    k_scz(const float* in, float* out, long long nlines, const float2* __restrict__ tw,
          const float2* __restrict__ tq, float scale) {
  using C = SZCfg<N>;
  constexpr int G = C::G, S = C::S;
  constexpr int LOGN = Log2<N>::value;
  __shared__ float2 sm[C::LPC * N];
  const int li = threadIdx.x / S, j = threadIdx.x % S;
  const long long la = 2 * ((long long)blockIdx.x * C::LPC + li);
  const bool va = la < nlines, vb = la + 1 < nlines;
  const LineX<C::WARP> xc{sm + li * N};
  const float* ia = in + la * N;
  const float* ib = ia + N;
  float* oa = out + la * N;
  float* ob = oa + N;
  float2 v[G];
  if (DIR < 0) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int i = j + m * S;
      float2 x = make_float2(va ? ia[i] : 0.f, vb ? ib[i] : 0.f);
      if (SINE && (i & 1)) x = make_float2(-x.x, -x.y);
      xc.st(mk_unperm(i, N), x);
    }
    xc.sync();
#pragma unroll
    for (int m = 0; m < G; ++m) v[m] = xc.ld(j + m * S);
    xc.sync();
    fft_line<N, G, -1, LOGN>(v, j, xc, tw);
#pragma unroll
    for (int m = 0; m < G; ++m) xc.st(j + m * S, v[m]);
    xc.sync();
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 ck = mk_post(v[m], xc.ld((N - k) & (N - 1)), __ldg(&tq[k]));
      const float f = (k == 0 ? 0.5f : 1.f) * scale;
      const int row = SINE ? N - 1 - k : k;
      if (va) oa[row] = ck.x * f;
      if (vb) ob[row] = ck.y * f;
    }
  } else {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const int row = SINE ? N - 1 - k : k;
      float2 x = make_float2(va ? ia[row] : 0.f, vb ? ib[row] : 0.f);
      if (k == 0) x = cscale(x, 2.f);
      v[m] = x;
      xc.st(k, x);
    }
    xc.sync();
    float2 w[G];
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 cn = k == 0 ? make_float2(0.f, 0.f) : xc.ld(N - k);
      w[m] = mk_pre(v[m], cn, __ldg(&tq[k]));
    }
    xc.sync();
    fft_line<N, G, +1, LOGN>(w, j, xc, tw);
#pragma unroll
    for (int m = 0; m < G; ++m) xc.st(j + m * S, w[m]);
    xc.sync();
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int i = j + m * S;
      float2 x = xc.ld(mk_unperm(i, N));
      if (SINE && (i & 1)) x = make_float2(-x.x, -x.y);
      if (va) oa[i] = x.x * scale;
      if (vb) ob[i] = x.y * scale;
    }
  }
}

// ------------------------------------------------------------ launchers --
template <int L, bool SINE, int DIR>
static cudaError_t scpass_l(fftk_plan p, const float2* in, float2* out, long long P, long long Q, float scale,
                            int kind, cudaStream_t st) {
  using C = SCfg<L>;
  static PerDevice once;
  const cudaError_t attr_err = once.run([](int) {
    return cudaFuncSetAttribute(k_scpass<L, SINE, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const long long qtiles = (Q + C::T - 1) / C::T;
  LaunchScope ls(p, kind, st);
  k_scpass<L, SINE, DIR><<<(unsigned)(P * qtiles), C::THREADS, C::SMEM, st>>>(in, out, Q, qtiles, twiddles(p, L),
                                                                              twiddles(p, 4 * L), scale);
  return cudaGetLastError();
}

template <int N, bool SINE, int DIR>
static cudaError_t scz_n(fftk_plan p, const float* in, float* out, long long nlines, float scale, int kind,
                         cudaStream_t st) {
  using C = SZCfg<N>;
  const long long pairs = (nlines + 1) / 2;
  LaunchScope ls(p, kind, st);
  k_scz<N, SINE, DIR><<<(unsigned)((pairs + C::LPC - 1) / C::LPC), C::THREADS, 0, st>>>(
      in, out, nlines, twiddles(p, N), twiddles(p, 4 * N), scale);
  return cudaGetLastError();
}

template <int L, bool SINE, int DIR>
static cudaError_t scpass_pr_l(fftk_plan p, const float2* in, float2* out, long long B, float scale,
                               cudaStream_t st) {
  using C = SCfg<L>;
  static PerDevice once;
  const cudaError_t attr_err = once.run([](int) {
    return cudaFuncSetAttribute(k_scpass_pr<L, SINE, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  constexpr int KD = (L - 1) / 3, KC = KD + 1;
  const int ktiles = (KC + C::T - 1) / C::T;
  LaunchScope ls(p, DIR < 0 ? KK_SC_FWD : KK_SC_INV, st);
  k_scpass_pr<L, SINE, DIR><<<(unsigned)(B * (2 * KD + 1) * ktiles), C::THREADS, C::SMEM, st>>>(
      in, out, ktiles, twiddles(p, L), twiddles(p, 4 * L), scale);
  return cudaGetLastError();
}

#define FFTK_SC_SIZES(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t launch_scpass(fftk_plan p, int L, bool sine, int dir, const float2* in, float2* out, long long P,
                          long long Q, float scale, int kind, cudaStream_t st) {
  if (P <= 0 || Q <= 0) return cudaSuccess;
#define CASE(n)                                                                                   \
  case n:                                                                                         \
    if (sine)                                                                                     \
      return dir < 0 ? scpass_l<n, true, -1>(p, in, out, P, Q, scale, kind, st)                   \
                     : scpass_l<n, true, +1>(p, in, out, P, Q, scale, kind, st);                  \
    return dir < 0 ? scpass_l<n, false, -1>(p, in, out, P, Q, scale, kind, st)                    \
                   : scpass_l<n, false, +1>(p, in, out, P, Q, scale, kind, st);
  switch (L) { FFTK_SC_SIZES(CASE) }
#undef CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_scz(fftk_plan p, bool sine, int dir, const float* in, float* out, long long nlines,
                       float scale, int kind, cudaStream_t st) {
  if (nlines <= 0) return cudaSuccess;
#define CASE(n)                                                                                   \
  case n:                                                                                         \
    if (sine)                                                                                     \
      return dir < 0 ? scz_n<n, true, -1>(p, in, out, nlines, scale, kind, st)                    \
                     : scz_n<n, true, +1>(p, in, out, nlines, scale, kind, st);                   \
    return dir < 0 ? scz_n<n, false, -1>(p, in, out, nlines, scale, kind, st)                     \
                   : scz_n<n, false, +1>(p, in, out, nlines, scale, kind, st);
  switch (p->nz) { FFTK_SC_SIZES(CASE) }
#undef CASE
  return cudaErrorInvalidValue;
}

}  // namespace fftk

namespace fftk {

cudaError_t launch_scpass_pruned(fftk_plan p, bool sine, int dir, const float2* in, float2* out, long long B,
                                 float scale, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
#define CASE(n)                                                                                   \
  case n:                                                                                         \
    if (sine)                                                                                     \
      return dir < 0 ? scpass_pr_l<n, true, -1>(p, in, out, B, scale, st)                         \
                     : scpass_pr_l<n, true, +1>(p, in, out, B, scale, st);                        \
    return dir < 0 ? scpass_pr_l<n, false, -1>(p, in, out, B, scale, st)                          \
                   : scpass_pr_l<n, false, +1>(p, in, out, B, scale, st);
  switch (p->nx) { CASE(8) CASE(16) CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) }
#undef CASE
  return cudaErrorInvalidValue;
}

}  // namespace fftk
