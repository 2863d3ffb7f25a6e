// Device-side 1D FFT engine shared by every pass kernel.
//
// A line of length L (power of two) is held by S = L/G threads, G complex
// values per thread in the "natural" pattern v[m] = x[j + m*S] (j = thread
// index within the line).  The transform is a sequence of self-sorting
// (Stockham) radix-R stages, R = min(16, G, remaining length): every thread
// runs G/R radix-R butterflies in registers, and consecutive stages exchange
// data through a shared-memory buffer.  After the last stage the output is
// again in the natural pattern, so a pass can load and store global memory
// directly from registers with the same coalesced pattern.
//
// This replaces the FFTW 1D line transforms used by FFTK (paper Sec. 3);
// the radix-16/8/4/2 factorisation is fixed at compile time by Stage below.
//
// Sign convention: SIGN = -1 computes X[k] = sum_n x[n] exp(-2 pi i n k / L)
// (forward), SIGN = +1 the unnormalised inverse.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Complex sums and real scalings use the paired FP32 instructions of sm_100
// and later (two correctly rounded operations per instruction: the results
// are those of the scalar operations).  They cut the instruction count of
// the issue-bound kernels (the fused Navier-Stokes passes); a translation
// unit whose kernels are bound by their global accesses instead (the plain
// strided passes, measured slower with them) defines FFTK_PAIRED_FP32 as 0
// before including this header.  The engine lives in an inline namespace
// named after the choice, so the two forms never meet at link time.
#ifndef FFTK_PAIRED_FP32
#define FFTK_PAIRED_FP32 1
#endif

namespace fftk {
#if FFTK_PAIRED_FP32
inline namespace paired_fp32 {
#else
inline namespace scalar_fp32 {
#endif

// ---------------------------------------------------------------- complex --
#if FFTK_PAIRED_FP32
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
#if FFTK_PAIRED_FP32
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
#else
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
#endif
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * (SIGN * i)
template <int SIGN>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int N>
struct Log2 {
  static constexpr int value = 1 + Log2<N / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

// Mathematical constants of the 8- and 16-point DFTs.
#define FFTK_C8 0.70710678118654752440f   // cos(pi/4)
#define FFTK_C16 0.92387953251128675613f  // cos(pi/8)
#define FFTK_S16 0.38268343236508977173f  // sin(pi/8)

// a * exp(SIGN i theta) with (cos, sin) = (c, s)
template <int SIGN>
__device__ __forceinline__ float2 rot(float2 a, float c, float s) {
  return cmul(a, make_float2(c, SIGN * s));
}

// cos and sin of pi/16 and 3 pi/16
#define FFTK_C32A 0.98078528040323044913f
#define FFTK_S32A 0.19509032201612826785f
#define FFTK_C32B 0.83146961230254523708f
#define FFTK_S32B 0.55557023301960222474f

// a * exp(-2 pi i q / 32) for a q (0 <= q < 32) known at compile time after
// unrolling: the eighth-turn remainder by its (cos, sin) constants, then the
// quarter and half turns exactly.  The Hermitian-split factor exp(-2 pi i k / N)
// of a real line of N = 2 G S points at k = j + m S (G values per thread on S
// threads) is W_j mul_root32 by q = m 16 / G: one table load per thread.
__device__ __forceinline__ float2 mul_root32(float2 a, int q) {
  float2 r;
  switch (q & 7) {
    case 0: r = a; break;
    case 1: r = rot<-1>(a, FFTK_C32A, FFTK_S32A); break;
    case 2: r = rot<-1>(a, FFTK_C16, FFTK_S16); break;
    case 3: r = rot<-1>(a, FFTK_C32B, FFTK_S32B); break;
    case 4: r = rot<-1>(a, FFTK_C8, FFTK_C8); break;
    case 5: r = rot<-1>(a, FFTK_S32B, FFTK_C32B); break;
    case 6: r = rot<-1>(a, FFTK_S16, FFTK_C16); break;
    default: r = rot<-1>(a, FFTK_S32A, FFTK_C32A); break;
  }
  if (q & 8) r = mul_si<-1>(r);
  return (q & 16) ? make_float2(-r.x, -r.y) : r;
}

// --------------------------------------------------------------- codelets --
// In-place DFT of R values held in registers, natural order in and out.
template <int SIGN>
__device__ __forceinline__ void dft2(float2& x0, float2& x1) {
  float2 t = x0;
  x0 = cadd(t, x1);
  x1 = csub(t, x1);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a = cadd(x0, x2), b = csub(x0, x2);
  float2 c = cadd(x1, x3), d = mul_si<SIGN>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

template <int SIGN>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  dft4<SIGN>(x[0], x[2], x[4], x[6]);  // even samples: E0..E3 in x0,x2,x4,x6
  dft4<SIGN>(x[1], x[3], x[5], x[7]);  // odd samples:  O0..O3 in x1,x3,x5,x7
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  float2 o0 = x[1];
  float2 o1 = rot<SIGN>(x[3], FFTK_C8, FFTK_C8);   // W8^1
  float2 o2 = mul_si<SIGN>(x[5]);                  // W8^2
  float2 o3 = rot<SIGN>(x[7], -FFTK_C8, FFTK_C8);  // W8^3
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1);
  x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2);
  x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3);
  x[7] = csub(e3, o3);
}

// 16 = 4 x 4: X[k1 + 4 k2] = sum_{n2} W16^{n2 k1} W4^{n2 k2} sum_{n1} x[4 n1 + n2] W4^{n1 k1}
template <int SIGN>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<SIGN>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // y[n2][k1] now sits at x[n2 + 4 k1]; apply W16^{n2 k1}
  x[5] = rot<SIGN>(x[5], FFTK_C16, FFTK_S16);      // n2=1,k1=1: W^1
  x[9] = rot<SIGN>(x[9], FFTK_C8, FFTK_C8);        // n2=1,k1=2: W^2
  x[13] = rot<SIGN>(x[13], FFTK_S16, FFTK_C16);    // n2=1,k1=3: W^3
  x[6] = rot<SIGN>(x[6], FFTK_C8, FFTK_C8);        // n2=2,k1=1: W^2
  x[10] = mul_si<SIGN>(x[10]);                     // n2=2,k1=2: W^4
  x[14] = rot<SIGN>(x[14], -FFTK_C8, FFTK_C8);     // n2=2,k1=3: W^6
  x[7] = rot<SIGN>(x[7], FFTK_S16, FFTK_C16);      // n2=3,k1=1: W^3
  x[11] = rot<SIGN>(x[11], -FFTK_C8, FFTK_C8);     // n2=3,k1=2: W^6
  x[15] = rot<SIGN>(x[15], -FFTK_C16, -FFTK_S16);  // n2=3,k1=3: W^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  // X[k1 + 4 k2] sits at x[4 k1 + k2]: transpose the 4x4 index grid
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = x[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int R, int SIGN>
__device__ __forceinline__ void dftR(float2 (&a)[R]) {
  if constexpr (R == 2) {
    dft2<SIGN>(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4<SIGN>(a[0], a[1], a[2], a[3]);
  } else if constexpr (R == 8) {
    dft8<SIGN>(a);
  } else if constexpr (R == 16) {
    dft16<SIGN>(a);
  }
}

// --------------------------------------------------------- smem swizzle ----
// Position `pos` of a tile with T columns (T a power of two; column c added by
// the caller).  For T < 16 the 16/T rows that share a 16-element block are
// placed by an XOR fold of pos's digits, so every access pattern of the engine
// (unit-stride rows, and radix-R strided rows) is bank-conflict free for
// 64-bit accesses (a half warp covers all 32 banks once).
template <int T>
__device__ __forceinline__ int swz(int pos) {
  if constexpr (T >= 16) {
    return pos * T;
  } else {
    constexpr int t = Log2<T>::value;
    constexpr int s = 4 - t;
    int f = pos;
#pragma unroll
    for (int sh = s; sh < 16; sh += s) f ^= pos >> sh;
    f &= (1 << s) - 1;
    return ((pos >> s) << 4) + (f << t);
  }
}

// Exchange buffer for a column tile: element (pos, c) of a [L][T] tile.
template <int T>
struct ColX {
  static constexpr bool kStageTables = false;  // a warp spans 32/T butterflies: gathers are near-broadcasts
  float2* s;
  int c;
  __device__ __forceinline__ void st(int pos, float2 v) const { s[swz<T>(pos) + c] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return s[swz<T>(pos) + c]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Position of element `pos` of one contiguous line: an XOR permutation within
// each 16-element block, keyed by the block index B = pos >> 4 through the
// map bits(B) -> {1, 2, 12, 8, then 1, 2, 4, 8, ...}.  Block bit 2 flips slot
// bits 2 and 3, which makes the radix-8 exchanges (8 values per thread) as
// well as the radix-16 ones conflict free for 64-bit accesses.
__device__ __forceinline__ int swz_line(int pos) {
  const int b = pos >> 4;
  const int lo = b & 15;
  const int h = lo ^ ((lo & 4) << 1) ^ (b >> 4) ^ (b >> 8);
  return (pos & ~15) | ((pos ^ h) & 15);
}

// Exchange buffer for one contiguous line; WARP_SYNC when a line's threads
// live in one warp.
template <bool WARP_SYNC>
struct LineX {
  static constexpr bool kStageTables = true;  // a warp spans 32 consecutive butterflies
  float2* s;
  __device__ __forceinline__ void st(int pos, float2 v) const { s[swz_line(pos)] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return s[swz_line(pos)]; }
  __device__ __forceinline__ void sync() const {
    if constexpr (WARP_SYNC)
      __syncwarp();
    else
      __syncthreads();
  }
};

// ---------------------------------------------------------------- engine ---
// Twiddle tables: the plan holds, for every power of two L' <= 4 LT, the
// table exp(-2 pi i m / L'), m < L', at offset L' of one array (entries
// computed in FP64 on the host and rounded once to FP32).  A kernel gets the
// table of size 2^TL >= L, which locates the array's base at compile time.
//
// A stage of span M = NS R (radix R after NS points) multiplies input r of
// butterfly k by exp(-2 pi i r k / M).  In a contiguous line (LineX) one warp
// holds 32 consecutive butterflies, and a gather from the size-L table at
// index r k L / M spreads each load over up to 32 scattered entries; so the
// plan also stores, for every M <= 4096 and R in {2, 4, 8, 16}, the table
// exp(-2 pi i r k / M) r-major (entry r NS + k), which those stages read.
// These tables lie kStageTwiddles entries below the base of the pyramid (the
// same FP64-built values, rounded the same way).  Column tiles (ColX) keep the
// pyramid: their warps span 32/T butterflies, so the gathers are already
// near-broadcasts.
constexpr int kStageTwiddles = 32768;
__host__ __device__ constexpr int stage_tw_offset(int M, int R) {
  return 4 * M + (R == 2 ? 0 : (R == 4 ? 1 : (R == 8 ? 2 : 3))) * M;
}

template <int L, int G>
struct Shape {
  static_assert(L >= 1 && (L & (L - 1)) == 0, "L must be a power of two");
  static constexpr int g = G;
  static constexpr int S = L / G;  // threads per line
};

__host__ __device__ constexpr int fftk_min3(int a, int b, int c) {
  return a < b ? (a < c ? a : c) : (b < c ? b : c);
}

template <int L, int G, int SIGN, int NS, int TL>
struct Stage {
  template <class X>
  __device__ __forceinline__ static void run(float2 (&v)[G], int j, const X& xc,
                                             const float2* __restrict__ tw) {
    if constexpr (NS < L) {
      constexpr int REM = L / NS;
      constexpr int R = fftk_min3(16, G, REM);
      constexpr int B = G / R;   // butterflies per thread
      constexpr int S = L / G;   // threads per line
      constexpr bool LAST = (NS * R == L);
      constexpr int LOG_NSR = Log2<NS * R>::value;
#pragma unroll
      for (int t = 0; t < B; ++t) {
        const int b = j + t * S;   // butterfly index in [0, L/R)
        const int k = b & (NS - 1);
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[t + r * B];
        if constexpr (NS > 1) {
          // exp(SIGN 2 pi i r k / (NS R)): from this stage's r-major table for
          // contiguous lines, else from the size-2^TL table (tw, at offset 2^TL
          // of the pyramid) at index r k 2^TL / (NS R)
          const float2* ts = tw - (1 << TL) - kStageTwiddles + stage_tw_offset(NS * R, R);
#pragma unroll
          for (int r = 1; r < R; ++r) {
            const float2 w = X::kStageTables ? __ldg(&ts[r * NS + k]) : __ldg(&tw[(r * k) << (TL - LOG_NSR)]);
            a[r] = SIGN < 0 ? cmul(a[r], w) : cmulc(a[r], w);
          }
        }
        dftR<R, SIGN>(a);
        if constexpr (LAST) {
#pragma unroll
          for (int r = 0; r < R; ++r) v[t + r * B] = a[r];
        } else {
          const int base = (b - k) * R + k;  // (b / NS) * NS * R + k
#pragma unroll
          for (int r = 0; r < R; ++r) xc.st(base + r * NS, a[r]);
        }
      }
      if constexpr (!LAST) {
        xc.sync();
#pragma unroll
        for (int m = 0; m < G; ++m) v[m] = xc.ld(j + m * S);
        xc.sync();
        Stage<L, G, SIGN, NS * R, TL>::run(v, j, xc, tw);
      }
    }
  }
};

// Full L-point transform of the line held in v (natural pattern in and out).
// The exchange buffer must be free on entry; it is free again on exit.
// tw: the twiddle table of size 2^TL (TL >= log2 L; by default the size-L one).
template <int L, int G, int SIGN, int TL = Log2<L>::value, class X>
__device__ __forceinline__ void fft_line(float2 (&v)[G], int j, const X& xc, const float2* __restrict__ tw) {
  static_assert((1 << TL) >= L, "twiddle table too short");
  Stage<L, G, SIGN, 1, TL>::run(v, j, xc, tw);
}

// Elements per thread used by the passes for a line of length L.
__host__ __device__ constexpr int elems_per_thread(int L) { return L < 16 ? L : 16; }

}  // inline namespace
}  // namespace fftk
