// Pseudo-spectral incompressible Navier-Stokes (paper Sec. 2.2, Eqs. (7)-(8))
// in rotational form, fused into the FFT passes of Sec. 3.
//
// One evaluation of the nonlinear term is five kernels:
//   1. ns_invx_curl : uhat (3) -> inverse x pass of u and omega = i k x u (6)
//   2. ns_invy      : inverse y pass of the 6 fields
//   3. ns_z_product : per z line: c2r of the 6 fields, n = u x omega in
//                     registers, r2c of the 3 products (real fields never
//                     touch global memory)
//   4. ns_fwdy      : forward y pass of the 3 fields
//   5. ns_fwdx      : forward x pass + 1/N^3 + 2/3 dealias + projection
//                     + forcing + the RK2 integrating-factor update
//
// Dealiasing (2/3 rule, "filling up only 2/3 of the array in each direction")
// is exploited throughout: modes with 3|k| >= n on any axis are zero in the
// state, so every pass reads only the rows and columns that can be nonzero
// and writes only those a later pass reads.  The arrays keep the full
// [n][n][n/2+1] layout; the untouched parts are never read.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {

fftk_status from_cuda(cudaError_t e);

struct NSGeom {
  int n;         // grid size
  int h1;        // n/2 + 1
  int kd;        // largest kept |k| = (n-1)/3
  int kc;        // kept k_z count = kd + 1
  int nk;        // kept count on x and y = 2 kd + 1
  long long M;   // n * n * h1 (complex elements per field)
};

__device__ __forceinline__ bool kept_xy(int a, int n, int kd) { return a <= kd || a >= n - kd; }
// wavenumber of index a on the x or y axis
__device__ __forceinline__ int kwav(int a, int n) { return 2 * a < n ? a : a - n; }
// index of the d-th kept x/y mode (d in [0, 2kd]): 0..kd, then n-kd..n-1
__device__ __forceinline__ int dense_to_a(int d, int n, int kd) {
  return d <= kd ? d : n - (2 * kd + 1 - d);
}
__device__ __forceinline__ float2 mul_i(float2 a, float k) {  // a * (i k)
  return make_float2(-k * a.y, k * a.x);
}

// ------------------------------------------------------------ x/y config ---
// Single-field passes (inverse x with the curl, both y passes): the strided
// FFT pass configuration, 16 values per thread, 16 k_z columns per tile
// (128-byte row segments), 32 warps per SM at <= 64 registers.
template <int N>
struct NXCfg {
  static constexpr int G = N < 16 ? N : 16;
  static constexpr int S = N / G;
  static constexpr int T = S <= 16 ? 16 : (S <= 64 ? 16 : 1024 / S);
  static constexpr int THREADS = T * S;
  static constexpr int MINB = THREADS <= 512 ? (THREADS <= 256 ? 4 : 2) : 1;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)N * T;
};

// 2./4. y pass, columns (x, k_z < kc), blockIdx -> (field, x, k_z tile).
//    SIGN=+1: only kept k_y rows are read, every y row is written;
//    SIGN=-1: every y row is read, only kept k_y rows are written.
template <int N, int SIGN>
__global__ void __launch_bounds__(NXCfg<N>::THREADS, NXCfg<N>::MINB)
    k_ns_ypass(float2* w, NSGeom g, int ktiles, const float2* __restrict__ tw) {
  constexpr long long H1 = N / 2 + 1, MM = (long long)N * N * H1;  // geometry of the n^3 grid
  constexpr int KD = (N - 1) / 3;                                  // largest kept |k| (2/3 rule)
  using C = NXCfg<N>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smn[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int kt = blockIdx.x % ktiles;
  const int rest = blockIdx.x / ktiles;
  const int x = rest % N;
  const int f = rest / N;
  const int kz = kt * T + c;
  const bool valid = kz < (KD + 1);
  float2* base = w + f * MM + (long long)x * N * H1 + kz;
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int pos = j + m * S;
    const bool rd = valid && (SIGN < 0 || kept_xy(pos, N, KD));
    v[m] = rd ? base[(long long)pos * H1] : make_float2(0.f, 0.f);
  }
  fft_line<N, G, SIGN>(v, j, ColX<T>{smn, c}, tw);
  if (valid) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int pos = j + m * S;
      if (SIGN > 0 || kept_xy(pos, N, KD)) base[(long long)pos * H1] = v[m];
    }
  }
}

// Forward x pass (three fields held at once): 8 values per thread.
template <int N>
struct NFCfg {
  static constexpr int G = N < 8 ? N : 8;
  static constexpr int S = N / G;
  static constexpr int T = S >= 32 ? (S == 32 ? 16 : (S == 64 ? 8 : 4)) : 16;
  static constexpr int THREADS = T * S;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)N * T;
};

// Inverse x pass (two fields held at once): 16 values per thread for
// n >= 512, 16 columns per tile (128-byte row segments) at n = 512 and 8 at
// n = 1024; smaller grids as NFCfg.
template <int N>
struct NICfg {
  static constexpr int G = N >= 512 ? 16 : NFCfg<N>::G;
  static constexpr int S = N / G;
  static constexpr int T = N == 512 ? 16 : (N == 1024 ? 8 : NFCfg<N>::T);
  static constexpr int THREADS = T * S;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)N * T;
};

// Forward x pass (one field in registers, two parked): 1024 threads, 8 values
// per thread, 16 columns per tile at n = 512 and 8 at n = 1024.
template <int N>
struct NUCfg {
  static constexpr int G = NFCfg<N>::G;
  static constexpr int S = N / G;
  static constexpr int T = N == 512 ? 16 : (N == 1024 ? 8 : NFCfg<N>::T);
  static constexpr int THREADS = T * S;
  static constexpr size_t SMEM = sizeof(float2) * ((size_t)N * T + 2 * G * THREADS);
  static constexpr int MINB = 1024 / THREADS < 16 ? 1024 / THREADS : 16;  // 64 registers
};

// 1. inverse x pass with the curl.  Columns: kept (k_y, k_z); rows: k_x.
//    U_c = F^-1_x(u_c), D_c = F^-1_x(i k_x u_c), then
//    omega_x = i (k_y U_z - k_z U_y), omega_y = i k_z U_x - D_z,
//    omega_z = D_y - i k_y U_x   (five transforms instead of six).
//    Output field order: u_x, u_y, u_z, omega_x, omega_y, omega_z.
template <int N>
__global__ void __launch_bounds__(NICfg<N>::THREADS)
    k_ns_invx(const float2* __restrict__ u, float2* __restrict__ w, NSGeom g, int ktiles,
              const float2* __restrict__ tw) {
  constexpr long long H1 = N / 2 + 1, MM = (long long)N * N * H1;  // geometry of the n^3 grid
  constexpr int KD = (N - 1) / 3;                                  // largest kept |k| (2/3 rule)
  using C = NICfg<N>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smn[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int dky = blockIdx.x / ktiles;
  const int kz = (blockIdx.x - dky * ktiles) * T + c;
  const bool valid = kz < (KD + 1);
  const int ay = dense_to_a(dky, N, KD);
  const long long q = (long long)ay * H1 + kz;
  const long long rs = (long long)N * H1;
  const float ky = (float)kwav(ay, N), kzf = (float)kz;
  const ColX<T> xc{smn, c};
  auto load = [&](int f, float2(&v)[G], bool ikx) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int pos = j + m * S;
      float2 a = make_float2(0.f, 0.f);
      if (valid && kept_xy(pos, N, KD)) a = u[f * MM + pos * rs + q];
      v[m] = ikx ? mul_i(a, (float)kwav(pos, N)) : a;
    }
  };
  auto store = [&](int f, const float2(&v)[G]) {
    if (valid) {
#pragma unroll
      for (int m = 0; m < G; ++m) w[f * MM + (j + m * S) * rs + q] = v[m];
    }
  };
  float2 a[G], b[G];
  load(1, a, true);
  fft_line<N, G, +1>(a, j, xc, tw);  // D_y
  load(0, b, false);
  fft_line<N, G, +1>(b, j, xc, tw);  // U_x
  store(0, b);
#pragma unroll
  for (int m = 0; m < G; ++m) a[m] = csub(a[m], mul_i(b[m], ky));  // omega_z
  store(5, a);
  load(2, a, true);
  fft_line<N, G, +1>(a, j, xc, tw);  // D_z
#pragma unroll
  for (int m = 0; m < G; ++m) a[m] = csub(mul_i(b[m], kzf), a[m]);  // omega_y
  store(4, a);
  load(1, a, false);
  fft_line<N, G, +1>(a, j, xc, tw);  // U_y
  store(1, a);
  load(2, b, false);
  fft_line<N, G, +1>(b, j, xc, tw);  // U_z
  store(2, b);
#pragma unroll
  for (int m = 0; m < G; ++m)
    b[m] = make_float2(-(ky * b[m].y - kzf * a[m].y), ky * b[m].x - kzf * a[m].x);  // omega_x
  store(3, b);
}

// ------------------------------------------------------------- z product ---
template <int N>
struct NZCfg {
  static constexpr int H = N / 2;
  static constexpr int G = H < 8 ? H : 8;
  static constexpr int S = H / G;
  static constexpr int LPC = S >= 128 ? 1 : 128 / S;
  static constexpr int THREADS = LPC * S;
  static constexpr bool WARP = S <= 32;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)LPC * H * 4;  // exchange + 3 parked fields
};

// 3. per (x, y) line: the six c2r transforms, the product n = u x omega and
//    the three r2c transforms.  Reads k_z < kc of fields 0..5, writes k_z < kc
//    of fields 0..2 (in place: a line is fully read before it is written).
//    The three velocity components are parked in real space in shared memory;
//    each vorticity component is then transformed and folded into the
//    accumulators of n, so at most 3 fields are held in registers.
template <int N>
__global__ void __launch_bounds__(NZCfg<N>::THREADS, 3)
    k_ns_z(float2* w, NSGeom g, const float2* __restrict__ tw) {
  constexpr long long H1 = N / 2 + 1, MM = (long long)N * N * H1;  // geometry of the n^3 grid
  constexpr int KD = (N - 1) / 3;                                  // largest kept |k| (2/3 rule)
  using C = NZCfg<N>;
  constexpr int H = C::H, G = C::G, S = C::S;
  constexpr int LOGN = Log2<N>::value;
  constexpr int KC = KD + 1;  // kept k_z count
  extern __shared__ float2 smz[];
  const int li = threadIdx.x / S, j = threadIdx.x % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < (long long)N * N;
  const LineX<C::WARP> xc{smz + li * H};
  float2* park = smz + C::LPC * H + li * 3 * H + j;  // [3][G][S] per line, this thread's column

  // inverse z transform of field f (half-complex -> N real points, two per slot)
  auto c2r = [&](int f, float2 (&U)[G]) {
    const float2* src = w + f * MM + line * H1;
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
      if (valid && k < KC) A = src[k];
      if (valid && H - k < KC) B = src[H - k];
      if (k == 0) {
        A.y = 0.f;
        B.y = 0.f;
      }
      const float2 Bc = cconj(B);
      const float2 E = cadd(A, Bc);
      const float2 W = __ldg(&tw[k]);
      const float2 O = cmulc(csub(A, Bc), W);
      U[m] = make_float2(E.x - O.y, E.y + O.x);
    }
    fft_line<H, G, +1, LOGN>(U, j, xc, tw);
  };

  {
    float2 U[G];
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
      c2r(f, U);
#pragma unroll
      for (int m = 0; m < G; ++m) park[(f * G + m) * S] = U[m];
    }
  }
  // forward z transforms of n (N real points -> half-complex), k_z < kc written
  auto r2c = [&](int f, float2 (&U)[G]) {
    fft_line<H, G, -1, LOGN>(U, j, xc, tw);
#pragma unroll
    for (int m = 0; m < G; ++m) xc.st(j + m * S, U[m]);
    xc.sync();
    float2* dst = w + f * MM + line * H1;
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 A = U[m];
      const float2 Bc = cconj(xc.ld((H - k) & (H - 1)));
      const float2 E = cscale(cadd(A, Bc), 0.5f);
      const float2 D = csub(A, Bc);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
      const float2 W = __ldg(&tw[k]);
      if (valid && k < KC) dst[k] = cadd(E, cmul(W, O));
    }
    xc.sync();
  };
  // n = u x omega at the two real points held by each slot:
  //   n_x = u_y w_z - u_z w_y,  n_y = u_z w_x - u_x w_z,  n_z = u_x w_y - u_y w_x
  // n_z is complete after omega_y and is transformed before omega_z is loaded.
  float2 Ny[G], Nx[G];
  {
    float2 Nz[G];
    {
      float2 W[G];
      c2r(3, W);  // omega_x
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const float2 uy = park[(1 * G + m) * S], uz = park[(2 * G + m) * S];
        Ny[m] = make_float2(uz.x * W[m].x, uz.y * W[m].y);
        Nz[m] = make_float2(-uy.x * W[m].x, -uy.y * W[m].y);
      }
      c2r(4, W);  // omega_y
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const float2 ux = park[(0 * G + m) * S], uz = park[(2 * G + m) * S];
        Nx[m] = make_float2(-uz.x * W[m].x, -uz.y * W[m].y);
        Nz[m] = make_float2(fmaf(ux.x, W[m].x, Nz[m].x), fmaf(ux.y, W[m].y, Nz[m].y));
      }
    }
    r2c(2, Nz);
  }
  {
    float2 W[G];
    c2r(5, W);  // omega_z
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const float2 ux = park[(0 * G + m) * S], uy = park[(1 * G + m) * S];
      Nx[m] = make_float2(fmaf(uy.x, W[m].x, Nx[m].x), fmaf(uy.y, W[m].y, Nx[m].y));
      Ny[m] = make_float2(fmaf(-ux.x, W[m].x, Ny[m].x), fmaf(-ux.y, W[m].y, Ny[m].y));
    }
  }
  r2c(0, Nx);
  r2c(1, Ny);
}

// ----------------------------------------------------- x pass + update -----
enum NSMode : int {
  NS_RHS = 0,
  NS_STAGE1 = 1,
  NS_STAGE2 = 2,
  NS_RK4_1 = 3,
  NS_RK4_2 = 4,
  NS_RK4_3 = 5,
  NS_RK4_4 = 6
};

struct NSUpdate {
  const float2* etab;  // exp(-nu k^2 dt) = hi + lo (two FP32 parts), indexed by integer k^2;
                       // exp(-nu k^2 dt/2) follows at offset etab_len (the RK4 half steps)
  int etab_len;
  float2* acc;         // RK4 accumulator (3 fields)
  const double* ef;    // forced-mode energy (device scalar)
  double feps;         // injected power (0 = off)
  int k2min, k2max;
  float dt;
  float scale;         // 1 / n^3
};

// One kept mode (k_x, k_y, k_z) at index idx of each field: N = P[n] (Eq. (8)),
// + subgrid force, + forcing, then
//   RHS:    out = N
//   STAGE1: out = E (u0 + dt N)                      (out = u1)
//   STAGE2: out = 1/2 E u0 + 1/2 (u1 + dt N)         (out = u0, in place)
// or one stage of RK4 with H = exp(-nu k^2 dt/2), state u0, stage state u1,
// accumulator A (N from the stage's input: u0 in RK4_1, u1 after):
//   RK4_1:  A = E u0 + dt/6 E N,   out = H (u0 + dt/2 N)   (out = u1)
//   RK4_2:  A += dt/3 H N,         out = H u0 + dt/2 N     (out = u1)
//   RK4_3:  A += dt/3 H N,         out = E u0 + dt H N     (out = u1)
//   RK4_4:  out = A + dt/6 N                                (out = u0)
__device__ __forceinline__ void ns_mode_update(float2 nx, float2 ny, float2 nz, int kx, int ky, int kz,
                                               long long idx, long long M, const NSUpdate& upd, int mode,
                                               float gforce, const float2* u0, const float2* u1,
                                               const float2* __restrict__ extra, float2* out) {
  const int k2 = kx * kx + ky * ky + kz * kz;
  if (k2 == 0) {
    nx = ny = nz = make_float2(0.f, 0.f);
  } else {
    const float fkx = (float)kx, fky = (float)ky, fkz = (float)kz;
    const float inv = 1.f / (float)k2;
    const float2 kn = make_float2((fkx * nx.x + fky * ny.x + fkz * nz.x) * inv,
                                  (fkx * nx.y + fky * ny.y + fkz * nz.y) * inv);
    nx = csub(nx, cscale(kn, fkx));
    ny = csub(ny, cscale(kn, fky));
    nz = csub(nz, cscale(kn, fkz));
  }
  if (extra) {  // subgrid force, already dealiased and projected
    nx = cadd(nx, extra[idx]);
    ny = cadd(ny, extra[idx + M]);
    nz = cadd(nz, extra[idx + 2 * M]);
  }
  const bool forced = gforce != 0.f && k2 >= upd.k2min && k2 <= upd.k2max;
  const float2* ucur = (mode == NS_STAGE2 || mode >= NS_RK4_2) ? u1 : u0;
  if (forced) {
    nx = cadd(nx, cscale(ucur[idx], gforce));
    ny = cadd(ny, cscale(ucur[idx + M], gforce));
    nz = cadd(nz, cscale(ucur[idx + 2 * M], gforce));
  }
  if (mode == NS_RHS) {
    out[idx] = nx;
    out[idx + M] = ny;
    out[idx + 2 * M] = nz;
    return;
  }
  // E = hi + lo carries the factor to ~2^-48; v * E is formed as
  // fma(v, hi, v * lo), one rounding, so repeated steps do not bias the decay.
  const float2 E = __ldg(&upd.etab[k2]);
  const float dt = upd.dt;
  const float2 n3[3] = {nx, ny, nz};
  if (mode >= NS_RK4_1) {
    const float2 H = __ldg(&upd.etab[upd.etab_len + k2]);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const long long i = idx + f * M;
      const float2 nv = n3[f];
      if (mode == NS_RK4_4) {
        const float2 a = upd.acc[i];
        out[i] = make_float2(fmaf(dt / 6.f, nv.x, a.x), fmaf(dt / 6.f, nv.y, a.y));
        continue;
      }
      const float2 a = u0[i];
      const float2 ea = make_float2(fmaf(a.x, E.x, a.x * E.y), fmaf(a.y, E.x, a.y * E.y));  // E u0
      const float2 ha = make_float2(fmaf(a.x, H.x, a.x * H.y), fmaf(a.y, H.x, a.y * H.y));  // H u0
      const float2 hn = make_float2(fmaf(nv.x, H.x, nv.x * H.y), fmaf(nv.y, H.x, nv.y * H.y));  // H N
      if (mode == NS_RK4_1) {
        const float2 en = make_float2(fmaf(nv.x, E.x, nv.x * E.y), fmaf(nv.y, E.x, nv.y * E.y));
        upd.acc[i] = make_float2(fmaf(dt / 6.f, en.x, ea.x), fmaf(dt / 6.f, en.y, ea.y));
        const float sx = a.x + 0.5f * dt * nv.x, sy = a.y + 0.5f * dt * nv.y;
        out[i] = make_float2(fmaf(sx, H.x, sx * H.y), fmaf(sy, H.x, sy * H.y));
      } else {
        const float2 ac = upd.acc[i];
        upd.acc[i] = make_float2(fmaf(dt / 3.f, hn.x, ac.x), fmaf(dt / 3.f, hn.y, ac.y));
        out[i] = (mode == NS_RK4_2) ? make_float2(fmaf(0.5f * dt, nv.x, ha.x), fmaf(0.5f * dt, nv.y, ha.y))
                                    : make_float2(fmaf(dt, hn.x, ea.x), fmaf(dt, hn.y, ea.y));
      }
    }
    return;
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float2 a = u0[idx + f * M];
    float2 r;
    if (mode == NS_STAGE1) {
      const float sx = a.x + dt * n3[f].x, sy = a.y + dt * n3[f].y;
      r = make_float2(fmaf(sx, E.x, sx * E.y), fmaf(sy, E.x, sy * E.y));
    } else {
      const float2 b = u1[idx + f * M];
      const float ex = fmaf(a.x, E.x, a.x * E.y), ey = fmaf(a.y, E.x, a.y * E.y);
      r = make_float2(0.5f * (ex + (b.x + dt * n3[f].x)), 0.5f * (ey + (b.y + dt * n3[f].y)));
    }
    out[idx + f * M] = r;
  }
}

// 5. forward x pass of the 3 nonlinear fields, then on every kept mode:
//    N = P[n] (Eq. (8)), + forcing, and
//    RHS:    out = N
//    STAGE1: out = E (u0 + dt N)                      (out = u1)
//    STAGE2: out = 1/2 E u0 + 1/2 (u1 + dt N)         (out = u0, in place)
template <int N>
__global__ void __launch_bounds__(NUCfg<N>::THREADS, NUCfg<N>::MINB)
    k_ns_fwdx(const float2* __restrict__ nh, const float2* u0, const float2* u1, float2* out,
              NSGeom g, int ktiles, NSUpdate upd, int mode, const float2* __restrict__ extra,
              const float2* __restrict__ tw) {
  constexpr long long H1 = N / 2 + 1, MM = (long long)N * N * H1;  // geometry of the n^3 grid
  constexpr int KD = (N - 1) / 3;                                  // largest kept |k| (2/3 rule)
  using C = NUCfg<N>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smn[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int dky = blockIdx.x / ktiles;
  const int kz = (blockIdx.x - dky * ktiles) * T + c;
  const bool valid = kz < (KD + 1);
  const int ay = dense_to_a(dky, N, KD);
  const long long q = (long long)ay * H1 + kz;
  const long long rs = (long long)N * H1;
  const ColX<T> xc{smn, c};
  // fields 0 and 1 are parked in shared memory after their transforms (this
  // thread's slots only), so one field at a time is held in registers
  float2* park = smn + (size_t)N * T + threadIdx.x;
  float2 V[G];
#pragma unroll 1
  for (int f = 0; f < 3; ++f) {
#pragma unroll
    for (int m = 0; m < G; ++m)
      V[m] = valid ? nh[f * MM + (j + m * S) * rs + q] : make_float2(0.f, 0.f);
    fft_line<N, G, -1>(V, j, xc, tw);
    if (f < 2) {
#pragma unroll
      for (int m = 0; m < G; ++m) park[(f * G + m) * C::THREADS] = V[m];
    }
  }
  if (!valid) return;
  const int ky = kwav(ay, N);
  float gforce = 0.f;
  if (upd.feps > 0.0) {
    const double ef = *upd.ef;
    gforce = ef > 0.0 ? (float)(upd.feps / (2.0 * ef)) : 0.f;
  }
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int pos = j + m * S;
    if (!kept_xy(pos, N, KD)) continue;
    ns_mode_update(cscale(park[m * C::THREADS], upd.scale), cscale(park[(G + m) * C::THREADS], upd.scale),
                   cscale(V[m], upd.scale), kwav(pos, N), ky, kz, pos * rs + q, MM, upd, mode, gforce, u0, u1,
                   extra, out);
  }
}

// ------------------------------------------------------------ reductions ---
// Energy of the forced modes, 1/2 sum w |u|^2 over k2min <= |k|^2 <= k2max,
// in FP64; one block, fixed order.
__global__ void k_forced_energy(const float2* __restrict__ u, NSGeom g, int kr, int k2min,
                                int k2max, double* ef) {
  __shared__ double red[256];
  const int side = 2 * kr + 1;
  const int count = side * side * (kr + 1);
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int kz = i % (kr + 1);
    const int t = i / (kr + 1);
    const int ky = t % side - kr, kx = t / side - kr;
    const int k2 = kx * kx + ky * ky + kz * kz;
    if (k2 < k2min || k2 > k2max) continue;
    const int ax = kx < 0 ? kx + g.n : kx, ay = ky < 0 ? ky + g.n : ky;
    const long long idx = ((long long)ax * g.n + ay) * g.h1 + kz;
    const double w = kz == 0 ? 1.0 : 2.0;
    double s = 0.0;
    for (int f = 0; f < 3; ++f) {
      const float2 v = u[idx + f * g.M];
      s += (double)v.x * v.x + (double)v.y * v.y;
    }
    acc += 0.5 * w * s;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *ef = red[0];
}

// nint(|k|) for integer |k|^2, exact: an FP32 square root corrected by
// integer comparisons; |k| >= K + 1/2 exactly when k2 >= K^2 + K + 1.
__device__ __forceinline__ long long shell_index(long long k2) {
  long long K = (long long)floorf(sqrtf((float)k2));
  while (K * K > k2) --K;
  while ((K + 1) * (K + 1) <= k2) ++K;
  if (k2 >= K * K + K + 1) ++K;
  return K;
}

constexpr int DIAG_WARPS = 8;
constexpr size_t kNoAllocScratchDoubles = 262144;  // 2 MiB of partials for tarang_diag_noalloc

// Blocks of the diagnostics reduction for a result of `width` doubles: up to
// eight per SM of 152, as many as the no-allocation scratch holds partials
// for (the same count on both paths, so both sum in the same order).
static int diag_blocks(int width) {
  const long long cap = (long long)(kNoAllocScratchDoubles / (size_t)width);
  return (int)(cap < 152 * 8 ? cap : 152 * 8);
}

// Unevaluated FP32 pair hi + lo.  Sums use Knuth's TwoSum and products
// the FMA-based TwoProduct (both error-free), accumulated as in Ogita, Rump
// and Oishi's Sum2/Dot2 ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 2005): the result is as accurate as a sum in twice the working
// precision (~2^-48 relative to the sum of magnitudes).  The __f*_rn
// intrinsics keep the compiler from contracting the steps into FMAs.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return F2{s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}

// a * b exactly, as a pair
__device__ __forceinline__ F2 f2_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return F2{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ double f2_to_double(F2 a) { return (double)a.hi + (double)a.lo; }

// The biased exponent field of a non-negative float (0 for zero and subnormals).
__device__ __forceinline__ int exp_field(float a) { return (__float_as_int(a) >> 23) & 0xff; }

// 2^k for k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Scale exponent that maps a warp's largest magnitude (exponent field E) to
// [2^40, 2^41): products stay below 2^82, their sums over a mode (x 2^3),
// the weight (x 2), a warp's run (x 2^5) and the factor k^2 < 2^19 of the
// dissipation below 2^128; magnitudes down to 2^-103 of the largest keep
// normal products.
__device__ __forceinline__ int warp_scale_exp(float amax) {
  const unsigned E = __reduce_max_sync(0xffffffffu, (unsigned)exp_field(amax));
  return 167 - (int)E;  // 40 - (E - 127); in [-88, 167]
}

// v * 2^k exactly (two steps keep each factor representable)
__device__ __forceinline__ float scale2(float v, int k) {
  const int k1 = k >> 1;
  return __fmul_rn(__fmul_rn(v, pow2f(k1)), pow2f(k - k1));
}

// Deterministic diagnostics over the kept modes.  A work item is 32
// consecutive k_z of one (k_x, k_y) line; along a line the shell index is
// non-decreasing, so a warp sums each shell's run with a segmented shuffle
// reduction (fixed order) and one lane adds it to the warp's FP64 histogram.
// The per-mode values and run sums are FP32 pairs: products exact, sums in
// twice the working precision, on values scaled by a power of two common to
// the warp (exact; undone in FP64).  FP64 arithmetic, slow on this GPU, is
// left to one histogram update per run.  Items are assigned to warps by a
// fixed grid stride over diag_blocks(width) blocks; partials per block are
// summed in block order by k_diag_final.
// With nh == nullptr the per-mode value is the energy 1/2 w |u|^2 (slots:
// E, eps, E(K)); otherwise it is the transfer w Re(conj(u) . nh) (slots:
// sum_K T(K), 0, T(K)).  Slot 0 is the sum of the shells.
__global__ void __launch_bounds__(DIAG_WARPS * 32)
    k_diag(const float2* __restrict__ u, const float2* __restrict__ nh, NSGeom g, double nu, int kmax,
           double* part) {
  extern __shared__ double hist[];  // [DIAG_WARPS][kmax+1]
  __shared__ double wd[DIAG_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = kmax + 1;
  for (int i = threadIdx.x; i < DIAG_WARPS * nb; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  double* h = hist + warp * nb;
  const int nchunk = (g.kc + 31) / 32;
  const long long items = (long long)g.nk * g.nk * nchunk;
  const bool dissip = !nh;
  double accD = 0.0;
  for (long long it = (long long)blockIdx.x * DIAG_WARPS + warp; it < items;
       it += (long long)gridDim.x * DIAG_WARPS) {
    const long long line = it / nchunk;
    const int chunk = (int)(it - line * nchunk);
    const int ax = dense_to_a((int)(line / g.nk), g.n, g.kd);
    const int ay = dense_to_a((int)(line % g.nk), g.n, g.kd);
    const int kz = chunk * 32 + lane;
    const bool valid = kz < g.kc;
    float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, b[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int shell = kmax + 1;
    long long k2 = 0;
    if (valid) {
      const long long idx = ((long long)ax * g.n + ay) * g.h1 + kz;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const float2 v = u[idx + f * g.M];
        a[2 * f] = v.x;
        a[2 * f + 1] = v.y;
        if (nh) {
          const float2 q = nh[idx + f * g.M];
          b[2 * f] = q.x;
          b[2 * f + 1] = q.y;
        }
      }
      const long long kx = kwav(ax, g.n), ky = kwav(ay, g.n);
      k2 = kx * kx + ky * ky + (long long)kz * kz;
      const long long K = shell_index(k2);
      shell = K <= kmax ? (int)K : kmax + 1;
    }
    float amax = 0.f, bmax = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      amax = fmaxf(amax, fabsf(a[i]));
      bmax = fmaxf(bmax, fabsf(b[i]));
    }
    const int ka = warp_scale_exp(amax);
    const int kb = nh ? warp_scale_exp(bmax) : ka;
    F2 e{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float x = scale2(a[i], ka);
      const float y = nh ? scale2(b[i], kb) : x;
      e = f2_add(e, f2_prod(x, y));
    }
    // w = 1 on k_z = 0 and k_z = n/2, else 2; the energy carries 1/2 w
    // (powers of two: exact)
    const float wf = (kz == 0 || 2 * kz == g.n) ? (nh ? 1.f : 0.5f) : (nh ? 2.f : 1.f);
    e.hi *= wf;
    e.lo *= wf;
    F2 d{0.f, 0.f};
    if (dissip) {  // k^2 e, k^2 < 2^24 exact in FP32
      const float fk2 = (float)k2;
      d = f2_prod(fk2, e.hi);
      d.lo = __fmaf_rn(fk2, e.lo, d.lo);
    }
    // segmented suffix sums over lanes with the same shell
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, e.hi, o);
      const float ol = __shfl_down_sync(0xffffffffu, e.lo, o);
      float dh = 0.f, dl = 0.f;
      if (dissip) {
        dh = __shfl_down_sync(0xffffffffu, d.hi, o);
        dl = __shfl_down_sync(0xffffffffu, d.lo, o);
      }
      const int os = __shfl_down_sync(0xffffffffu, shell, o);
      if (lane + o < 32 && os == shell) {
        e = f2_add(e, F2{oh, ol});
        if (dissip) d = f2_add(d, F2{dh, dl});
      }
    }
    const int prev = __shfl_up_sync(0xffffffffu, shell, 1);
    if (valid && shell <= kmax && (lane == 0 || prev != shell)) {
      // undo the scale: 2^-(ka + kb) in FP64 (exact)
      const double un = __longlong_as_double((long long)(1023 - ka - kb) << 52);
      h[shell] += f2_to_double(e) * un;
      if (dissip) accD += f2_to_double(d) * un;
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) accD += __shfl_down_sync(0xffffffffu, accD, o);
  if (lane == 0) wd[warp] = accD;
  __syncthreads();
  double* out = part + (long long)blockIdx.x * (2 + nb);
  for (int s = threadIdx.x; s < nb; s += blockDim.x) {
    double t = 0.0;
    for (int w2 = 0; w2 < DIAG_WARPS; ++w2) t += hist[w2 * nb + s];
    out[2 + s] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int s = 0; s < nb; ++s) a += out[2 + s];
    for (int w2 = 0; w2 < DIAG_WARPS; ++w2) b += wd[w2];
    out[0] = a;
    out[1] = 2.0 * nu * b;
  }
}

__global__ void k_diag_final(const double* __restrict__ part, int width, int nblocks, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= width) return;
  double t = 0.0;
  for (int b = 0; b < nblocks; ++b) t += part[(long long)b * width + s];
  out[s] = t;
}

// ------------------------------------------------------------ workspace ----
struct NSWork {
  NSGeom g;
  float2* w = nullptr;     // 6 fields
  float2* u1 = nullptr;    // 3 fields
  float2* etab = nullptr;  // exp(-nu k^2 dt) as hi + lo, k^2 in [0, 3 kd^2]
  int etab_len = 0;
  double etab_nu = -1.0, etab_dt = -1.0;
  double* ef = nullptr;    // forced energy
  double* part = nullptr;  // diag partials
  double* dout = nullptr;  // diag result (device)
  double* hout = nullptr;  // diag result (pinned host)
  fftk_sgs_work* sgs = nullptr;  // learned-closure scratch
  float* r6 = nullptr;     // 6 real fields (unfused split-precision right-hand side)
  float* r3 = nullptr;     // 3 real fields (shell-to-shell transfer: the advection term)
  float2* acc = nullptr;   // 3 fields (RK4 accumulator)
  double* sout = nullptr;  // per-giver shell sums of the shell-to-shell transfer
  int sout_rows = 0;
  int kmax = 0;
  int diag_smem = 0;
};

static int ns_kmax(int n) { return (int)std::floor(std::sqrt(3.0) * (n / 2) + 0.5) + 1; }

static NSGeom make_geom(int n) {
  NSGeom g;
  g.n = n;
  g.h1 = n / 2 + 1;
  g.kd = (n - 1) / 3;
  g.kc = g.kd + 1;
  g.nk = 2 * g.kd + 1;
  g.M = (long long)n * n * g.h1;
  return g;
}

// The dynamic shared-memory limit is an attribute of the kernel (per device),
// not of a plan: it is raised once per device to what the largest grid needs,
// so that no plan lowers it under another plan's launches.
static cudaError_t diag_attr() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  const int smem = (int)(sizeof(double) * DIAG_WARPS * (ns_kmax(1024) + 1));
  e = cudaFuncSetAttribute(k_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

static fftk_status ns_ensure(fftk_plan p) {
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->ns) return FFTK_OK;
  NSWork* s = new (std::nothrow) NSWork;
  if (!s) return FFTK_ERR_OOM;
  s->g = make_geom(p->nx);
  s->kmax = ns_kmax(p->nx);
  s->etab_len = 3 * s->g.kd * s->g.kd + 1;
  const size_t fb = sizeof(float2) * (size_t)s->g.M;
  const int width = 2 + s->kmax + 1;
  cudaError_t e = cudaMalloc(&s->w, 6 * fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->u1, 3 * fb);
  if (e == cudaSuccess) e = cudaMemset(s->u1, 0, 3 * fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->etab, sizeof(float2) * 2 * (size_t)s->etab_len);
  if (e == cudaSuccess) e = cudaMalloc(&s->ef, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s->ef, 0, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->part, sizeof(double) * (size_t)diag_blocks(width) * width);
  if (e == cudaSuccess) e = cudaMalloc(&s->dout, sizeof(double) * (size_t)width);
  if (e == cudaSuccess) e = cudaMallocHost(&s->hout, sizeof(double) * (size_t)width);
  s->diag_smem = (int)(sizeof(double) * DIAG_WARPS * (s->kmax + 1));
  if (e == cudaSuccess) e = diag_attr();
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->w);
    cudaFree(s->u1);
    cudaFree(s->etab);
    cudaFree(s->ef);
    cudaFree(s->part);
    cudaFree(s->dout);
    if (s->hout) cudaFreeHost(s->hout);
    delete s;
    return e == cudaErrorMemoryAllocation ? FFTK_ERR_OOM : FFTK_ERR_CUDA;
  }
  p->ns = s;
  return FFTK_OK;
}

// exp(-nu k^2 dt) for integer k^2, FP64 on the host, split into an FP32 pair
// hi = fl(E), lo = fl(E - hi).
static fftk_status ns_etab(fftk_plan p, double nu, double dt) {
  NSWork* s = p->ns;
  if (s->etab_nu == nu && s->etab_dt == dt) return FFTK_OK;
  std::vector<float2> h(2 * (size_t)s->etab_len);
  for (int half = 0; half < 2; ++half)
    for (int k2 = 0; k2 < s->etab_len; ++k2) {
      const double E = std::exp(-nu * (double)k2 * (half ? 0.5 * dt : dt));
      const float hi = (float)E;
      h[(size_t)half * s->etab_len + k2] = make_float2(hi, (float)(E - (double)hi));
    }
  cudaError_t e = cudaMemcpy(s->etab, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return from_cuda(e);
  s->etab_nu = nu;
  s->etab_dt = dt;
  return FFTK_OK;
}

// --------------------------------------------------------------- launchers --
template <int N>
struct NSLaunch {
  static cudaError_t attrs() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
      const int sx = (int)NXCfg<N>::SMEM;
      err = cudaFuncSetAttribute(k_ns_invx<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)NICfg<N>::SMEM);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_ypass<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_ypass<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_fwdx<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)NUCfg<N>::SMEM);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_z<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)NZCfg<N>::SMEM);
    });
    return err;
  }

  // One evaluation of N(u) followed by the update selected by `mode`.
  static cudaError_t rhs(fftk_plan p, const float2* u, const float2* u0, const float2* u1,
                         float2* out, const NSUpdate& upd, int mode, const float2* extra,
                         cudaStream_t st) {
    using X = NXCfg<N>;
    using F = NFCfg<N>;
    using Z = NZCfg<N>;
    cudaError_t e = attrs();
    if (e != cudaSuccess) return e;
    NSWork* s = p->ns;
    const NSGeom g = s->g;
    const int kx = (g.kc + X::T - 1) / X::T;
    const int kf = (g.kc + F::T - 1) / F::T;
    using I = NICfg<N>;
    const int ki = (g.kc + I::T - 1) / I::T;
    using U = NUCfg<N>;
    const int ku = (g.kc + U::T - 1) / U::T;
    {
      LaunchScope ls(p, KK_NS_INVX, st);
      k_ns_invx<N><<<g.nk * ki, I::THREADS, I::SMEM, st>>>(u, s->w, g, ki, twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_INVY, st);
      k_ns_ypass<N, 1><<<6 * N * kx, X::THREADS, X::SMEM, st>>>(s->w, g, kx, twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_Z, st);
      const long long lines = (long long)N * N;
      k_ns_z<N><<<(unsigned)((lines + Z::LPC - 1) / Z::LPC), Z::THREADS, Z::SMEM, st>>>(s->w, g,
                                                                                       twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_FWDY, st);
      k_ns_ypass<N, -1><<<3 * N * kx, X::THREADS, X::SMEM, st>>>(s->w, g, kx, twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_FWDX, st);
      k_ns_fwdx<N><<<g.nk * ku, U::THREADS, U::SMEM, st>>>(s->w, u0, u1, out, g, ku, upd, mode,
                                                          extra, twiddles(p, N));
    }
    return cudaGetLastError();
  }
};

// ---------------------------------------------- split-precision NS step ----
// Plans of dtype FFTK_R32_SPLIT16 evaluate the right-hand side unfused through
// the library's own transforms, whose radix-16 stages then run on the tensor
// cores: u and omega = i k x u on the spectrum, c2r of the six fields, n = u x
// omega in real space, r2c of n, and the per-mode update of the fused path.

// w6 = (u, i k x u); the derivative of the Nyquist wavenumber is 0
__global__ void k_curl_full(const float2* __restrict__ u, float2* __restrict__ w6, NSGeom g) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    const int ka = kwav(a, g.n), kb = kwav(b, g.n);
    const float kx = (2 * abs(ka) == g.n) ? 0.f : (float)ka, ky = (2 * abs(kb) == g.n) ? 0.f : (float)kb;
    const float kz = (2 * c == g.n) ? 0.f : (float)c;
    const float2 ux = u[idx], uy = u[idx + g.M], uz = u[idx + 2 * g.M];
    w6[idx] = ux;
    w6[idx + g.M] = uy;
    w6[idx + 2 * g.M] = uz;
    w6[idx + 3 * g.M] = csub(mul_i(uz, ky), mul_i(uy, kz));
    w6[idx + 4 * g.M] = csub(mul_i(ux, kz), mul_i(uz, kx));
    w6[idx + 5 * g.M] = csub(mul_i(uy, kx), mul_i(ux, ky));
  }
}

// n = u x omega in place of u (fields 0..2 of the six real fields)
__global__ void k_cross_real(float* __restrict__ r6, long long R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R;
       i += (long long)gridDim.x * blockDim.x) {
    const float ux = r6[i], uy = r6[R + i], uz = r6[2 * R + i];
    const float wx = r6[3 * R + i], wy = r6[4 * R + i], wz = r6[5 * R + i];
    r6[i] = uy * wz - uz * wy;
    r6[R + i] = uz * wx - ux * wz;
    r6[2 * R + i] = ux * wy - uy * wx;
  }
}

// the update of every kept mode from n_hat (already scaled by the transform)
__global__ void k_update_full(const float2* __restrict__ nh, const float2* u0, const float2* u1, float2* out,
                              NSGeom g, NSUpdate upd, int mode, const float2* __restrict__ extra) {
  float gforce = 0.f;
  if (upd.feps > 0.0) {
    const double ef = *upd.ef;
    gforce = ef > 0.0 ? (float)(upd.feps / (2.0 * ef)) : 0.f;
  }
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    if (!(kept_xy(a, g.n, g.kd) && kept_xy(b, g.n, g.kd) && c < g.kc)) continue;
    ns_mode_update(nh[idx], nh[idx + g.M], nh[idx + 2 * g.M], kwav(a, g.n), kwav(b, g.n), c, idx, g.M, upd, mode,
                   gforce, u0, u1, extra, out);
  }
}

static cudaError_t ns_rhs_split(fftk_plan p, const float2* u, const float2* u0, const float2* u1, float2* out,
                                const NSUpdate& upd, int mode, const float2* extra, cudaStream_t st) {
  NSWork* s = p->ns;
  const NSGeom g = s->g;
  const long long R = (long long)g.n * g.n * g.n;
  if (!s->r6) {
    cudaError_t e = cudaMalloc(&s->r6, sizeof(float) * 6 * (size_t)R);
    if (e != cudaSuccess) return e;
  }
  const unsigned grid = 152 * 8;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_curl_full<<<grid, 256, 0, st>>>(u, s->w, g);
  }
  if (fftk_c2r(p, s->w, s->r6, 6, st) != FFTK_OK) return cudaErrorLaunchFailure;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_cross_real<<<grid, 256, 0, st>>>(s->r6, R);
  }
  if (fftk_r2c(p, s->r6, s->w, 3, st) != FFTK_OK) return cudaErrorLaunchFailure;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_update_full<<<grid, 256, 0, st>>>(s->w, u0, u1, out, g, upd, mode, extra);
  }
  return cudaGetLastError();
}

// ------------------------------------------- shell-to-shell transfer ----
// The giver shell's gradient for one component i: w3[j] = i k_j u_i on the
// kept modes with kmin <= nint|k| < kmax_excl, 0 elsewhere.
__global__ void k_shell_grad(const float2* __restrict__ u, float2* __restrict__ w3, NSGeom g, int comp, int kmin,
                             int kmax_excl) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
    if (kept_xy(a, g.n, g.kd) && kept_xy(b, g.n, g.kd) && c < g.kc) {
      const long long kx = kwav(a, g.n), ky = kwav(b, g.n);
      const long long K = shell_index(kx * kx + ky * ky + (long long)c * c);
      if (K >= kmin && K < kmax_excl) {
        const float2 v = u[idx + comp * g.M];
        gx = mul_i(v, (float)kx);
        gy = mul_i(v, (float)ky);
        gz = mul_i(v, (float)c);
      }
    }
    w3[idx] = gx;
    w3[idx + g.M] = gy;
    w3[idx + 2 * g.M] = gz;
  }
}

// p = u_j G_j (real space): one component of (u . grad) u_giver
__global__ void k_shell_advect(const float* __restrict__ ur, const float* __restrict__ gr, float* __restrict__ p,
                               long long R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = ur[i] * gr[i] + ur[R + i] * gr[R + i] + ur[2 * R + i] * gr[2 * R + i];
}

#define NS_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

static cudaError_t ns_rhs_dispatch(fftk_plan p, const float2* u, const float2* u0, const float2* u1,
                                   float2* out, const NSUpdate& upd, int mode, const float2* extra,
                                   cudaStream_t st) {
  if (p->dtype == FFTK_R32_SPLIT16) return ns_rhs_split(p, u, u0, u1, out, upd, mode, extra, st);
  switch (p->nx) {
#define CASE(n) \
  case n:       \
    return NSLaunch<n>::rhs(p, u, u0, u1, out, upd, mode, extra, st);
    NS_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

static cudaError_t forced_energy(fftk_plan p, const float2* u, const tarang_params* prm,
                                 cudaStream_t st) {
  int kr = 0;
  while ((kr + 1) * (kr + 1) <= prm->force_k2max) ++kr;
  LaunchScope ls(p, KK_NS_REDUCE, st);
  k_forced_energy<<<1, 256, 0, st>>>(u, p->ns->g, kr, prm->force_k2min, prm->force_k2max,
                                     p->ns->ef);
  return cudaGetLastError();
}

static cudaError_t diag_launch(fftk_plan p, const float2* u, const float2* nh, double nu, cudaStream_t st) {
  NSWork* s = p->ns;
  const int width = 2 + s->kmax + 1;
  {
    LaunchScope ls(p, KK_NS_REDUCE, st);
    k_diag<<<diag_blocks(width), DIAG_WARPS * 32, s->diag_smem, st>>>(u, nh, s->g, nu, s->kmax, s->part);
  }
  {
    LaunchScope ls(p, KK_NS_REDUCE, st);
    k_diag_final<<<(width + 127) / 128, 128, 0, st>>>(s->part, width, diag_blocks(width), s->dout);
  }
  return cudaGetLastError();
}

static bool misaligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0; }

static fftk_status ns_check(fftk_plan p, const tarang_params* prm, bool need_dt) {
  if (!p || !prm) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (p->nx < 8 || p->nx > 1024) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (!(prm->nu >= 0.0) || !std::isfinite(prm->nu)) return FFTK_ERR_INVALID_ARG;
  if (need_dt && (!(prm->dt > 0.0) || !std::isfinite(prm->dt))) return FFTK_ERR_INVALID_ARG;
  if (prm->sgs_model && !prm->sgs_model->params) return FFTK_ERR_INVALID_ARG;
  if (prm->scheme != TARANG_RK2 && prm->scheme != TARANG_RK4) return FFTK_ERR_INVALID_ARG;
  if (prm->force_eps != 0.0) {
    const int kd = (p->nx - 1) / 3;
    if (!(prm->force_eps > 0.0) || prm->force_k2min < 1 || prm->force_k2max < prm->force_k2min ||
        prm->force_k2max > kd * kd)
      return FFTK_ERR_INVALID_ARG;
  }
  return FFTK_OK;
}

}  // namespace fftk

using namespace fftk;

void ns_free(fftk_plan p) {
  NSWork* s = p->ns;
  if (!s) return;
  cudaFree(s->w);
  cudaFree(s->u1);
  cudaFree(s->etab);
  cudaFree(s->ef);
  cudaFree(s->part);
  cudaFree(s->dout);
  if (s->hout) cudaFreeHost(s->hout);
  cudaFree(s->r6);
  cudaFree(s->r3);
  cudaFree(s->acc);
  cudaFree(s->sout);
  sgs_free(s->sgs);
  delete s;
  p->ns = nullptr;
}

extern "C" int tarang_diag_kmax(fftk_plan p) { return p ? ns_kmax(p->nx) : -1; }

extern "C" fftk_status tarang_ns_rhs(fftk_plan p, const void* uhat, void* nhat,
                                     const tarang_params* prm, void* cuda_stream) {
  fftk_status s = ns_check(p, prm, false);
  if (s != FFTK_OK) return s;
  if (!uhat || !nhat || uhat == nhat || misaligned16(uhat) || misaligned16(nhat))
    return FFTK_ERR_INVALID_ARG;
  s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const NSGeom g = p->ns->g;
  const float2* u = static_cast<const float2*>(uhat);
  float2* out = static_cast<float2*>(nhat);
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float2) * 3 * (size_t)g.M, st);
  NSUpdate upd{p->ns->etab, p->ns->etab_len, nullptr, p->ns->ef, prm->force_eps, prm->force_k2min,
               prm->force_k2max, 0.f,
               (float)(1.0 / ((double)g.n * g.n * g.n))};
  if (e == cudaSuccess && prm->force_eps > 0.0) e = forced_energy(p, u, prm, st);
  const float2* extra = nullptr;
  if (e == cudaSuccess && prm->sgs_model) e = sgs_term(p, &p->ns->sgs, u, prm->sgs_model, st, &extra);
  if (e == cudaSuccess) e = ns_rhs_dispatch(p, u, u, nullptr, out, upd, NS_RHS, extra, st);
  return from_cuda(e);
}

extern "C" fftk_status tarang_diag(fftk_plan p, const void* uhat, double nu, double* diag_host,
                                   void* cuda_stream) {
  if (!p || !uhat || !diag_host || misaligned16(uhat)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || p->nx > 1024)
    return FFTK_ERR_UNSUPPORTED_SIZE;
  fftk_status s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NSWork* w = p->ns;
  const int width = 2 + w->kmax + 1;
  cudaError_t e = diag_launch(p, static_cast<const float2*>(uhat), nullptr, nu, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->hout, w->dout, sizeof(double) * width, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  std::memcpy(diag_host, w->hout, sizeof(double) * width);
  return std::isfinite(diag_host[0]) ? FFTK_OK : FFTK_ERR_NONFINITE;
}

extern "C" fftk_status tarang_transfer(fftk_plan p, const void* uhat, const tarang_params* prm,
                                       double* out_host, void* cuda_stream) {
  if (!p || !uhat || !out_host || misaligned16(uhat)) return FFTK_ERR_INVALID_ARG;
  tarang_params none{};
  fftk_status s = ns_check(p, prm ? prm : &none, false);
  if (s != FFTK_OK) return s;
  s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NSWork* w = p->ns;
  const int nb = w->kmax + 1, width = 2 + nb;
  // the right-hand side goes to the stage buffer, free between steps
  s = tarang_ns_rhs(p, uhat, w->u1, prm ? prm : &none, cuda_stream);
  if (s != FFTK_OK) return s;
  cudaError_t e = diag_launch(p, static_cast<const float2*>(uhat), w->u1, 0.0, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->hout, w->dout, sizeof(double) * width, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  out_host[0] = w->hout[0];
  double pi = 0.0;
  for (int K = 0; K < nb; ++K) {
    out_host[1 + K] = w->hout[2 + K];
    pi -= w->hout[2 + K];
    out_host[1 + nb + K] = pi;
  }
  return std::isfinite(out_host[0]) ? FFTK_OK : FFTK_ERR_NONFINITE;
}

extern "C" fftk_status tarang_shell_transfer(fftk_plan p, const void* uhat, int nshells, const int* bounds,
                                             double* out_host, void* cuda_stream) {
  if (!p || !uhat || !bounds || !out_host || misaligned16(uhat)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || p->nx > 1024) return FFTK_ERR_UNSUPPORTED_SIZE;
  const int kmax = ns_kmax(p->nx);
  if (nshells < 1 || nshells > kmax + 1 || bounds[0] < 0 || bounds[nshells] > kmax + 1)
    return FFTK_ERR_INVALID_ARG;
  for (int i = 0; i < nshells; ++i)
    if (bounds[i + 1] <= bounds[i]) return FFTK_ERR_INVALID_ARG;
  fftk_status st0 = ns_ensure(p);
  if (st0 != FFTK_OK) return st0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NSWork* s = p->ns;
  const NSGeom g = s->g;
  const long long R = (long long)g.n * g.n * g.n;
  const int nb = s->kmax + 1, width = 2 + nb;
  cudaError_t e = cudaSuccess;
  if (!s->r6) e = cudaMalloc(&s->r6, sizeof(float) * 6 * (size_t)R);
  if (e == cudaSuccess && !s->r3) e = cudaMalloc(&s->r3, sizeof(float) * 3 * (size_t)R);
  if (e == cudaSuccess && s->sout_rows < nshells) {
    cudaFree(s->sout);
    s->sout = nullptr;
    s->sout_rows = 0;
    e = cudaMalloc(&s->sout, sizeof(double) * (size_t)nshells * width);
    if (e == cudaSuccess) s->sout_rows = nshells;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FFTK_ERR_OOM : FFTK_ERR_CUDA;
  }
  const float2* u = static_cast<const float2*>(uhat);
  float* ur = s->r6;                 // u in real space
  float* gr = s->r6 + 3 * R;         // one row of the giver's gradient in real space
  float2* gh = s->w;                 // the same row on the spectrum
  float2* ph = s->w + 3 * g.M;       // (u . grad) u_giver on the spectrum
  const unsigned grid = 152 * 8;
  // the largest nint|k| among the kept modes: givers beyond it are empty
  const int kd = g.kd;
  const int kfar = (int)std::floor(std::sqrt(3.0 * kd * kd) + 0.5);
  if (fftk_c2r(p, u, ur, 3, cuda_stream) != FFTK_OK) return FFTK_ERR_CUDA;
  std::vector<char> live(nshells, 0);
  for (int gi = 0; gi < nshells && e == cudaSuccess; ++gi) {
    if (bounds[gi] > kfar) continue;
    live[gi] = 1;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
      {
        LaunchScope ls(p, KK_AUX, st);
        k_shell_grad<<<grid, 256, 0, st>>>(u, gh, g, i, bounds[gi], bounds[gi + 1]);
      }
      if (fftk_c2r(p, gh, gr, 3, cuda_stream) != FFTK_OK) return FFTK_ERR_CUDA;
      {
        LaunchScope ls(p, KK_AUX, st);
        k_shell_advect<<<grid, 256, 0, st>>>(ur, gr, s->r3 + i * R, R);
      }
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) break;
    if (fftk_r2c(p, s->r3, ph, 3, cuda_stream) != FFTK_OK) return FFTK_ERR_CUDA;
    {
      LaunchScope ls(p, KK_NS_REDUCE, st);
      k_diag<<<diag_blocks(width), DIAG_WARPS * 32, s->diag_smem, st>>>(u, ph, g, 0.0, s->kmax, s->part);
    }
    {
      LaunchScope ls(p, KK_NS_REDUCE, st);
      k_diag_final<<<(width + 127) / 128, 128, 0, st>>>(s->part, width, diag_blocks(width),
                                                         s->sout + (size_t)gi * width);
    }
    e = cudaGetLastError();
  }
  std::vector<double> h((size_t)nshells * width, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), s->sout, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  // T[r][g] = -sum over the receiver's integer shells of w Re(conj(u) . (u . grad) u_g)
  bool finite = true;
  for (int r = 0; r < nshells; ++r)
    for (int gi = 0; gi < nshells; ++gi) {
      double t = 0.0;
      if (live[gi])
        for (int K = bounds[r]; K < bounds[r + 1]; ++K) t -= h[(size_t)gi * width + 2 + K];
      out_host[(size_t)r * nshells + gi] = t;
      finite = finite && std::isfinite(t);
    }
  return finite ? FFTK_OK : FFTK_ERR_NONFINITE;
}

extern "C" fftk_status tarang_ns_step(fftk_plan p, void* uhat, const tarang_params* prm, int nsteps,
                                      double* diag_host, void* cuda_stream) {
  fftk_status s = ns_check(p, prm, true);
  if (s != FFTK_OK) return s;
  if (!uhat || nsteps < 0 || misaligned16(uhat)) return FFTK_ERR_INVALID_ARG;
  s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  s = ns_etab(p, prm->nu, prm->dt);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NSWork* w = p->ns;
  const NSGeom g = w->g;
  float2* u = static_cast<float2*>(uhat);
  if (prm->scheme == TARANG_RK4 && !w->acc) {
    cudaError_t ea = cudaMalloc(&w->acc, sizeof(float2) * 3 * (size_t)g.M);
    if (ea != cudaSuccess) {
      cudaGetLastError();
      return from_cuda(ea);
    }
  }
  NSUpdate upd{w->etab, w->etab_len, w->acc, w->ef, prm->force_eps, prm->force_k2min, prm->force_k2max,
               (float)prm->dt, (float)(1.0 / ((double)g.n * g.n * g.n))};
  cudaError_t e = cudaSuccess;
  if (prm->scheme == TARANG_RK4) {
    // four evaluations of N: from u, then from the stage state u1
    for (int it = 0; it < nsteps && e == cudaSuccess; ++it)
      for (int stage = 0; stage < 4 && e == cudaSuccess; ++stage) {
        const float2* in = stage == 0 ? u : w->u1;
        const float2* extra = nullptr;
        if (prm->force_eps > 0.0) e = forced_energy(p, in, prm, st);
        if (e == cudaSuccess && prm->sgs_model) e = sgs_term(p, &w->sgs, in, prm->sgs_model, st, &extra);
        if (e == cudaSuccess)
          e = ns_rhs_dispatch(p, in, u, w->u1, stage == 3 ? u : w->u1, upd, NS_RK4_1 + stage, extra, st);
      }
    if (e != cudaSuccess) return from_cuda(e);
    if (diag_host) return tarang_diag(p, u, prm->nu, diag_host, cuda_stream);
    return FFTK_OK;
  }
  for (int it = 0; it < nsteps && e == cudaSuccess; ++it) {
    const float2* extra = nullptr;
    if (prm->force_eps > 0.0) e = forced_energy(p, u, prm, st);
    if (e == cudaSuccess && prm->sgs_model) e = sgs_term(p, &w->sgs, u, prm->sgs_model, st, &extra);
    if (e == cudaSuccess) e = ns_rhs_dispatch(p, u, u, nullptr, w->u1, upd, NS_STAGE1, extra, st);
    if (e == cudaSuccess && prm->force_eps > 0.0) e = forced_energy(p, w->u1, prm, st);
    if (e == cudaSuccess && prm->sgs_model) e = sgs_term(p, &w->sgs, w->u1, prm->sgs_model, st, &extra);
    if (e == cudaSuccess) e = ns_rhs_dispatch(p, w->u1, u, w->u1, u, upd, NS_STAGE2, extra, st);
  }
  if (e != cudaSuccess) return from_cuda(e);
  if (diag_host) return tarang_diag(p, u, prm->nu, diag_host, cuda_stream);
  return FFTK_OK;
}

// --------------------------------------------------------- initial field ---
namespace fftk {

// Zero every mode outside the 2/3 set and project the kept ones (Eq. (8)).
__global__ void k_ic_shape(float2* u, NSGeom g) {
  const long long total = g.M;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % g.h1);
    const long long ab = i / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    if (!(kept_xy(a, g.n, g.kd) && kept_xy(b, g.n, g.kd) && c < g.kc)) {
      u[i] = u[i + g.M] = u[i + 2 * g.M] = make_float2(0.f, 0.f);
      continue;
    }
    const float kx = (float)kwav(a, g.n), ky = (float)kwav(b, g.n), kz = (float)c;
    const float k2 = kx * kx + ky * ky + kz * kz;
    if (k2 == 0.f) {
      u[i] = u[i + g.M] = u[i + 2 * g.M] = make_float2(0.f, 0.f);
      continue;
    }
    const float2 ux = u[i], uy = u[i + g.M], uz = u[i + 2 * g.M];
    const float2 kd = make_float2((kx * ux.x + ky * uy.x + kz * uz.x) / k2,
                                  (kx * ux.y + ky * uy.y + kz * uz.y) / k2);
    u[i] = csub(ux, cscale(kd, kx));
    u[i + g.M] = csub(uy, cscale(kd, ky));
    u[i + 2 * g.M] = csub(uz, cscale(kd, kz));
  }
}

// Make the k_z = 0 plane exactly Hermitian: f(-kx,-ky) = conj f(kx,ky).
__global__ void k_ic_herm(float2* u, NSGeom g) {
  const long long total = 3LL * g.n * g.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / ((long long)g.n * g.n));
    const int ab = (int)(i % ((long long)g.n * g.n));
    const int a = ab / g.n, b = ab % g.n;
    const int a2 = (g.n - a) % g.n, b2 = (g.n - b) % g.n;
    const long long i1 = ((long long)a * g.n + b) * g.h1, i2 = ((long long)a2 * g.n + b2) * g.h1;
    if (i2 < i1) continue;
    float2* base = u + f * g.M;
    if (i1 == i2) {
      base[i1].y = 0.f;
    } else {
      const float2 p = base[i1], q = base[i2];
      const float2 avg = make_float2(0.5f * (p.x + q.x), 0.5f * (p.y - q.y));
      base[i1] = avg;
      base[i2] = cconj(avg);
    }
  }
}

// u *= s[nint|k|] on the kept modes.
__global__ void k_ic_rescale(float2* u, NSGeom g, const double* __restrict__ s, int kmax) {
  const long long total = (long long)g.nk * g.nk * g.kc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(i % g.kc);
    const long long t = i / g.kc;
    const int a = dense_to_a((int)(t / g.nk), g.n, g.kd), b = dense_to_a((int)(t % g.nk), g.n, g.kd);
    const long long kx = kwav(a, g.n), ky = kwav(b, g.n);
    const long long k2 = kx * kx + ky * ky + (long long)kz * kz;
    long long K = (long long)floor(sqrt((double)k2));
    while (K * K > k2) --K;
    while ((K + 1) * (K + 1) <= k2) ++K;
    if (k2 >= K * K + K + 1) ++K;
    const float sc = K <= kmax ? (float)s[K] : 0.f;
    const long long idx = ((long long)a * g.n + b) * g.h1 + kz;
    for (int f = 0; f < 3; ++f) u[idx + f * g.M] = cscale(u[idx + f * g.M], sc);
  }
}

}  // namespace fftk

extern "C" fftk_status tarang_ic_random(fftk_plan p, const float* normals, void* uhat, double k0,
                                        double E0, void* cuda_stream) {
  if (!p || !normals || !uhat || !(k0 > 0.0) || !(E0 > 0.0) || !std::isfinite(k0) ||
      !std::isfinite(E0))
    return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || p->nx > 1024)
    return FFTK_ERR_UNSUPPORTED_SIZE;
  fftk_status s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NSWork* w = p->ns;
  const NSGeom g = w->g;
  float2* u = static_cast<float2*>(uhat);
  s = fftk_r2c(p, normals, uhat, 3, cuda_stream);
  if (s != FFTK_OK) return s;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_ic_shape<<<152 * 8, 256, 0, st>>>(u, g);
  }
  {
    LaunchScope ls(p, KK_AUX, st);
    k_ic_herm<<<152 * 4, 256, 0, st>>>(u, g);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return from_cuda(e);
  const int kmax = w->kmax;
  std::vector<double> d((size_t)(2 + kmax + 1));
  s = tarang_diag(p, uhat, 0.0, d.data(), cuda_stream);
  if (s != FFTK_OK) return s;
  // per-shell factors so that E(K) ~ K^4 exp(-2 (K/k0)^2), then total E0
  std::vector<double> sc((size_t)kmax + 1, 0.0);
  double tsum = 0.0;
  for (int K = 1; K <= kmax; ++K) {
    const double eK = d[(size_t)(2 + K)];
    if (eK > 0.0) {
      const double t = std::pow((double)K, 4.0) * std::exp(-2.0 * ((double)K / k0) * ((double)K / k0));
      sc[(size_t)K] = std::sqrt(t / eK);
      tsum += t;
    }
  }
  if (!(tsum > 0.0)) return FFTK_ERR_NONFINITE;
  const double gscale = std::sqrt(E0 / tsum);
  for (auto& v : sc) v *= gscale;
  double* dsc = nullptr;
  e = cudaMalloc(&dsc, sizeof(double) * sc.size());
  if (e == cudaSuccess) e = cudaMemcpy(dsc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    LaunchScope ls(p, KK_AUX, st);
    k_ic_rescale<<<152 * 8, 256, 0, st>>>(u, g, dsc, kmax);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dsc) cudaFree(dsc);
  return from_cuda(e);
}

// Dealias and project a caller's state (Eq. (8) and the 2/3 rule): the entry
// point that turns any transformed velocity, e.g. a filtered resolved field on
// a coarse grid, into a valid solver state.
extern "C" fftk_status tarang_dealias_project(fftk_plan p, void* uhat, void* cuda_stream) {
  if (!p || !uhat || misaligned16(uhat)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || p->nx > 1024)
    return FFTK_ERR_UNSUPPORTED_SIZE;
  fftk_status s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  {
    LaunchScope ls(p, KK_AUX, st);
    k_ic_shape<<<152 * 8, 256, 0, st>>>(static_cast<float2*>(uhat), p->ns->g);
  }
  return from_cuda(cudaGetLastError());
}

// ------------------------------------------- diagnostics without allocation --
// Callers that cannot allocate device memory (a real-time loop that must not
// pay cudaMalloc's implicit device synchronisation, or a host application
// whose memory manager forbids allocations it does not own) get the same
// FP64 diagnostics through tarang_diag_noalloc.  Its scratch space, the
// per-block partial sums, lives in this file-scope array for the life of the
// process on every device that loads the library.
namespace fftk {

static __device__ __align__(256) double g_diag_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (the host-side symbol is only a stand-in), with the reduction
// kernel's shared-memory limit raised for the largest n.
static fftk_status noalloc_setup(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return from_cuda(e);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return FFTK_ERR_UNSUPPORTED_SIZE;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_diag_scratch);
    if (e != cudaSuccess) return from_cuda(e);
    e = diag_attr();
    if (e != cudaSuccess) return from_cuda(e);
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return FFTK_OK;
}

}  // namespace fftk

extern "C" fftk_status tarang_diag_noalloc(int n, const void* uhat, double nu, double* diag_dev,
                                           void* cuda_stream) {
  if (!uhat || !diag_dev || misaligned16(uhat) ||
      (reinterpret_cast<uintptr_t>(diag_dev) & 7u) != 0 || !(nu >= 0.0) || !std::isfinite(nu))
    return FFTK_ERR_INVALID_ARG;
  if (!is_pow2(n) || n < 8 || n > 1024) return FFTK_ERR_UNSUPPORTED_SIZE;
  const int kmax = ns_kmax(n);
  const int width = 2 + kmax + 1;
  if ((size_t)diag_blocks(width) * (size_t)width > kNoAllocScratchDoubles) return FFTK_ERR_UNSUPPORTED_SIZE;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return FFTK_ERR_NO_DEVICE;
  }
  double* scratch = nullptr;
  fftk_status s = noalloc_setup(&scratch);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const NSGeom g = make_geom(n);
  // Every entry of the partials that k_diag_final reads is written by k_diag
  // in the same call, so nothing in the shared scratch needs clearing.
  const int smem = (int)(sizeof(double) * DIAG_WARPS * (kmax + 1));
  k_diag<<<diag_blocks(width), DIAG_WARPS * 32, smem, st>>>(static_cast<const float2*>(uhat), nullptr, g, nu, kmax,
                                                   scratch);
  k_diag_final<<<(width + 127) / 128, 128, 0, st>>>(scratch, width, diag_blocks(width), diag_dev);
  return from_cuda(cudaGetLastError());
}
