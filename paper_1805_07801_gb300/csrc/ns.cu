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
// The 2/3 rule is used throughout, not only to zero the products: modes
// with 3|k| >= n on any axis are zero in the state, so every pass reads only
// the rows and columns that can be nonzero and writes only those a later
// pass reads.  The arrays keep the full [n][n][n/2+1] layout; the untouched
// parts are never read.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft_engine.cuh"
#include "internal.h"
#include "ns_common.cuh"
#include "tcgen05.cuh"

namespace fftk {
// ---------------------------------------------------- padded workspace ---
// Row length of the fused passes' six-field workspace: n/2 + 1 rounded up to
// a multiple of 16 complex values (272 at n = 512, 528 at n = 1024), so that
// every (x, y) row starts on a 128-byte line and a tile of 16 (or 8) k_z
// columns covers whole lines.  With rows of n/2 + 1 values each 128-byte row
// segment straddles two lines: measured on the access patterns alone, the
// inverse x pass's writes ran at 2.5 TB/s against 4.3 TB/s on lines, the y
// passes' at 5.2 against 6.4 TB/s.  The caller's spectra keep n/2 + 1.
__host__ __device__ constexpr long long ns_row(int n) { return ((long long)(n / 2 + 1) + 15) / 16 * 16; }

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
    k_ns_ypass(const float2* w, float2* wo, NSGeom g, int ktiles, const float2* __restrict__ tw) {  // wo may be w
  constexpr long long H1 = ns_row(N), MM = (long long)N * N * H1;  // the padded workspace
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
  const long long off = f * MM + (long long)x * N * H1 + kz;
  float2 v[G];
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const int pos = j + m * S;
    const bool rd = valid && (SIGN < 0 || kept_xy(pos, N, KD));
    v[m] = rd ? (SIGN < 0 ? wo[off + (long long)pos * H1] : __ldg(&w[off + (long long)pos * H1]))
              : make_float2(0.f, 0.f);
  }
  fft_line<N, G, SIGN>(v, j, ColX<T>{smn, c}, tw);
  if (valid) {
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int pos = j + m * S;
      if (SIGN > 0 || kept_xy(pos, N, KD)) wo[off + (long long)pos * H1] = v[m];
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
  static constexpr int MINB = THREADS <= 256 ? 2 : 1;
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
__global__ void __launch_bounds__(NICfg<N>::THREADS, NICfg<N>::MINB)
    k_ns_invx(const float2* __restrict__ u, float2* __restrict__ w, NSGeom g, int ktiles,
              const float2* __restrict__ tw) {
  constexpr long long H1 = N / 2 + 1, MM = (long long)N * N * H1;  // geometry of the n^3 grid
  constexpr long long HW = ns_row(N), MW = (long long)N * N * HW;  // the padded workspace
  constexpr int KD = (N - 1) / 3;                                  // largest kept |k| (2/3 rule)
  using C = NICfg<N>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smn[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int dky = blockIdx.x / ktiles;
  const int ay = dense_to_a(dky, N, KD);
  const int kz = (blockIdx.x - dky * ktiles) * T + c;
  const bool valid = kz < (KD + 1);
  const long long q = (long long)ay * H1 + kz;
  const long long rs = (long long)N * H1;
  const long long qw = (long long)ay * HW + kz, rw = (long long)N * HW;
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
      for (int m = 0; m < G; ++m) w[f * MW + (j + m * S) * rw + qw] = v[m];
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
// The z kernel holds a 256-point line (n = 512) as 16 values per thread on 16
// threads, two lines per warp: each transform is two radix-16 stages with one
// exchange through shared memory (8 values per thread would need three stages
// and two exchanges, and the exchanges dominated the L1 traffic).  A thread
// holds up to four such arrays (u x omega accumulators and a vorticity
// component), 230 registers at n = 512: two CTAs of 128 threads per SM.
// Measured and dropped: three CTAs per SM with one staging buffer (168
// registers, 1.120 against 1.126 ms), CTAs of 64 or 32 threads with five or
// ten per SM (spills; 1.20 ms), the velocity parked in TMEM (slower).
template <int N>
struct NZCfg {
  static constexpr int H = N / 2;
  static constexpr int G = H < 16 ? H : 16;
  static constexpr int S = H / G;
  static constexpr int LPC = S >= 128 ? 1 : 128 / S;
  static constexpr int NBUF = 2;                  // staging buffers per line
  static constexpr int THREADS = LPC * S;
  static constexpr bool WARP = S <= 32;
  static constexpr int KC = (N - 1) / 3 + 1;      // kept k_z count (2/3 rule)
  static constexpr int KCP = (KC + 2) & ~1;       // staged values per line and buffer (KC + alignment slack)
  static constexpr size_t FIELDS = sizeof(float2) * (size_t)LPC * H * 4;  // exchange + 3 parked fields
  static constexpr size_t STAGE = sizeof(float2) * (size_t)LPC * NBUF * KCP;  // staging buffers
  static constexpr size_t SMEM = FIELDS + STAGE + sizeof(uint64_t) * NBUF * LPC;  // + one mbarrier per buffer
  static constexpr int MINB = G == 16 ? 2 : 4;    // CTAs per SM the registers must allow
};

// 3. per (x, y) line: the six c2r transforms, the product n = u x omega and
//    the three r2c transforms.  Reads k_z < kc of fields 0..5 of w, writes
//    k_z < kc of fields 0..2 of wo (wo may be w: a line is fully read before
//    it is written).
//    The three velocity components are parked in real space in shared memory;
//    each vorticity component is then transformed and folded into the
//    accumulators of n, so at most 4 fields are held in registers.
//    A line's kept coefficients of each input field arrive by one bulk
//    asynchronous copy into one of two staging buffers, issued two fields
//    ahead of their use, so the global loads' latency overlaps the transforms
//    of the field before; the c2r reads X[k] and its mirror X[H - k] from there.
template <int N, int HW>  // HW: row length of the workspace (n/2 + 1, or the fused path's padded rows)
__global__ void __launch_bounds__(NZCfg<N>::THREADS, NZCfg<N>::MINB)
    k_ns_z(const float2* w, float2* wo, NSGeom g, const float2* __restrict__ tw, int* err) {
  constexpr long long H1 = HW, MM = (long long)N * N * H1;  // geometry of the workspace
  using C = NZCfg<N>;
  constexpr int H = C::H, G = C::G, S = C::S;
  constexpr int LOGN = Log2<N>::value;
  constexpr int KC = C::KC;  // kept k_z count
  extern __shared__ __align__(16) float2 smz[];
  const int li = threadIdx.x / S, j = threadIdx.x % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < (long long)N * N;
  const LineX<C::WARP> xc{smz + li * H};
  float2* park = smz + C::LPC * H + li * 3 * H + j;  // [3][G][S] per line, this thread's column
  constexpr int NB = C::NBUF;
  float2* stage = smz + C::FIELDS / sizeof(float2) + li * NB * C::KCP;  // this line's buffers
  uint64_t* bar = reinterpret_cast<uint64_t*>(smz + (C::FIELDS + C::STAGE) / sizeof(float2)) + NB * li;

  // Field f's element k of this line sits at element f MM + line H1 + k.  MM
  // is even; with H1 odd (rows of n/2 + 1) the line starts 16-byte aligned for
  // even lines and 8 bytes past a 16-byte boundary for odd ones: the copy then
  // starts `lead` elements early (the previous line's last value, k_z = n/2,
  // which this kernel never writes) and ends at k_z <= kc, inside the line.
  // With padded rows (H1 a multiple of 16) every line is aligned.
  const int lead = (int)((line * H1) & 1);
  const uint32_t bytes = (uint32_t)(sizeof(float2) * ((KC + lead + 1) & ~1));
  auto issue = [&](int f) {  // one thread of the line; buffer f % NB was last read NB fields ago
    uint64_t* b = bar + f % NB;
    tcg::fence_smem_async();
    tcg::mbar_expect(b, bytes);
    tcg::bulk_g2s(stage + (f % NB) * C::KCP, w + f * MM + line * H1 - lead, bytes, b);
  };
  bool ok = true;
  auto arrive = [&](int f) {  // wait for field f's copy (bounded; an expired wait is reported)
    if (!valid) return;
    const uint32_t par = (uint32_t)((f / NB) & 1);
    if (!tcg::mbar_wait(bar + f % NB, par)) {
      if (j == 0 && ok) atomicOr(err, 1);
      ok = false;
      tcg::mbar_wait(bar + f % NB, par);  // once more for the copy still in flight
    }
  };
  if (j == 0 && valid) {
    for (int b = 0; b < NB; ++b) tcg::mbar_init(bar + b);
    for (int b = 0; b < NB; ++b) issue(b);
  }
  xc.sync();  // the barriers are initialised before anyone polls them
  // exp(-2 pi i k / N) at k = j + m S is Wj exp(-2 pi i m / (2G)) (N = 2 G S):
  // one table load per thread instead of one per value
  // (measured against one table load per value at 16 values per thread:
  // 1.126 against 1.190 ms per launch at 512^3)
  const float2 Wj = __ldg(&tw[j]);
  auto twk = [&](int m) { return mul_root32(Wj, m * (16 / G)); };

  // inverse z transform of field f (half-complex -> N real points, two per slot)
  auto c2r = [&](int f, float2 (&U)[G]) {
    const float2* src = stage + (f % NB) * C::KCP + lead;
    arrive(f);
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
      if (k < KC) A = src[k];
      if (H - k < KC) B = src[H - k];
      if (k == 0) {
        A.y = 0.f;
        B.y = 0.f;
      }
      const float2 Bc = cconj(B);
      const float2 E = cadd(A, Bc);
      const float2 O = cmulc(csub(A, Bc), twk(m));
      U[m] = make_float2(E.x - O.y, E.y + O.x);
    }
    if constexpr (S == 1) xc.sync();  // (one thread per line: the transform has no exchange)
    fft_line<H, G, +1, LOGN>(U, j, xc, tw);
    // every thread of the line has passed an exchange barrier since it read
    // the buffer: refill it with field f + NB
    if (f + NB < 6 && j == 0 && valid) issue(f + NB);
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
    float2* dst = wo + f * MM + line * H1;
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 A = U[m];
      const float2 Bc = cconj(xc.ld((H - k) & (H - 1)));
      const float2 E = cscale(cadd(A, Bc), 0.5f);
      const float2 D = csub(A, Bc);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
      if (valid && k < KC) dst[k] = cadd(E, cmul(twk(m), O));
    }
    xc.sync();
  };
  // n = u x omega at the two real points held by each slot (elementwise
  // products of the (even, odd) point pairs, paired FP32 instructions):
  //   n_x = u_y w_z - u_z w_y,  n_y = u_z w_x - u_x w_z,  n_z = u_x w_y - u_y w_x
  // n_z is complete after omega_y and is transformed before omega_z is loaded.
  auto neg = [](float2 a) { return make_float2(-a.x, -a.y); };
  float2 Ny[G], Nx[G];
  {
    float2 Nz[G];
    {
      float2 W[G];
      c2r(3, W);  // omega_x
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const float2 uy = park[(1 * G + m) * S], uz = park[(2 * G + m) * S];
        Ny[m] = __fmul2_rn(uz, W[m]);
        Nz[m] = __fmul2_rn(neg(uy), W[m]);
      }
      c2r(4, W);  // omega_y
#pragma unroll
      for (int m = 0; m < G; ++m) {
        const float2 ux = park[(0 * G + m) * S], uz = park[(2 * G + m) * S];
        Nx[m] = __fmul2_rn(neg(uz), W[m]);
        Nz[m] = __ffma2_rn(ux, W[m], Nz[m]);
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
      Nx[m] = __ffma2_rn(uy, W[m], Nx[m]);
      Ny[m] = __ffma2_rn(neg(ux), W[m], Ny[m]);
    }
  }
  r2c(0, Nx);
  r2c(1, Ny);
}

// ----------------------------------------------------- x pass + update -----

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
  constexpr long long HW = ns_row(N), MW = (long long)N * N * HW;  // the padded workspace (nh)
  constexpr int KD = (N - 1) / 3;                                  // largest kept |k| (2/3 rule)
  using C = NUCfg<N>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ float2 smn[];
  const int c = threadIdx.x % T, j = threadIdx.x / T;
  const int dky = blockIdx.x / ktiles;
  const int ay = dense_to_a(dky, N, KD);
  const int kz = (blockIdx.x - dky * ktiles) * T + c;
  const bool valid = kz < (KD + 1);
  const long long q = (long long)ay * H1 + kz;
  const long long rs = (long long)N * H1;
  const long long qw = (long long)ay * HW + kz, rw = (long long)N * HW;
  const ColX<T> xc{smn, c};
  // fields 0 and 1 are parked in shared memory after their transforms (this
  // thread's slots only), so one field at a time is held in registers
  float2* park = smn + (size_t)N * T + threadIdx.x;
  float2 V[G];
#pragma unroll 1
  for (int f = 0; f < 3; ++f) {
#pragma unroll
    for (int m = 0; m < G; ++m)
      V[m] = valid ? nh[f * MW + (j + m * S) * rw + qw] : make_float2(0.f, 0.f);
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


int ns_kmax(int n) { return (int)std::floor(std::sqrt(3.0) * (n / 2) + 0.5) + 1; }

NSGeom make_geom(int n) {
  NSGeom g;
  g.n = n;
  g.h1 = n / 2 + 1;
  g.kd = (n - 1) / 3;
  g.kc = g.kd + 1;
  g.nk = 2 * g.kd + 1;
  g.M = (long long)n * n * g.h1;
  return g;
}

fftk_status ns_ensure(fftk_plan p) {
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->ns) return FFTK_OK;
  NSWork* s = new (std::nothrow) NSWork;
  if (!s) return FFTK_ERR_OOM;
  s->g = make_geom(p->nx);
  s->kmax = ns_kmax(p->nx);
  s->etab_len = 3 * s->g.kd * s->g.kd + 1;
  const size_t fb = sizeof(float2) * (size_t)s->g.M;
  const size_t fw = sizeof(float2) * (size_t)p->nx * p->nx * (size_t)ns_row(p->nx);  // padded rows (fused path)
  const int width = 2 + s->kmax + 1;
  cudaError_t e = cudaMalloc(&s->w, 6 * (fw > fb ? fw : fb));
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

// The fused passes' second six-field workspace (padded rows), on first use.
static cudaError_t ns_second_workspace(fftk_plan p) {
  NSWork* s = p->ns;
  std::lock_guard<std::mutex> lk(p->mu);
  if (s->w2) return cudaSuccess;
  const size_t fw = sizeof(float2) * (size_t)p->nx * p->nx * (size_t)ns_row(p->nx);
  cudaError_t e = cudaMalloc(&s->w2, 6 * fw);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->w2 = nullptr;
  }
  return e;
}

// --------------------------------------------------------------- launchers --
template <int N>
struct NSLaunch {
  static cudaError_t attrs() {
    static PerDevice once;
    return once.run([](int) {
      const int sx = (int)NXCfg<N>::SMEM;
      cudaError_t err = cudaFuncSetAttribute(k_ns_invx<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)NICfg<N>::SMEM);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_ypass<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_ypass<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_fwdx<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)NUCfg<N>::SMEM);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_z<N, (int)ns_row(N)>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)NZCfg<N>::SMEM);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_ns_z<N, N / 2 + 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)NZCfg<N>::SMEM);
      return err;
    });
  }

  // The fused z pass alone (c2r of the six fields in s->w, u x omega, r2c of
  // n into fields 0..2), for the split-precision right-hand side.
  static cudaError_t z(fftk_plan p, cudaStream_t st) {
    using Z = NZCfg<N>;
    cudaError_t e = attrs();
    if (e != cudaSuccess) return e;
    NSWork* s = p->ns;
    LaunchScope ls(p, KK_NS_Z, st);
    const long long lines = (long long)N * N;
    k_ns_z<N, N / 2 + 1><<<(unsigned)((lines + Z::LPC - 1) / Z::LPC), Z::THREADS, Z::SMEM, st>>>(
        s->w, s->w, s->g, twiddles(p, N), p->d_err);
    return cudaGetLastError();
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
    // invx u -> A, inverse y A -> B, z B -> A (fields 0..2), forward y A -> A,
    // forward x A -> out.  The inverse y pass out of place measured 0.684 ->
    // 0.647 ms at 512^3; the forward y pass, which writes only the kept rows,
    // measured slower out of place (0.313 -> 0.331 ms), so it stays in place.
    e = ns_second_workspace(p);
    if (e != cudaSuccess) return e;
    float2* A = s->w;
    float2* Bw = s->w2;
    {
      LaunchScope ls(p, KK_NS_INVX, st);
      k_ns_invx<N><<<g.nk * ki, I::THREADS, I::SMEM, st>>>(u, A, g, ki, twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_INVY, st);
      k_ns_ypass<N, 1><<<6 * N * kx, X::THREADS, X::SMEM, st>>>(A, Bw, g, kx, twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_Z, st);
      const long long lines = (long long)N * N;
      k_ns_z<N, (int)ns_row(N)><<<(unsigned)((lines + Z::LPC - 1) / Z::LPC), Z::THREADS, Z::SMEM, st>>>(
          Bw, A, g, twiddles(p, N), p->d_err);
    }
    {
      LaunchScope ls(p, KK_NS_FWDY, st);
      k_ns_ypass<N, -1><<<3 * N * kx, X::THREADS, X::SMEM, st>>>(A, A, g, kx, twiddles(p, N));
    }
    {
      LaunchScope ls(p, KK_NS_FWDX, st);
      k_ns_fwdx<N><<<g.nk * ku, U::THREADS, U::SMEM, st>>>(A, u0, u1, out, g, ku, upd, mode,
                                                          extra, twiddles(p, N));
    }
    return cudaGetLastError();
  }
};

// ---------------------------------------------- split-precision NS step ----
// Plans of dtype FFTK_R32_SPLIT16 evaluate the right-hand side with the x and
// y passes on the tensor cores (split FP16 radix-16 stages, restricted to the
// 2/3-rule set): u and omega = i k x u on the kept modes, inverse x and y
// passes of the six fields, the fused FP32 z pass (u x omega in registers),
// forward y and x passes of n, and the per-mode update of the fused path.

// w6 = (u, i k x u) on the kept modes; the derivative of the Nyquist wavenumber is 0
__global__ void k_curl_full(const float2* __restrict__ u, float2* __restrict__ w6, NSGeom g) {
  const long long items = (long long)g.nk * g.nk * g.kc;  // k_z fastest
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % g.kc);
    const long long ab = it / g.kc;
    const int a = dense_to_a((int)(ab / g.nk), g.n, g.kd), b = dense_to_a((int)(ab % g.nk), g.n, g.kd);
    const long long idx = ((long long)a * g.n + b) * g.h1 + c;
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

// the update of every kept mode from n_hat (already scaled by the transform)
__global__ void k_update_full(const float2* __restrict__ nh, const float2* u0, const float2* u1, float2* out,
                              NSGeom g, NSUpdate upd, int mode, const float2* __restrict__ extra) {
  float gforce = 0.f;
  if (upd.feps > 0.0) {
    const double ef = *upd.ef;
    gforce = ef > 0.0 ? (float)(upd.feps / (2.0 * ef)) : 0.f;
  }
  const long long items = (long long)g.nk * g.nk * g.kc;  // the kept modes, k_z fastest
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % g.kc);
    const long long ab = it / g.kc;
    const int a = dense_to_a((int)(ab / g.nk), g.n, g.kd), b = dense_to_a((int)(ab % g.nk), g.n, g.kd);
    const long long idx = ((long long)a * g.n + b) * g.h1 + c;
    ns_mode_update(nh[idx], nh[idx + g.M], nh[idx + 2 * g.M], kwav(a, g.n), kwav(b, g.n), c, idx, g.M, upd, mode,
                   gforce, u0, u1, extra, out);
  }
}

static cudaError_t ns_z_dispatch(fftk_plan p, cudaStream_t st);

static cudaError_t ns_rhs_split(fftk_plan p, const float2* u, const float2* u0, const float2* u1, float2* out,
                                const NSUpdate& upd, int mode, const float2* extra, cudaStream_t st) {
  NSWork* s = p->ns;
  const NSGeom g = s->g;
  const unsigned grid = 152 * 8;
  const bool tc = cpass_tc_supported(g.n) && g.n <= 1024;
  const float scale = (float)(1.0 / ((double)g.n * g.n * g.n));
  {
    LaunchScope ls(p, KK_AUX, st);
    k_curl_full<<<grid, 256, 0, st>>>(u, s->w, g);
  }
  cudaError_t e = tc ? launch_cpass_tc_pruned(p, 0, +1, s->w, s->w, 6, 1.f, KK_X_INV, st)
                     : launch_pruned_x(p, +1, s->w, s->w, 6, 1.f, st);
  if (e == cudaSuccess)
    e = tc ? launch_cpass_tc_pruned(p, 1, +1, s->w, s->w, 6, 1.f, KK_Y_INV, st)
           : launch_pruned_y(p, +1, s->w, s->w, 6, 1.f, st);
  if (e == cudaSuccess) e = ns_z_dispatch(p, st);
  if (e == cudaSuccess)
    e = tc ? launch_cpass_tc_pruned(p, 1, -1, s->w, s->w, 3, 1.f, KK_Y_FWD, st)
           : launch_pruned_y(p, -1, s->w, s->w, 3, 1.f, st);
  if (e == cudaSuccess)
    e = tc ? launch_cpass_tc_pruned(p, 0, -1, s->w, s->w, 3, scale, KK_X_FWD, st)
           : launch_pruned_x(p, -1, s->w, s->w, 3, scale, st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_update_full<<<grid, 256, 0, st>>>(s->w, u0, u1, out, g, upd, mode, extra);
  }
  return cudaGetLastError();
}

// ------------------------------------------- right-hand side on 3 * 2^m -----
// Grids of 3 * 2^m points (the paper's XC40 runs use 768^3, 1536^3 and 3072^3)
// have no fused passes: the right-hand side runs through the plan's
// transforms, whose 1D passes take one radix-3 step over power-of-two
// sub-lines, with u x omega formed pointwise in real space:
//   (u, omega = i k x u) on the kept modes -> c2r of the six fields ->
//   n = u x omega -> r2c of n -> the per-mode update of the fused path
//   (2/3 rule, projection, forcing, integrating-factor stage).

// r: six real fields u_x, u_y, u_z, omega_x, omega_y, omega_z (R points each);
// n = u x omega overwrites fields 0..2 (each point is read before it is written)
__global__ void k_cross(float* __restrict__ r, long long R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += (long long)gridDim.x * blockDim.x) {
    const float ux = r[i], uy = r[i + R], uz = r[i + 2 * R];
    const float wx = r[i + 3 * R], wy = r[i + 4 * R], wz = r[i + 5 * R];
    r[i] = fmaf(uy, wz, -uz * wy);
    r[i + R] = fmaf(uz, wx, -ux * wz);
    r[i + 2 * R] = fmaf(ux, wy, -uy * wx);
  }
}

static cudaError_t ns_rhs_unfused(fftk_plan p, const float2* u, const float2* u0, const float2* u1, float2* out,
                                  const NSUpdate& upd, int mode, const float2* extra, cudaStream_t st) {
  NSWork* s = p->ns;
  const NSGeom g = s->g;
  const long long R = (long long)g.n * g.n * g.n;
  if (!s->r6) {
    cudaError_t ea = cudaMalloc(&s->r6, sizeof(float) * 6 * (size_t)R);
    if (ea != cudaSuccess) {
      cudaGetLastError();
      s->r6 = nullptr;
      return ea;
    }
  }
  const unsigned grid = 152 * 8;
  cudaError_t e = cudaMemsetAsync(s->w, 0, sizeof(float2) * 6 * (size_t)g.M, st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_curl_full<<<grid, 256, 0, st>>>(u, s->w, g);
  }
  // the second six-field workspace holds the strided passes' intermediate
  // spectra (they run out of place)
  e = ns_second_workspace(p);
  if (e != cudaSuccess) return e;
  e = c2r_overwrite(p, s->w, s->r6, 6, st, s->w2);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_cross<<<grid, 256, 0, st>>>(s->r6, R);
  }
  e = r2c_scaled(p, s->r6, s->w, 3, (float)(1.0 / ((double)g.n * g.n * g.n)), st, s->w2);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_update_full<<<grid, 256, 0, st>>>(s->w, u0, u1, out, g, upd, mode, extra);
  }
  return cudaGetLastError();
}

#define NS_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

static cudaError_t ns_z_dispatch(fftk_plan p, cudaStream_t st) {
  switch (p->nx) {
#define CASE(n) \
  case n:       \
    return NSLaunch<n>::z(p, st);
    NS_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

static cudaError_t ns_rhs_dispatch(fftk_plan p, const float2* u, const float2* u0, const float2* u1,
                                   float2* out, const NSUpdate& upd, int mode, const float2* extra,
                                   cudaStream_t st) {
  if (!is_pow2(p->nx)) return ns_rhs_unfused(p, u, u0, u1, out, upd, mode, extra, st);
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

fftk_status ns_check(fftk_plan p, const tarang_params* prm, bool need_dt) {
  if (!p || !prm) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (!ns_size_ok(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (!(prm->nu >= 0.0) || !std::isfinite(prm->nu)) return FFTK_ERR_INVALID_ARG;
  if (need_dt && (!(prm->dt > 0.0) || !std::isfinite(prm->dt))) return FFTK_ERR_INVALID_ARG;
  if (prm->sgs_model && !prm->sgs_model->params) return FFTK_ERR_INVALID_ARG;
  if (prm->sgs_model && !is_pow2(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;  // the learned closure: 2^m grids
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
  cudaFree(s->w2);
  cudaFree(s->u1);
  cudaFree(s->etab);
  cudaFree(s->ef);
  cudaFree(s->part);
  cudaFree(s->dout);
  if (s->hout) cudaFreeHost(s->hout);
  cudaFree(s->r6);
  cudaFree(s->r3);
  cudaFree(s->acc);
  rbc_free(s->rbc);
  cudaFree(s->sout);
  sgs_free(s->sgs);
  delete s;
  p->ns = nullptr;
}


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
  if (p->nx != p->ny || p->nx != p->nz || !ns_size_ok(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
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
  if (p->nx != p->ny || p->nx != p->nz || !ns_size_ok(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  fftk_status s = ns_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  {
    LaunchScope ls(p, KK_AUX, st);
    k_ic_shape<<<152 * 8, 256, 0, st>>>(static_cast<float2*>(uhat), p->ns->g);
  }
  return from_cuda(cudaGetLastError());
}
