// Split-FP16 tensor-core radix-16 stages for the strided passes (dtype
// FFTK_R32_SPLIT16).
//
// A line of length L = R0 * 256 (R0 in {1, 2, 4, 8}) is transformed as one
// FP32 radix-R0 stage in registers followed by two radix-16 stages on the
// 5th-generation tensor cores.  A radix-16 stage over a batch of DFT rows is
// the product D = A B:
//   A [rows x 64] FP16: for each of the row's 16 complex inputs x (already
//     twiddled, scaled by a power of two), the four values hi.re, hi.im,
//     lo.re, lo.im with hi = fp16(x), lo = fp16(x - hi);
//   B = B1 + B2 [64 x 32] FP16: the real form of W16 = exp(SIGN 2 pi i r k/16)
//     split W = W_hi + W_lo; B1 multiplies both hi and lo by W_hi, B2 the hi
//     part by W_lo, so D = (x_hi + x_lo) W_hi + x_hi W_lo (FP32 accumulate in
//     TMEM), dropping only x_lo W_lo (2^-22 relative).
// Twiddles, scaling and the radix-R0 stage stay in FP32.  Per stage, one
// thread writes its A values to shared memory and, after the MMAs, reads one
// TMEM row back with tcgen05.ld; the second stage's rows go straight to global
// memory, so no FP32 exchange through shared memory remains.  Thread 0 issues
// tcgen05.mma (M = 128, N = 32, K = 16) and completion is signalled through an
// mbarrier.  Operands use the canonical K-major layout without swizzle: 8-row
// x 16-byte core matrices, 128 bytes apart along K (LBO) and 1024 bytes apart
// along M/N (SBO).
#include <cuda_fp16.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "fft_engine.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace fftk {
namespace tc {

constexpr uint32_t kLBO = 128;           // bytes between core matrices along K
constexpr uint32_t kSBO = 1024;          // bytes between 8-row groups (64 FP16 per row)
constexpr int kBlkBytes = 16 * 1024;     // one M block of A
constexpr int kBlkStride = kBlkBytes + 16;  // + 16 bytes: spreads blocks over banks
constexpr int kBBytes = 4 * 1024;        // one 32 x 64 operand

using tcg::su32;
using tcg::ld32;
using tcg::mbar_wait;

__device__ __forceinline__ uint64_t desc(uint32_t addr) { return tcg::desc(addr, kLBO, kSBO); }

// byte offset of element (row, k) inside the A tile
__device__ __forceinline__ int a_off(int row, int k) {
  const int r = row & 127;
  return (row >> 7) * kBlkStride + (r >> 3) * (int)kSBO + (k >> 3) * (int)kLBO + (r & 7) * 16 + (k & 7) * 2;
}

// D = F32, A = B = F16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = tcg::idesc_f16(128, 32, false);

__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc) {
  tcg::mma_f16(dtm, ad, bd, kIdesc, acc);
}

// hi/lo split of one complex value, packed (hi.re, hi.im, lo.re, lo.im)
__device__ __forceinline__ uint2 split2(float2 a) {
  const __half2 hi = __floats2half2_rn(a.x, a.y);
  const float2 hf = __half22float2(hi);
  const __half2 lo = __floats2half2_rn(a.x - hf.x, a.y - hf.y);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&hi), *reinterpret_cast<const uint32_t*>(&lo));
}

// power of two that brings max |v| to [2^10, 2^11), at most 2^100 (columns
// whose largest value is below 2^-89, e.g. far dissipation-range modes, keep
// a finite scale and a finite inverse; their operands then sit among FP16's
// subnormals, an absolute error far below the rest of the column)
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f)) return 1.f;
  int e;
  frexpf(m, &e);
  return ldexpf(1.f, 11 - e < 100 ? 11 - e : 100);
}

}  // namespace tc

// Tile = T adjacent columns (contiguous index q) x the whole line.  The line
// L = R0 * 16 * 16 is transformed as
//   stage 0 (FP32, registers): for each a < 256 the R0-point DFT of
//     x[a + 256 m], m < R0, times the twiddle W_L^(a r)  -> Z_r[a];
//   stage 1 (tensor cores): for each (r, a0 < 16) the DFT-16 over a1 of
//     Z_r[a0 + 16 a1]  -> U[k0'], times W_256^(a0 k0');
//   stage 2 (tensor cores): for each (r, k0') the DFT-16 over a0
//     -> X[R0 (k0' + 16 k1') + r]  (stored straight from TMEM).
// One stage row per thread: T * L / 16 = 1024 threads (T = 16384 / L columns:
// 64 at L = 256 down to 8 at L = 2048, the widest row segments one CTA can
// hold; 8-column tiles at L = 1024 and two CTAs per SM measured 0.64 of the
// FP32 pair rate, 16 columns and one CTA 0.74), 128-row M blocks, one TMEM
// lane per thread.  Every value handed to the tensor cores is scaled by the
// same power of two per column: s brings the column's largest stage-0 output
// component into [2^10, 2^11); stage-1 outputs are bounded by 16 times that,
// so stage 2 takes them times 1/16 (folded into its twiddles).
// The CTA is persistent (one TMEM allocation for all its tiles).
template <int L>
struct TC2 {
  static constexpr int T = 16384 / L;  // columns per tile: the widest a 1024-thread CTA holds
  static constexpr int R0 = L / 256;                   // leading FP32 radix
  static constexpr int A1 = 16 / R0;                   // stage-0 butterflies per thread
  static constexpr int THREADS = T * L / 16;           // DFT-16 rows per stage
  static constexpr int BLOCKS = THREADS / 128;         // M = 128 blocks
  static constexpr int COLS = BLOCKS * 32;             // TMEM columns (a power of two >= 32)
  static constexpr int LOGT = Log2<T>::value;
  static constexpr int LOGL = Log2<L>::value;
  static constexpr int ABYTES = BLOCKS * tc::kBlkStride;
  static constexpr size_t SMEM =
      1024 + ABYTES + 2 * tc::kBBytes + (256 + L) * sizeof(float2) + sizeof(float) * T + 64;
  static constexpr int MINB = 1024 / THREADS;  // 64 registers
  static_assert(THREADS % 128 == 0 && (COLS & (COLS - 1)) == 0 && SMEM <= 227 * 1024, "tile shape");
};

// Physical stage row of logical row (jj, cc) (jj = 16 r + a0 in stage 1,
// 16 r + k0' in stage 2; cc the column).  Thread t owns physical row t.  For
// T = 16 bits 3 and 4 are swapped so that a half warp's 64-bit operand stores
// cover 8 rows x 2 K slots (no bank conflicts).
template <int T>
__device__ __forceinline__ int phys_row(int jj, int cc) {
  if constexpr (T == 16) {
    return (cc & 7) | ((jj & 1) << 3) | (((cc >> 3) & 1) << 4) | ((jj >> 1) << 5);
  } else {
    return (jj << Log2<T>::value) | cc;
  }
}
template <int T>
__device__ __forceinline__ void thread_coords(int t, int& cc, int& jj) {
  if constexpr (T == 16) {
    cc = (t & 7) | (((t >> 4) & 1) << 3);
    jj = ((t >> 3) & 1) | ((t >> 5) << 1);
  } else {
    cc = t & (T - 1);
    jj = t >> Log2<T>::value;
  }
}


// B operands (K-major, 32 rows of 64) for one sign: [B1 | B2] in the
// canonical layout, built on the host in FP64 and rounded to FP16.
static void build_dft16_operands(int sign, std::vector<__half>& out) {
  out.assign(2 * 32 * 64, __float2half(0.f));
  auto off = [](int n, int k) {  // in halves
    return ((n >> 3) * 1024 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
  };
  const double two_pi = 6.283185307179586476925286766559;
  for (int r = 0; r < 16; ++r)
    for (int k = 0; k < 16; ++k) {
      const int m = (r * k) % 16;
      const double wr = std::cos(two_pi * m / 16.0), wi = sign * std::sin(two_pi * m / 16.0);
      const __half wr_hi = __float2half((float)wr), wi_hi = __float2half((float)wi);
      const __half wr_lo = __float2half((float)(wr - (double)__half2float(wr_hi)));
      const __half wi_lo = __float2half((float)(wi - (double)__half2float(wi_hi)));
      const __half nwi_hi = __float2half(-__half2float(wi_hi)), nwi_lo = __float2half(-__half2float(wi_lo));
      // output re (column 2k) and im (column 2k+1); inputs hi.re, hi.im, lo.re, lo.im (rows 4r..4r+3)
      __half* B1 = out.data();
      __half* B2 = out.data() + 32 * 64;
      B1[off(2 * k, 4 * r + 0)] = wr_hi;
      B1[off(2 * k, 4 * r + 1)] = nwi_hi;
      B1[off(2 * k, 4 * r + 2)] = wr_hi;
      B1[off(2 * k, 4 * r + 3)] = nwi_hi;
      B1[off(2 * k + 1, 4 * r + 0)] = wi_hi;
      B1[off(2 * k + 1, 4 * r + 1)] = wr_hi;
      B1[off(2 * k + 1, 4 * r + 2)] = wi_hi;
      B1[off(2 * k + 1, 4 * r + 3)] = wr_hi;
      B2[off(2 * k, 4 * r + 0)] = wr_lo;
      B2[off(2 * k, 4 * r + 1)] = nwi_lo;
      B2[off(2 * k + 1, 4 * r + 0)] = wi_lo;
      B2[off(2 * k + 1, 4 * r + 1)] = wr_lo;
    }
}


// Strided pass [P][L][Q] along L with split-FP16 tensor-core radix-16 stages.
// PM = 0: every column q < Q.  PM = 1, 2: the pass of an L^3 spectrum
// restricted to its 2/3-rule set, as the FP32 k_pcpass: x lines (rows of
// stride L (L/2+1)) over the kept (k_y, k_z) columns (PM = 1), or y lines
// (stride L/2+1) over the kept k_z columns of every x (PM = 2); the inverse
// reads only kept rows, the forward writes only kept rows.  `outer` is the
// number of k_y (PM = 1) or x (PM = 2) indices per batch element.
template <int L, int SIGN, int PM>
__global__ void __launch_bounds__(TC2<L>::THREADS, TC2<L>::MINB)
    k_cpass_tc(const float2* in, float2* out, long long Q, long long qtiles, long long ntiles, int outer,
               const float2* __restrict__ tw, float out_scale,  // tw: size-L table
               const __half* __restrict__ bops, int* err) {
  using C = TC2<L>;
  constexpr int T = C::T, R0 = C::R0, A1 = C::A1, NT = C::THREADS;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = smraw + ((1024 - (tc::su32(smraw) & 1023)) & 1023);
  unsigned char* As = base;                                          // A tile (both stages)
  unsigned char* Bs = base + C::ABYTES;                              // B1, B2
  float2* w256 = reinterpret_cast<float2*>(Bs + 2 * tc::kBBytes);   // W_256^m / 16
  float2* wL = w256 + 256;                                            // W_L^m (conjugated for SIGN > 0)
  float* colmax = reinterpret_cast<float*>(wL + L);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(colmax + T);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5;

  // thread coordinates: column c; j splits into a0 (stage-0 a mod 16, stage-1
  // row a0, stage-2 row k0') and u (stage-0 block of a1, stage row r)
  int c, j;
  thread_coords<T>(t, c, j);
  const int a0 = j & 15, u = j >> 4;

  for (int i = t; i < 2 * tc::kBBytes / 16; i += NT)
    reinterpret_cast<uint4*>(Bs)[i] = reinterpret_cast<const uint4*>(bops)[i];
  for (int i = t; i < 256; i += NT) {
    float2 w = __ldg(&tw[i * (L / 256)]);
    if (SIGN > 0) w.y = -w.y;
    w256[i] = make_float2(w.x * 0.0625f, w.y * 0.0625f);
  }
  for (int i = t; i < L; i += NT) {
    float2 w = __ldg(&tw[i]);
    if (SIGN > 0) w.y = -w.y;
    wL[i] = w;
  }
  if (t < T) colmax[t] = 0.f;
  if (warp == 0) tcg::tmem_alloc(tslot, C::COLS);
  if (t == 0) tcg::mbar_init(mbar);
  tcg::fence_smem_async();
  tcg::fence_before_sync();
  __syncthreads();
  tcg::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t a_sa = tc::su32(As), b1_sa = tc::su32(Bs), b2_sa = b1_sa + tc::kBBytes;
  // this thread's TMEM row: lane 32 (warp % 4) + lane id of M block warp / 4 = stage row t
  const uint32_t row_addr = tmem + (((uint32_t)(warp & 3) * 32u) << 16) + 32u * (uint32_t)(warp >> 2);
  uint32_t phase = 0;
  bool failed = false;

  auto run_mma = [&]() -> bool {
    tcg::fence_smem_async();
    tcg::fence_before_sync();
    __syncthreads();
    tcg::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int blk = 0; blk < C::BLOCKS; ++blk) {
        const uint32_t d = tmem + 32u * blk;
        const uint32_t a = a_sa + blk * tc::kBlkStride;
#pragma unroll
        for (int s = 0; s < 4; ++s) tc::mma(d, tc::desc(a + 256 * s), tc::desc(b1_sa + 256 * s), s > 0);
#pragma unroll
        for (int s = 0; s < 4; ++s) tc::mma(d, tc::desc(a + 256 * s), tc::desc(b2_sa + 256 * s), 1);
      }
      tcg::commit(mbar);
    }
    // thread 0 alone polls the mbarrier; the others wait at the barrier
    // without taking issue slots, and the tcgen05 fences around it order their
    // TMEM reads after the MMAs
    bool ok = true;
    if (t == 0) {
      ok = tc::mbar_wait(mbar, phase);
      tcg::fence_after_sync();
      tcg::fence_before_sync();
    }
    phase ^= 1;
    const bool all = __syncthreads_and(ok) != 0;
    tcg::fence_after_sync();
    return all;
  };

  constexpr int KD = (L - 1) / 3;  // the 2/3 rule (PM > 0)
  auto kept = [](int row) { return row <= KD || row >= L - KD; };
  for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    long long col0, rs;
    bool valid;
    if constexpr (PM == 0) {
      const long long pl = tile / qtiles;
      const long long q0 = (tile - pl * qtiles) * T;
      valid = q0 + c < Q;
      col0 = pl * (long long)L * Q + q0 + c;
      rs = Q;
    } else {
      constexpr long long H1 = L / 2 + 1, MM = (long long)L * L * H1;
      const long long bo = tile / qtiles;
      const int kz = (int)(tile - bo * qtiles) * T + c;
      const long long b = bo / outer;
      const int o = (int)(bo - b * outer);
      valid = kz < KD + 1;
      if constexpr (PM == 1) {
        const int ay = o <= KD ? o : L - (2 * KD + 1 - o);
        col0 = b * MM + (long long)ay * H1 + kz;
        rs = (long long)L * H1;
      } else {
        col0 = b * MM + (long long)o * L * H1 + kz;
        rs = H1;
      }
    }
    float2* dst = out + col0;
    // ---- stage 0: R0-point DFTs of x[a + 256 m] for a = a0 + 16 (A1 u + i)
    float2 z[A1][R0];
    {
      const float2* src = in + col0;
#pragma unroll
      for (int i = 0; i < A1; ++i) {
        const int a = a0 + 16 * (A1 * u + i);
#pragma unroll
        for (int m = 0; m < R0; ++m) {
          const bool rd = valid && (PM == 0 || SIGN < 0 || kept(a + 256 * m));
          z[i][m] = rd ? src[(long long)(a + 256 * m) * rs] : make_float2(0.f, 0.f);
        }
      }
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < A1; ++i) {
      if constexpr (R0 > 1) {
        const int a = a0 + 16 * (A1 * u + i);
        dftR<R0, SIGN>(z[i]);
#pragma unroll
        for (int r = 1; r < R0; ++r) z[i][r] = cmul(z[i][r], wL[a * r]);
      }
#pragma unroll
      for (int r = 0; r < R0; ++r) mx = fmaxf(mx, fmaxf(fabsf(z[i][r].x), fabsf(z[i][r].y)));
    }
    // column maximum: lanes of a warp that share the column
    if constexpr (T == 16) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
    } else {
#pragma unroll
      for (int o = T; o < 32; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if constexpr (T == 16) {
      if (((t >> 3) & 1) == 0) atomicMax(reinterpret_cast<int*>(&colmax[c]), __float_as_int(mx));
    } else {
      if ((t & 31) < T) atomicMax(reinterpret_cast<int*>(&colmax[c]), __float_as_int(mx));
    }
    __syncthreads();
    const float s = tc::pow2_scale(colmax[c]);
    // stage-1 rows (r, a0, c); this thread fills K slots a1 = A1 u .. A1 u + A1 - 1
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int row = phys_row<T>(r * 16 + a0, c);
#pragma unroll
      for (int i = 0; i < A1; i += 2) {
        const uint2 v0 = tc::split2(cscale(z[i][r], s)), v1 = tc::split2(cscale(z[i + 1][r], s));
        *reinterpret_cast<uint4*>(As + tc::a_off(row, 4 * (A1 * u + i))) = make_uint4(v0.x, v0.y, v1.x, v1.y);
      }
    }
    if (!run_mma()) {
      failed = true;
      break;
    }
    if (t < T) colmax[t] = 0.f;  // every thread has read it (before the barrier in run_mma)

    // ---- stage 1 -> 2: row t = (r = u, a0, c) holds U[k0'] (times s); it
    //      feeds K slot a0 of stage-2 row (u, k0', c), twiddled by W_256^(a0 k0') / 16
    {
      float d[32];
      tc::ld32(row_addr, d);
#pragma unroll
      for (int k0 = 0; k0 < 16; ++k0) {
        const float2 y = cmul(make_float2(d[2 * k0], d[2 * k0 + 1]), w256[a0 * k0]);
        *reinterpret_cast<uint2*>(As + tc::a_off(phys_row<T>(u * 16 + k0, c), 4 * a0)) = tc::split2(y);
      }
    }
    if (!run_mma()) {
      failed = true;
      break;
    }
    // ---- stage 2 output: row t = (r = u, k0' = a0, c) holds X[R0 (k0' + 16 k1') + r] (times s / 16)
    {
      const float f = out_scale * 16.f / s;
      float d[32];
      tc::ld32(row_addr, d);
      if (valid) {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
          const int row = R0 * (a0 + 16 * k1) + u;
          if (PM == 0 || SIGN > 0 || kept(row))
            dst[(long long)row * rs] = make_float2(d[2 * k1] * f, d[2 * k1 + 1] * f);
        }
      }
    }
  }
  if (failed && t == 0) atomicOr(err, 1);
  if (failed && t == 0) tc::mbar_wait(mbar, phase ^ 1);  // let in-flight MMAs drain (bounded) before freeing TMEM
  tcg::fence_before_sync();
  __syncthreads();
  if (warp == 0) tcg::tmem_dealloc(tmem, C::COLS);
}

// P: batch (PM = 0: P lines of Q columns; PM > 0: P spectra of L^3)
template <int L, int SIGN, int PM>
static cudaError_t cpass_tc_l(fftk_plan p, const float2* in, float2* out, long long P, long long Q,
                              float scale, int kind, cudaStream_t st) {
  using C = TC2<L>;
  static PerDevice once;
  static int per_sm_dev[kMaxDevices];
  int dev = 0;
  const cudaError_t attr_err = once.run(
      [](int d) {
        const cudaError_t e = cudaFuncSetAttribute(k_cpass_tc<L, SIGN, PM>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        int n = 1;
        if (e == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cpass_tc<L, SIGN, PM>, C::THREADS, C::SMEM) !=
                cudaSuccess) {
          cudaGetLastError();
          n = 1;
        }
        if (n > 512 / C::COLS) n = 512 / C::COLS;  // TMEM: 512 columns per SM
        per_sm_dev[d] = n < 1 ? 1 : n;
        return e;
      },
      &dev);
  if (attr_err != cudaSuccess) return attr_err;
  const int per_sm = per_sm_dev[dev];
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  constexpr int KD = (L - 1) / 3;
  const int outer = PM == 1 ? 2 * KD + 1 : L;
  const long long qtiles = PM == 0 ? (Q + C::T - 1) / C::T : (KD + 1 + C::T - 1) / C::T;
  const long long ntiles = PM == 0 ? P * qtiles : P * outer * qtiles;
  const long long cap = (long long)per_sm * sms;
  const int blocks = (int)(ntiles < cap ? ntiles : cap);
  const __half* bops = p->d_dft16 + (SIGN < 0 ? 0 : 2 * 32 * 64);
  LaunchScope ls(p, kind, st);
  k_cpass_tc<L, SIGN, PM><<<blocks, C::THREADS, C::SMEM, st>>>(in, out, Q, qtiles, ntiles, outer, twiddles(p, L),
                                                             scale, bops, p->d_err);
  return cudaGetLastError();
}

bool cpass_tc_supported(int L) { return L == 256 || L == 512 || L == 1024 || L == 2048; }

cudaError_t launch_cpass_tc(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P,
                            long long Q, float scale, int kind, cudaStream_t st) {
  if (P <= 0 || Q <= 0) return cudaSuccess;
#define TC_CASE(n)                                                              \
  case n:                                                                       \
    return sign < 0 ? cpass_tc_l<n, -1, 0>(p, in, out, P, Q, scale, kind, st)   \
                    : cpass_tc_l<n, +1, 0>(p, in, out, P, Q, scale, kind, st);
  switch (L) {
    TC_CASE(256)
    TC_CASE(512)
    TC_CASE(1024)
    TC_CASE(2048)
  }
#undef TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_cpass_tc_pruned(fftk_plan p, int axis, int sign, const float2* in, float2* out, long long B,
                                   float scale, int kind, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
#define TC_CASE(n)                                                                                   \
  case n:                                                                                            \
    if (axis == 0)                                                                                   \
      return sign < 0 ? cpass_tc_l<n, -1, 1>(p, in, out, B, 0, scale, kind, st)                      \
                      : cpass_tc_l<n, +1, 1>(p, in, out, B, 0, scale, kind, st);                     \
    return sign < 0 ? cpass_tc_l<n, -1, 2>(p, in, out, B, 0, scale, kind, st)                        \
                    : cpass_tc_l<n, +1, 2>(p, in, out, B, 0, scale, kind, st);
  switch (axis == 0 ? p->nx : p->ny) {
    TC_CASE(256)
    TC_CASE(512)
    TC_CASE(1024)
  }
#undef TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t upload_dft16_operands(fftk_plan p) {
  std::vector<__half> fwd, inv;
  build_dft16_operands(-1, fwd);
  build_dft16_operands(+1, inv);
  const size_t n = fwd.size();
  cudaError_t e = cudaMalloc(&p->d_dft16, sizeof(__half) * 2 * n);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_dft16, fwd.data(), sizeof(__half) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_dft16 + n, inv.data(), sizeof(__half) * n, cudaMemcpyHostToDevice);
  return e;
}

}  // namespace fftk
