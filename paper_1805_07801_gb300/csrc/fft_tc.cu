// Split-FP16 tensor-core radix-16 stages for the strided passes (dtype
// FFTK_R32_SPLIT16).
//
// A line of length L = 256 * R3 (R3 in {1, 2, 4, 8}) is transformed as two
// radix-16 Stockham stages on the 5th-generation tensor cores and, when
// R3 > 1, one FP32 radix-R3 stage.  A radix-16 stage over a batch of DFT rows
// is the product D = A B:
//   A [rows x 64] FP16: for each of the row's 16 complex inputs x (already
//     twiddled, scaled by a power of two), the four values hi.re, hi.im,
//     lo.re, lo.im with hi = fp16(x), lo = fp16(x - hi);
//   B = B1 + B2 [64 x 32] FP16: the real form of W16 = exp(SIGN 2 pi i r k/16)
//     split W = W_hi + W_lo; B1 multiplies both hi and lo by W_hi, B2 the hi
//     part by W_lo, so D = (x_hi + x_lo) W_hi + x_hi W_lo (FP32 accumulate in
//     TMEM), dropping only x_lo W_lo (2^-22 relative).
// Twiddles, scaling and the radix-R3 stage stay in FP32.
//
// One CTA of 128 threads owns 512 DFT rows (four M = 128 blocks, one TMEM lane
// per thread and block); thread 0 issues tcgen05.mma (M = 128, N = 32,
// K = 16), completion is signalled through an mbarrier, and every thread
// reads its own rows back with tcgen05.ld.  Operands use the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices, 128 bytes
// apart along K (LBO) and 1024 bytes apart along M/N (SBO).
#include <cuda_fp16.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {
namespace tc {

constexpr int kThreads = 128;
constexpr int kRows = 512;               // DFT rows per stage per tile
constexpr int kBlocks = kRows / 128;     // M blocks
constexpr uint32_t kLBO = 128;           // bytes between core matrices along K
constexpr uint32_t kSBO = 1024;          // bytes between 8-row groups (64 FP16 per row)
constexpr int kBlkBytes = 16 * 1024;     // one M block of A
constexpr int kBlkStride = kBlkBytes + 16;  // + 16 bytes: spreads blocks over banks
constexpr int kABytes = kBlocks * kBlkStride;
constexpr int kBBytes = 4 * 1024;        // one 32 x 64 operand
constexpr int kTmemCols = 128;
constexpr long long kSpinLimit = 1LL << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // tcgen05 descriptor version; no swizzle
  return d;
}

// byte offset of element (row, k) inside the A tile
__device__ __forceinline__ int a_off(int row, int k) {
  const int r = row & 127;
  return (row >> 7) * kBlkStride + (r >> 3) * (int)kSBO + (k >> 3) * (int)kLBO + (r & 7) * 16 + (k & 7) * 2;
}

// D = F32, A = B = F16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (long long it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(phase));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// hi/lo split of one complex value, packed (hi.re, hi.im, lo.re, lo.im)
__device__ __forceinline__ uint2 split2(float2 a) {
  const __half2 hi = __floats2half2_rn(a.x, a.y);
  const float2 hf = __half22float2(hi);
  const __half2 lo = __floats2half2_rn(a.x - hf.x, a.y - hf.y);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&hi), *reinterpret_cast<const uint32_t*>(&lo));
}

// power of two that brings max |v| to [2^10, 2^11)
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f)) return 1.f;
  int e;
  frexpf(m, &e);
  return ldexpf(1.f, 11 - e);
}

}  // namespace tc

template <int L>
struct TCCfg {
  static constexpr int R3 = L / 256;
  static constexpr int S1 = L / 16;            // butterflies per column in each radix-16 stage
  static constexpr int T = tc::kRows / S1;     // columns per tile
  static constexpr int LOGS1 = Log2<S1>::value;
  static constexpr int LOGT = Log2<T>::value;
  static constexpr int LOGL = Log2<L>::value;
  static constexpr size_t SMEM = 1024 + tc::kABytes + 2 * tc::kBBytes + sizeof(float) * T + 64;
};

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
template <int L, int SIGN>
__global__ void __launch_bounds__(tc::kThreads)
    k_cpass_tc(const float2* in, float2* out, long long Q, long long qtiles, long long ntiles,
               const float2* __restrict__ tw, int twlog, float out_scale,
               const __half* __restrict__ bops, int* err) {
  using C = TCCfg<L>;
  constexpr int T = C::T, S1 = C::S1, R3 = C::R3;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = smraw + ((1024 - (tc::su32(smraw) & 1023)) & 1023);
  unsigned char* As = base;                                   // A tile, reused as FP32 exchange
  unsigned char* Bs = base + tc::kABytes;                     // B1, B2
  float* colmax = reinterpret_cast<float*>(Bs + 2 * tc::kBBytes);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(colmax + T + (T & 1));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5;

  for (int i = t; i < 2 * tc::kBBytes / 16; i += tc::kThreads)
    reinterpret_cast<uint4*>(Bs)[i] = reinterpret_cast<const uint4*>(bops)[i];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::su32(tslot)),
                 "r"(tc::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tc::su32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tslot;
  const uint32_t a_sa = tc::su32(As), b1_sa = tc::su32(Bs), b2_sa = b1_sa + tc::kBBytes;
  const uint32_t lane_base = tmem + (((uint32_t)warp * 32u) << 16);
  uint32_t phase = 0;
  bool failed = false;

  auto run_mma = [&]() -> bool {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (t == 0) {
#pragma unroll
      for (int blk = 0; blk < tc::kBlocks; ++blk) {
        const uint32_t d = tmem + 32u * blk;
        const uint32_t a = a_sa + blk * tc::kBlkStride;
#pragma unroll
        for (int s = 0; s < 4; ++s) tc::mma(d, tc::desc(a + 256 * s), tc::desc(b1_sa + 256 * s), s > 0);
#pragma unroll
        for (int s = 0; s < 4; ++s) tc::mma(d, tc::desc(a + 256 * s), tc::desc(b2_sa + 256 * s), 1);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          tc::su32(mbar)));
    }
    const bool ok = tc::mbar_wait(mbar, phase);
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    return __syncthreads_and(ok) != 0;
  };

  for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const long long p = tile / qtiles;
    const long long q0 = (tile - p * qtiles) * T;
    const float2* src = in + p * (long long)L * Q + q0;
    float2* dst = out + p * (long long)L * Q + q0;
    if (t < T) colmax[t] = 0.f;
    float s1[tc::kBlocks];
    // ---- stage 1: rows (b, c), inputs x[b + r S1][c], per-row power-of-two scale
#pragma unroll 1
    for (int blk = 0; blk < tc::kBlocks; ++blk) {
      const int row = t + 128 * blk;
      const int b = row >> C::LOGT, c = row & (T - 1);
      const bool valid = q0 + c < Q;
      float2 x[16];
      float m = 0.f;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        x[r] = valid ? src[(long long)(b + r * S1) * Q + c] : make_float2(0.f, 0.f);
        m = fmaxf(m, fmaxf(fabsf(x[r].x), fabsf(x[r].y)));
      }
      const float s = tc::pow2_scale(m);
      s1[blk] = s;
#pragma unroll
      for (int r = 0; r < 16; r += 2) {
        const uint2 u0 = tc::split2(cscale(x[r], s)), u1 = tc::split2(cscale(x[r + 1], s));
        *reinterpret_cast<uint4*>(As + tc::a_off(row, 4 * r)) = make_uint4(u0.x, u0.y, u1.x, u1.y);
      }
    }
    if (!run_mma()) {
      failed = true;
      break;
    }
    // ---- column maxima of the stage-1 output
#pragma unroll 1
    for (int blk = 0; blk < tc::kBlocks; ++blk) {
      float d[32];
      tc::ld32(lane_base + 32u * blk, d);
      float m = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) m = fmaxf(m, fabsf(d[i]));
      const int c = (t + 128 * blk) & (T - 1);
      atomicMax(reinterpret_cast<int*>(&colmax[c]), __float_as_int(m / s1[blk]));
    }
    __syncthreads();
    // ---- stage 2 inputs: output r' of row (b, c) sits at p = 16 b + r', which
    //      is input r = p / S1 of butterfly b2 = p mod S1, twiddle W_256^(r (b2 mod 16))
#pragma unroll 1
    for (int blk = 0; blk < tc::kBlocks; ++blk) {
      const int row = t + 128 * blk;
      const int b = row >> C::LOGT, c = row & (T - 1);
      const float inv = 1.f / s1[blk];
      const float s2 = tc::pow2_scale(colmax[c]);
      float d[32];
      tc::ld32(lane_base + 32u * blk, d);
#pragma unroll
      for (int rp = 0; rp < 16; ++rp) {
        const int pp = 16 * b + rp;
        const int b2 = pp & (S1 - 1), r2 = pp >> C::LOGS1;
        const int k2 = b2 & 15;
        const float2 w = __ldg(&tw[(r2 * k2) << (twlog - 8)]);
        float2 y = make_float2(d[2 * rp] * inv, d[2 * rp + 1] * inv);
        y = SIGN < 0 ? cmul(y, w) : cmulc(y, w);
        const uint2 u = tc::split2(cscale(y, s2));
        *reinterpret_cast<uint2*>(As + tc::a_off((b2 << C::LOGT) + c, 4 * r2)) = u;
      }
    }
    if (!run_mma()) {
      failed = true;
      break;
    }
    // ---- stage 2 outputs: row (b2, c), output r'' at (b2 - k2) 16 + k2 + 16 r''
    float2* X = reinterpret_cast<float2*>(As);  // FP32 exchange [L][T] for the radix-R3 stage
    if constexpr (R3 > 1) __syncthreads();
#pragma unroll 1
    for (int blk = 0; blk < tc::kBlocks; ++blk) {
      const int row = t + 128 * blk;
      const int b2 = row >> C::LOGT, c = row & (T - 1);
      const int k2 = b2 & 15;
      const float inv = 1.f / tc::pow2_scale(colmax[c]);
      float d[32];
      tc::ld32(lane_base + 32u * blk, d);
#pragma unroll
      for (int rp = 0; rp < 16; ++rp) {
        const int pos = (b2 - k2) * 16 + k2 + 16 * rp;
        const float2 y = make_float2(d[2 * rp] * inv, d[2 * rp + 1] * inv);
        if constexpr (R3 == 1) {
          if (q0 + c < Q) dst[(long long)pos * Q + c] = cscale(y, out_scale);
        } else {
          X[pos * T + c] = y;
        }
      }
    }
    if constexpr (R3 > 1) {
      // ---- radix-R3 stage in FP32: butterfly b3 < 256 reads b3 + r 256 with
      //      twiddle W_L^(r b3); outputs land at b3 + r' 256 (natural order)
      __syncthreads();
#pragma unroll 1
      for (int i = t; i < 256 * T; i += tc::kThreads) {
        const int b3 = i >> C::LOGT, c = i & (T - 1);
        float2 v[R3];
#pragma unroll
        for (int r = 0; r < R3; ++r) {
          v[r] = X[(b3 + 256 * r) * T + c];
          if (r > 0) {
            const float2 w = __ldg(&tw[(r * b3) << (twlog - C::LOGL)]);
            v[r] = SIGN < 0 ? cmul(v[r], w) : cmulc(v[r], w);
          }
        }
        dftR<R3, SIGN>(v);
        if (q0 + c < Q) {
#pragma unroll
          for (int r = 0; r < R3; ++r) dst[(long long)(b3 + 256 * r) * Q + c] = cscale(v[r], out_scale);
        }
      }
    }
    __syncthreads();
  }
  if (failed && t == 0) atomicOr(err, 1);
  if (failed) tc::mbar_wait(mbar, phase);  // let in-flight MMAs drain (bounded) before freeing TMEM
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tc::kTmemCols));
}

template <int L, int SIGN>
static cudaError_t cpass_tc_l(fftk_plan p, const float2* in, float2* out, long long P, long long Q,
                              float scale, int kind, cudaStream_t st) {
  using C = TCCfg<L>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int per_sm = 1;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_cpass_tc<L, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)C::SMEM);
    if (attr_err == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cpass_tc<L, SIGN>, tc::kThreads, C::SMEM) !=
            cudaSuccess)
      per_sm = 1;
    if (per_sm > 3) per_sm = 3;  // 3 x 128 TMEM columns fit in 512
    if (per_sm < 1) per_sm = 1;
  });
  if (attr_err != cudaSuccess) return attr_err;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long qtiles = (Q + C::T - 1) / C::T;
  const long long ntiles = P * qtiles;
  const long long cap = (long long)per_sm * sms;
  const int blocks = (int)(ntiles < cap ? ntiles : cap);
  const __half* bops = p->d_dft16 + (SIGN < 0 ? 0 : 2 * 32 * 64);
  LaunchScope ls(p, kind, st);
  k_cpass_tc<L, SIGN><<<blocks, tc::kThreads, C::SMEM, st>>>(in, out, Q, qtiles, ntiles, p->d_tw, p->twlog,
                                                           scale, bops, p->d_err);
  return cudaGetLastError();
}

bool cpass_tc_supported(int L) { return L == 256 || L == 512 || L == 1024 || L == 2048; }

cudaError_t launch_cpass_tc(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P,
                            long long Q, float scale, int kind, cudaStream_t st) {
  if (P <= 0 || Q <= 0) return cudaSuccess;
#define TC_CASE(n)                                                              \
  case n:                                                                       \
    return sign < 0 ? cpass_tc_l<n, -1>(p, in, out, P, Q, scale, kind, st)      \
                    : cpass_tc_l<n, +1>(p, in, out, P, Q, scale, kind, st);
  switch (L) {
    TC_CASE(256)
    TC_CASE(512)
    TC_CASE(1024)
    TC_CASE(2048)
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
