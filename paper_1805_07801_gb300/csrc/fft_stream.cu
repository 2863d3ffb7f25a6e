// Strided pass for lines of 512 points with TMA tile loads.
//
// The strided pass of the 3D transform (the y and x line transforms of
// Sec. 3) works on tiles of T = 16 adjacent columns x L rows.  Where the row
// stride Q is a multiple of 16 bytes (the x pass, Q = ny (nz/2+1)), a
// persistent CTA loads its tiles with TMA tiled copies (boxes of 16 columns x
// 256 rows) instead of 16 global loads per thread, and starts the next tile's
// copy as soon as the line engine has released the tile buffer, so the copy
// overlaps the last radix stage and the stores of the current tile.  Two
// such CTAs (512 threads, 64 KB each) share an SM.  For 1024-point lines the
// tile fills 128 KB and one CTA of 1024 threads holds the SM; there the copy
// has nothing to overlap and the pass with plain loads is the faster one.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "fft_engine.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace fftk {

template <int L>
struct PFCfg {
  static constexpr int G = 16;                                // values per thread
  static constexpr int S = L / G;                             // threads per line
  static constexpr int T = 16;                                // columns per tile (128-byte rows)
  static constexpr int THREADS = S * T;
  static constexpr int MINB = THREADS <= 512 ? 2 : 1;
  static constexpr int BOXR = 256;                            // rows per TMA box
  static constexpr int NBOX = L / BOXR;
  static constexpr size_t PBYTES = sizeof(float2) * (size_t)L * T;
  static constexpr size_t SMEM = PBYTES + 16;                 // + the tile mbarrier
};

using tcg::mbar_expect;
using tcg::tma_load3;

// Array [P][L][Q] of complex values, transform along L (element stride Q);
// tile t = (p, q-tile); in may equal out (tiles are disjoint column sets).
// The tile buffer doubles as the exchange buffer of the line engine; once the
// last exchange has been read, thread 0 starts the next tile's loads, which
// then overlap the last stage and the stores of this tile.
template <int L, int SIGN>
__global__ void __launch_bounds__(PFCfg<L>::THREADS, PFCfg<L>::MINB)
    k_cpass_tma(const __grid_constant__ CUtensorMap tmap, float2* out, int Q, int qtiles, int ntiles,
                const float2* __restrict__ tw, float scale, int* err) {
  using C = PFCfg<L>;
  constexpr int G = C::G, S = C::S, T = C::T;
  extern __shared__ __align__(128) float2 smf[];
  __shared__ int ok_flag;
  float2* P = smf;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smf + (size_t)L * T);
  const int tid = threadIdx.x;
  const int c = tid % T, j = tid / T;

  auto fetch = [&](int t) {  // thread 0: the NBOX boxes of tile t into P
    const int p = t / qtiles;
    const int q0 = (t - p * qtiles) * T;
    mbar_expect(bar, (uint32_t)C::PBYTES);
#pragma unroll 1
    for (int b = 0; b < C::NBOX; ++b) tma_load3(P + (size_t)b * C::BOXR * T, &tmap, 2 * q0, b * C::BOXR, p, bar);
  };

  if (tid == 0) tcg::mbar_init(bar);
  __syncthreads();
  uint32_t phase = 0;
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) fetch(t);
  for (; t < ntiles; t += gridDim.x) {
    if (tid == 0) ok_flag = tcg::mbar_wait(bar, phase) ? 1 : 0;
    __syncthreads();
    if (!ok_flag) {
      // The tile never arrived: its copy may still be pending, writing into
      // this CTA's shared memory and completing on the mbarrier there.  Thread
      // 0 reports, then waits once more (bounded) for that copy before the
      // CTA's shared memory is released; the other threads may leave.  The
      // error word is the only signal: the host treats it as fatal for the plan.
      if (tid == 0) {
        atomicOr(err, 1);
        tcg::mbar_wait(bar, phase);
      }
      return;
    }
    phase ^= 1;
    float2 v[G];
#pragma unroll
    for (int m = 0; m < G; ++m) v[m] = P[(j + m * S) * T + c];
    __syncthreads();  // the exchanges below overwrite P
    fft_line<L, G, SIGN>(v, j, ColX<T>{P, c}, tw);
    const int tn = t + (int)gridDim.x;
    if (tid == 0 && tn < ntiles) {  // every thread has read the last exchange: P is free
      tcg::fence_smem_async();
      fetch(tn);
    }
    const int p = t / qtiles;
    const int q = (t - p * qtiles) * T + c;
    if (q < Q) {
      float2* dst = out + (long long)p * L * Q + q;
#pragma unroll
      for (int m = 0; m < G; ++m) dst[(long long)(j + m * S) * Q] = cscale(v[m], scale);
    }
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

bool encode_f32_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                    const uint32_t* box) {
  if (rank < 1 || rank > 5 || reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
  for (int i = 0; i + 1 < rank; ++i)
    if (strides[i] % 16 != 0 || strides[i] >= (1ULL << 40)) return false;
  if ((box[0] * 4u) % 16 != 0) return false;
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  std::memset(m, 0, sizeof(*m));
  cuuint64_t d[5], s[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = (cuuint64_t)dims[i];
    b[i] = (cuuint32_t)box[i];
    e[i] = 1;
    if (i + 1 < rank) s[i] = (cuuint64_t)strides[i];
  }
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), d, s, b, e,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The 3D map [P][L][2Q] floats with boxes of 2T floats x 256 rows x 1; false
// where the layout breaks a TMA rule (row stride not a multiple of 16 bytes,
// base not 16-byte aligned, extents out of range) or no encoder exists.
template <int L>
static bool make_map(CUtensorMap* m, const float2* in, long long P, long long Q) {
  using C = PFCfg<L>;
  if (Q % 2 != 0 || reinterpret_cast<uintptr_t>(in) % 16 != 0) return false;
  if (2 * Q >= (1LL << 31) || P >= (1LL << 31) || (long long)L * Q * 8 >= (1LL << 40)) return false;
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  std::memset(m, 0, sizeof(*m));
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * Q), (cuuint64_t)L, (cuuint64_t)P};
  const cuuint64_t strides[2] = {(cuuint64_t)(8 * Q), (cuuint64_t)(8 * Q * L)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * C::T), (cuuint32_t)C::BOXR, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(in), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int L, int SIGN>
static cudaError_t cpass_tma_l(fftk_plan p, const CUtensorMap& m, float2* out, long long P, long long Q, float scale,
                               int kind, cudaStream_t st) {
  using C = PFCfg<L>;
  static PerDevice once;
  static int per_sm[kMaxDevices], nsm[kMaxDevices];
  int dev = 0;
  const cudaError_t attr_err = once.run(
      [](int d) {
        cudaError_t e =
            cudaFuncSetAttribute(k_cpass_tma<L, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[d], k_cpass_tma<L, SIGN>, C::THREADS, C::SMEM);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm[d], cudaDevAttrMultiProcessorCount, d);
        if (e == cudaSuccess && per_sm[d] < 1) e = cudaErrorInvalidConfiguration;
        return e;
      },
      &dev);
  if (attr_err != cudaSuccess) return attr_err;
  const long long qtiles = (Q + C::T - 1) / C::T;
  const long long ntiles = P * qtiles;
  const long long cap = (long long)nsm[dev] * per_sm[dev];
  const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
  LaunchScope ls(p, kind, st);
  k_cpass_tma<L, SIGN><<<grid, C::THREADS, C::SMEM, st>>>(m, out, (int)Q, (int)qtiles, (int)ntiles, twiddles(p, L),
                                                         scale, p->d_err);
  return cudaGetLastError();
}

template <int L>
static bool tma_map_l(CUtensorMap* m, const float2* in, long long P, long long Q) {
  using C = PFCfg<L>;
  if ((Q + C::T - 1) / C::T * P >= (1LL << 31)) return false;  // 32-bit tile indices
  return make_map<L>(m, in, P, Q);
}

bool launch_cpass_tma(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P, long long Q,
                      float scale, int kind, cudaStream_t st, cudaError_t* e) {
  if (P <= 0 || Q <= 0) return false;
  CUtensorMap m;
#define CASE(n)                                                                                  \
  case n:                                                                                        \
    if (!tma_map_l<n>(&m, in, P, Q)) return false;                                               \
    *e = sign < 0 ? cpass_tma_l<n, -1>(p, m, out, P, Q, scale, kind, st)                         \
                  : cpass_tma_l<n, +1>(p, m, out, P, Q, scale, kind, st);                        \
    return true;
  switch (L) { CASE(512) }
#undef CASE
  return false;
}

}  // namespace fftk
