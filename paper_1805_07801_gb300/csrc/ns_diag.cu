// Diagnostics of a velocity state (paper Sec. 1 and Sec. 7: energy spectrum
// and flux) and the scale-by-scale energy transfer: the deterministic
// per-shell reduction, the energy transfer spectrum T(K) and flux Pi(K), the
// shell-to-shell transfer, and the diagnostics without device allocation.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft_engine.cuh"
#include "ns_common.cuh"

namespace fftk {

// nint(|k|) for integer |k|^2, exact: an FP32 square root corrected by
// integer comparisons; |k| >= K + 1/2 exactly when k2 >= K^2 + K + 1.
__device__ __forceinline__ long long shell_index(long long k2) {
  long long K = (long long)floorf(sqrtf((float)k2));
  while (K * K > k2) --K;
  while ((K + 1) * (K + 1) <= k2) ++K;
  if (k2 >= K * K + K + 1) ++K;
  return K;
}


// Blocks of the diagnostics reduction for a result of `width` doubles: up to
// eight per SM of 152, as many as the no-allocation scratch holds partials
// for (the same count on both paths, so both sum in the same order).
int diag_blocks(int width) {
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
// sum_K T(K), 0, T(K)).  Slot 0 is the sum of the shells.  nf: the number
// of components (fields M apart) in the dot products, 1 to 3.
__global__ void __launch_bounds__(DIAG_WARPS * 32)
    k_diag(const float2* __restrict__ u, const float2* __restrict__ nh, NSGeom g, double nu, int kmax,
           double* part, int nf) {
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
        if (f >= nf) break;
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

// The dynamic shared-memory limit is an attribute of the kernel (per device),
// not of a plan: it is raised once per device to what the largest grid needs,
// so that no plan lowers it under another plan's launches.
cudaError_t diag_attr() {
  static PerDevice once;
  return once.run([](int) {
    const int smem = (int)(sizeof(double) * DIAG_WARPS * (ns_kmax(1024) + 1));
    return cudaFuncSetAttribute(k_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
}

cudaError_t diag_launch(fftk_plan p, const float2* u, const float2* nh, double nu, cudaStream_t st, int nf) {
  NSWork* s = p->ns;
  const int width = 2 + s->kmax + 1;
  {
    LaunchScope ls(p, KK_NS_REDUCE, st);
    k_diag<<<diag_blocks(width), DIAG_WARPS * 32, s->diag_smem, st>>>(u, nh, s->g, nu, s->kmax, s->part, nf);
  }
  {
    LaunchScope ls(p, KK_NS_REDUCE, st);
    k_diag_final<<<(width + 127) / 128, 128, 0, st>>>(s->part, width, diag_blocks(width), s->dout);
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

}  // namespace fftk

using namespace fftk;

extern "C" int tarang_diag_kmax(fftk_plan p) { return p ? ns_kmax(p->nx) : -1; }

extern "C" fftk_status tarang_diag(fftk_plan p, const void* uhat, double nu, double* diag_host,
                                   void* cuda_stream) {
  if (!p || !uhat || !diag_host || misaligned16(uhat)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || !ns_size_ok(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
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
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || p->nx > 1024 || !is_pow2(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
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
      k_diag<<<diag_blocks(width), DIAG_WARPS * 32, s->diag_smem, st>>>(u, ph, g, 0.0, s->kmax, s->part, 3);
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
  // diag_blocks(width) never exceeds kNoAllocScratchDoubles / width, so the
  // partials of every n accepted above fit the scratch: at n = 1024 (width
  // 891) the reduction runs on 294 blocks instead of the 1216 it uses below
  // n = 256, and the allocating path uses the same count.
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
                                                   scratch, 3);
  k_diag_final<<<(width + 127) / 128, 128, 0, st>>>(scratch, width, diag_blocks(width), diag_dev);
  return from_cuda(cudaGetLastError());
}
