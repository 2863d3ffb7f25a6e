// C ABI entry points for the transforms, the planner and instrumentation.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "fft_engine.cuh"
#include "internal.h"

namespace fftk {

const char* const kKernelNames[KK_COUNT] = {
    "z_r2c", "y_fwd", "x_fwd", "x_inv", "y_inv", "z_c2r",
    "ns_invx_curl", "ns_invy", "ns_z_product", "ns_fwdy", "ns_fwdx_update",
    "ns_reduce", "aux", "sc_fwd", "sc_inv", "rbc_prep", "rbc_z", "rbc_update"};

bool is_pow2(long long v) { return v >= 1 && (v & (v - 1)) == 0; }
bool is_pow2_or_3x(long long v) { return is_pow2(v) || (v % 3 == 0 && is_pow2(v / 3)); }

// A transform length the passes support: a power of two up to 4096, or
// 3 * 2^m (a radix-3 step over power-of-two sub-lines of at least 2 points)
// up to 3072; along z (halved by the real packing) at least 12.
static bool dim_ok(int n, bool z) {
  if (is_pow2(n)) return n <= 4096 && (!z || n >= 2);
  if (n % 3 != 0 || !is_pow2(n / 3)) return false;
  return n <= 3072 && n >= (z ? 12 : 6);
}
int ilog2(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

cudaEvent_t Profiler::take() {
  if (next < pool.size()) return pool[next++];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  pool.push_back(e);
  ++next;
  return e;
}

void Profiler::clear() {
  recs.clear();
  next = 0;
}

Profiler::~Profiler() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

LaunchScope::LaunchScope(fftk_plan p_, int kind_, cudaStream_t st_) : p(p_), kind(kind_), st(st_) {
  p->launches.fetch_add(1, std::memory_order_relaxed);
  if (p->prof.on) {
    cudaEvent_t a = p->prof.take();
    b = p->prof.take();
    if (a && b) {
      cudaEventRecord(a, st);
      p->prof.recs.push_back({kind, a, b});
    } else {
      b = nullptr;
    }
  }
}

LaunchScope::~LaunchScope() {
  if (b) cudaEventRecord(b, st);
}

static bool misaligned(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0; }

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

static thread_local cudaError_t g_last_cuda = cudaSuccess;

fftk_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FFTK_OK;
  g_last_cuda = e;
  if (e == cudaErrorMemoryAllocation) return FFTK_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return FFTK_ERR_NO_DEVICE;
  return FFTK_ERR_CUDA;
}

// Plan-owned workspace of at least `bytes`.
static fftk_status ensure_ws(fftk_plan p, size_t bytes, void** out) {
  std::lock_guard<std::mutex> g(p->mu);
  if (p->ws && p->ws_bytes >= bytes) {
    *out = p->ws;
    return FFTK_OK;
  }
  if (p->ws && !p->ws_owned) return FFTK_ERR_INVALID_ARG;  // caller's buffer is too small
  if (p->ws) cudaFree(p->ws);
  p->ws = nullptr;
  p->ws_bytes = 0;
  void* w = nullptr;
  cudaError_t e = cudaMalloc(&w, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FFTK_ERR_OOM;
  }
  p->ws = w;
  p->ws_bytes = bytes;
  p->ws_owned = true;
  *out = w;
  return FFTK_OK;
}

}  // namespace fftk

using namespace fftk;

extern "C" const char* fftk_status_string(fftk_status s) {
  switch (s) {
    case FFTK_OK: return "FFTK_OK";
    case FFTK_ERR_INVALID_ARG: return "FFTK_ERR_INVALID_ARG";
    case FFTK_ERR_UNSUPPORTED_SIZE: return "FFTK_ERR_UNSUPPORTED_SIZE";
    case FFTK_ERR_NO_DEVICE: return "FFTK_ERR_NO_DEVICE";
    case FFTK_ERR_OOM: return "FFTK_ERR_OOM";
    case FFTK_ERR_CUDA: return "FFTK_ERR_CUDA";
    case FFTK_ERR_NONFINITE: return "FFTK_ERR_NONFINITE";
    case FFTK_ERR_TIMEOUT: return "FFTK_ERR_TIMEOUT";
  }
  return "FFTK_ERR_UNKNOWN";
}

extern "C" const char* fftk_last_cuda_error(void) {
  return g_last_cuda == cudaSuccess ? "" : cudaGetErrorName(g_last_cuda);
}

extern "C" fftk_status fftk_plan_create(int nx, int ny, int nz, fftk_dtype dtype, fftk_plan* out) {
  if (!out) return FFTK_ERR_INVALID_ARG;
  *out = nullptr;
  if (dtype != FFTK_R32 && dtype != FFTK_R32_SPLIT16) return FFTK_ERR_INVALID_ARG;
  if (!dim_ok(nx, false) || !dim_ok(ny, false) || !dim_ok(nz, true)) return FFTK_ERR_UNSUPPORTED_SIZE;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return FFTK_ERR_NO_DEVICE;
  }
  fftk_plan p = new (std::nothrow) fftk_plan_s;
  if (!p) return FFTK_ERR_OOM;
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->hz = nz / 2 + 1;
  p->dtype = dtype;
  cudaGetDevice(&p->device);
  int lt = nx;
  if (ny > lt) lt = ny;
  if (nz > lt) lt = nz;
  p->twlog = ilog2(lt);
  // Twiddle tables in FP64 (host libm), rounded once to FP32: for every
  // power of two L <= 4 LT, exp(-2 pi i m / L), m < L, at offset L (8 LT
  // values; the sizes above LT are the sine/cosine passes' quarter waves).
  const int ltab = 4 * lt;
  std::vector<float2> h((size_t)fftk::kStageTwiddles + 2 * (size_t)ltab, make_float2(1.f, 0.f));
  float2* pyr = h.data() + fftk::kStageTwiddles;
  const double two_pi = 6.283185307179586476925286766559;
  for (int L = 1; L <= ltab; L *= 2)
    for (int m = 0; m < L; ++m) {
      const double ang = two_pi * (double)m / (double)L;
      pyr[(size_t)L + m] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
    }
  // Below the pyramid, the line engine's per-stage tables: for each stage
  // span M (a power of two up to the longest line) and radix R, the entry
  // r (M/R) + k is exp(-2 pi i r k / M), r < R, k < M/R.
  for (int M = 4; M <= lt && M <= 4096; M *= 2)
    for (int R = 2; R <= 16 && R <= M / 2; R *= 2) {
      const int ns = M / R;
      for (int r = 0; r < R; ++r)
        for (int k = 0; k < ns; ++k) {
          const double ang = two_pi * (double)(r * k) / (double)M;
          h[(size_t)fftk::stage_tw_offset(M, R) + (size_t)r * ns + k] =
              make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
        }
    }
  e = cudaMalloc(&p->d_tw_alloc, sizeof(float2) * h.size());
  if (e == cudaSuccess) {
    p->d_tw = p->d_tw_alloc + fftk::kStageTwiddles;
    e = cudaMemcpy(p->d_tw_alloc, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice);
  }
  // tables of size 3 * 2^j for the radix-3 lines, at offset L (2 L3 values)
  int lt3 = 0;
  for (int d : {nx, ny, nz})
    if (!is_pow2(d) && d > lt3) lt3 = d;
  if (e == cudaSuccess && lt3 > 0) {
    std::vector<float2> h3(2 * (size_t)lt3, make_float2(1.f, 0.f));
    for (int L = 3; L <= lt3; L *= 2)
      for (int m = 0; m < L; ++m) {
        const double ang = two_pi * (double)m / (double)L;
        h3[(size_t)L + m] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
      }
    e = cudaMalloc(&p->d_tw3, sizeof(float2) * h3.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_tw3, h3.data(), sizeof(float2) * h3.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e == cudaSuccess && dtype == FFTK_R32_SPLIT16) e = upload_dft16_operands(p);
  if (e != cudaSuccess) {
    fftk_status s = from_cuda(e);
    cudaGetLastError();
    if (p->d_tw_alloc) cudaFree(p->d_tw_alloc);
    if (p->d_tw3) cudaFree(p->d_tw3);
    if (p->d_err) cudaFree(p->d_err);
    if (p->d_dft16) cudaFree(p->d_dft16);
    delete p;
    return s;
  }
  *out = p;
  return FFTK_OK;
}

void ns_free(fftk_plan p);  // ns.cu

extern "C" fftk_status fftk_plan_destroy(fftk_plan p) {
  if (!p) return FFTK_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  ns_free(p);
  if (p->d_tw_alloc) cudaFree(p->d_tw_alloc);
  if (p->d_tw3) cudaFree(p->d_tw3);
  if (p->d_err) cudaFree(p->d_err);
  if (p->d_dft16) cudaFree(p->d_dft16);
  if (p->ws && p->ws_owned) cudaFree(p->ws);
  delete p;
  return FFTK_OK;
}

// bytes of `batch` half-complex spectra
static size_t spec_bytes(fftk_plan p, int batch) {
  return (size_t)batch * (size_t)p->nx * (size_t)p->ny * (size_t)p->hz * sizeof(float2);
}

// With both strided passes, r2c and c2r run each of them out of place (one
// spectrum-sized array of workspace for r2c, two for c2r); every pass then
// reads one array and writes another, which measured faster than the same
// pass in place (1024^3: forward y 2.19 -> 2.07 ms, forward x 2.10 -> 2.01 ms,
// inverse y 2.15 -> 2.04 ms).
extern "C" size_t fftk_workspace_bytes(fftk_plan p, int batch) {
  if (!p || batch < 1) return 0;
  return spec_bytes(p, batch) * ((p->nx > 1 && p->ny > 1) ? 2 : 1);
}

// Workspace for the strided passes: `want` spectrum-sized arrays (1 or 2) if
// the plan's workspace holds them or they can be allocated, else `need`
// arrays (the passes then run in place where the second array is missing);
// *got = the number of arrays obtained (0 when none were needed and none
// could be had).
static fftk_status pass_ws(fftk_plan p, size_t spec, int want, int need, float2** w, int* got) {
  void* wv = nullptr;
  *got = 0;
  for (int k = want; k >= 1; --k) {
    const fftk_status s = ensure_ws(p, (size_t)k * spec, &wv);
    if (s == FFTK_OK) {
      *w = static_cast<float2*>(wv);
      *got = k;
      return FFTK_OK;
    }
    if (k <= need) return s;
  }
  return FFTK_OK;
}

extern "C" fftk_status fftk_set_workspace(fftk_plan p, void* dev_ptr, size_t bytes) {
  if (!p) return FFTK_ERR_INVALID_ARG;
  if ((dev_ptr == nullptr) != (bytes == 0)) return FFTK_ERR_INVALID_ARG;
  if (dev_ptr && misaligned(dev_ptr)) return FFTK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(p->mu);
  if (p->ws && p->ws_owned) cudaFree(p->ws);
  p->ws = dev_ptr;
  p->ws_bytes = bytes;
  p->ws_owned = false;
  return FFTK_OK;
}

// y or x pass: the split-FP16 tensor-core kernel where the plan asks for it
// and the line length has two radix-16 stages, the FP32 kernel otherwise.
static cudaError_t strided_pass(fftk_plan p, int L, int sign, const float2* in, float2* out,
                                long long P, long long Q, float scale, int kind, cudaStream_t st) {
  if (!is_pow2(L)) return launch_cpass3(p, L, sign, in, out, P, Q, scale, kind, st);
  if (p->dtype == FFTK_R32_SPLIT16 && cpass_tc_supported(L))
    return launch_cpass_tc(p, L, sign, in, out, P, Q, scale, kind, st);
  cudaError_t e = cudaSuccess;
  if (launch_cpass_tma(p, L, sign, in, out, P, Q, scale, kind, st, &e)) return e;
  return launch_cpass(p, L, sign, in, out, P, Q, scale, kind, st);
}

namespace fftk {
cudaError_t r2c_scaled(fftk_plan p, const float* in, float2* out, long long B, float scale, cudaStream_t st,
                       float2* scratch) {
  const bool do_y = p->ny > 1, do_x = p->nx > 1;
  // with a scratch array the y pass writes it and the x pass reads it back
  float2* mid = (scratch && do_x && do_y) ? scratch : out;
  cudaError_t e = launch_z_r2c(p, in, out, B * p->nx * p->ny, (do_x || do_y) ? 1.f : scale, st);
  if (e == cudaSuccess && do_y)
    e = strided_pass(p, p->ny, -1, out, mid, B * p->nx, p->hz, do_x ? 1.f : scale, KK_Y_FWD, st);
  if (e == cudaSuccess && do_x)
    e = strided_pass(p, p->nx, -1, do_y ? mid : out, out, B, (long long)p->ny * p->hz, scale, KK_X_FWD, st);
  return e;
}

cudaError_t c2r_overwrite(fftk_plan p, float2* spec, float* out, long long B, cudaStream_t st, float2* scratch) {
  // with a scratch array of the spectrum's size the x pass writes it and the
  // y pass reads it back (both out of place)
  float2* mid = (scratch && p->nx > 1 && p->ny > 1) ? scratch : spec;
  cudaError_t e = cudaSuccess;
  if (p->nx > 1) e = strided_pass(p, p->nx, +1, spec, mid, B, (long long)p->ny * p->hz, 1.f, KK_X_INV, st);
  if (e == cudaSuccess && p->ny > 1)
    e = strided_pass(p, p->ny, +1, p->nx > 1 ? mid : spec, spec, B * p->nx, p->hz, 1.f, KK_Y_INV, st);
  if (e == cudaSuccess) e = launch_z_c2r(p, spec, out, B * p->nx * p->ny, st);
  return e;
}
}  // namespace fftk

extern "C" fftk_status fftk_r2c(fftk_plan p, const float* in, void* out, int batch,
                                void* cuda_stream) {
  if (!p || !in || !out || batch < 1) return FFTK_ERR_INVALID_ARG;
  if (misaligned(in) || misaligned(out)) return FFTK_ERR_INVALID_ARG;
  const long long B = batch;
  const size_t in_bytes = (size_t)B * p->nx * p->ny * p->nz * sizeof(float);
  const size_t out_bytes = spec_bytes(p, batch);
  if (overlap(in, in_bytes, out, out_bytes)) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float2* o = static_cast<float2*>(out);
  const float scale = (float)(1.0 / ((double)p->nx * (double)p->ny * (double)p->nz));
  const bool do_y = p->ny > 1, do_x = p->nx > 1;
  // with both strided passes, the y pass writes the plan's workspace and the
  // x pass reads it back into `out` (in place in `out` when no workspace can
  // be had)
  float2* mid = o;
  if (do_x && do_y) {
    float2* w = nullptr;
    int got = 0;
    fftk_status s = pass_ws(p, out_bytes, 1, 0, &w, &got);
    if (s != FFTK_OK) return s;
    if (got) {
      if (overlap(w, out_bytes, in, in_bytes) || overlap(w, out_bytes, out, out_bytes)) return FFTK_ERR_INVALID_ARG;
      mid = w;
    }
  }
  cudaError_t e = launch_z_r2c(p, in, o, B * p->nx * p->ny, (do_x || do_y) ? 1.f : scale, st);
  if (e == cudaSuccess && do_y)
    e = strided_pass(p, p->ny, -1, o, mid, B * p->nx, p->hz, do_x ? 1.f : scale, KK_Y_FWD, st);
  if (e == cudaSuccess && do_x)
    e = strided_pass(p, p->nx, -1, mid, o, B, (long long)p->ny * p->hz, scale, KK_X_FWD, st);
  return from_cuda(e);
}

extern "C" fftk_status fftk_c2r(fftk_plan p, const void* in, float* out, int batch,
                                void* cuda_stream) {
  if (!p || !in || !out || batch < 1) return FFTK_ERR_INVALID_ARG;
  if (misaligned(in) || misaligned(out)) return FFTK_ERR_INVALID_ARG;
  const long long B = batch;
  const size_t in_bytes = spec_bytes(p, batch);
  const size_t out_bytes = (size_t)B * p->nx * p->ny * p->nz * sizeof(float);
  if (overlap(in, in_bytes, out, out_bytes)) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const float2* src = static_cast<const float2*>(in);
  const bool do_x = p->nx > 1, do_y = p->ny > 1;
  cudaError_t e = cudaSuccess;
  if (do_x || do_y) {
    // x: in -> w0, y: w0 -> w1 (both passes out of place), z: -> out; with
    // one array of workspace the y pass runs in place in w0
    float2* w0 = nullptr;
    int got = 0;
    fftk_status s = pass_ws(p, in_bytes, (do_x && do_y) ? 2 : 1, 1, &w0, &got);
    if (s != FFTK_OK) return s;
    const size_t wb = (size_t)got * in_bytes;
    if (overlap(w0, wb, in, in_bytes) || overlap(w0, wb, out, out_bytes)) return FFTK_ERR_INVALID_ARG;
    float2* w1 = got == 2 ? w0 + in_bytes / sizeof(float2) : w0;
    if (do_x) {
      e = strided_pass(p, p->nx, +1, src, w0, B, (long long)p->ny * p->hz, 1.f, KK_X_INV, st);
      src = w0;
    }
    if (e == cudaSuccess && do_y) {
      e = strided_pass(p, p->ny, +1, src, w1, B * p->nx, p->hz, 1.f, KK_Y_INV, st);
      src = w1;
    }
  }
  if (e == cudaSuccess) e = launch_z_c2r(p, src, out, B * p->nx * p->ny, st);
  return from_cuda(e);
}

// ------------------------------------------------------ mixed bases ----
// Fourier axes trailing (FFF, SFF, SSF, SSS; Sec. 2.1); every axis of a
// sine/cosine basis longer than 1 point, z even.
static bool basis_ok(fftk_plan p, const int* b) {
  for (int d = 0; d < 3; ++d)
    if (b[d] != FFTK_FOURIER && b[d] != FFTK_SINE && b[d] != FFTK_COSINE) return false;
  if (b[0] == FFTK_FOURIER && (b[1] != FFTK_FOURIER || b[2] != FFTK_FOURIER)) return false;
  if (b[1] == FFTK_FOURIER && b[2] != FFTK_FOURIER) return false;
  if (b[0] != FFTK_FOURIER && (p->nx < 2 || !is_pow2(p->nx))) return false;
  if (b[1] != FFTK_FOURIER && (p->ny < 2 || !is_pow2(p->ny))) return false;
  if (b[2] != FFTK_FOURIER && !is_pow2(p->nz)) return false;
  return true;
}

static size_t basis_spectrum_bytes(fftk_plan p, const int* b, int batch) {
  const size_t cells = (size_t)batch * p->nx * p->ny;
  return b[2] == FFTK_FOURIER ? cells * p->hz * sizeof(float2) : cells * p->nz * sizeof(float);
}

// One x or y pass over float2 columns: Fourier (plan dtype) or sine/cosine.
static cudaError_t axis_pass(fftk_plan p, int basis, int L, int dir, const float2* in, float2* out, long long P,
                             long long Q, float scale, int fkind, cudaStream_t st) {
  if (basis == FFTK_FOURIER) return strided_pass(p, L, dir, in, out, P, Q, scale, fkind, st);
  return launch_scpass(p, L, basis == FFTK_SINE, dir, in, out, P, Q, scale, dir < 0 ? KK_SC_FWD : KK_SC_INV, st);
}

extern "C" fftk_status fftk_forward(fftk_plan p, const int* basis, const float* in, void* out, int batch,
                                    void* cuda_stream) {
  if (!p || !basis || !in || !out || batch < 1) return FFTK_ERR_INVALID_ARG;
  if (misaligned(in) || misaligned(out) || !basis_ok(p, basis)) return FFTK_ERR_INVALID_ARG;
  const long long B = batch;
  const size_t in_bytes = (size_t)B * p->nx * p->ny * p->nz * sizeof(float);
  if (overlap(in, in_bytes, out, basis_spectrum_bytes(p, basis, batch))) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const float sx = (float)(1.0 / p->nx), sy = (float)(1.0 / p->ny), sz = (float)(1.0 / p->nz);
  cudaError_t e;
  long long qy, qx;  // float2 columns of the y and x passes
  float2* o = static_cast<float2*>(out);
  if (basis[2] == FFTK_FOURIER) {
    e = launch_z_r2c(p, in, o, B * p->nx * p->ny, sz, st);
    qy = p->hz;
  } else {
    e = launch_scz(p, basis[2] == FFTK_SINE, -1, in, static_cast<float*>(out), B * p->nx * p->ny, sz, KK_SC_FWD,
                   st);
    qy = p->nz / 2;  // a real field read as pairs of adjacent z values
  }
  qx = (long long)p->ny * qy;
  if (e == cudaSuccess && p->ny > 1) e = axis_pass(p, basis[1], p->ny, -1, o, o, B * p->nx, qy, sy, KK_Y_FWD, st);
  if (e == cudaSuccess && p->nx > 1) e = axis_pass(p, basis[0], p->nx, -1, o, o, B, qx, sx, KK_X_FWD, st);
  return from_cuda(e);
}

extern "C" fftk_status fftk_inverse(fftk_plan p, const int* basis, const void* in, float* out, int batch,
                                    void* cuda_stream) {
  if (!p || !basis || !in || !out || batch < 1) return FFTK_ERR_INVALID_ARG;
  if (misaligned(in) || misaligned(out) || !basis_ok(p, basis)) return FFTK_ERR_INVALID_ARG;
  const long long B = batch;
  const size_t in_bytes = basis_spectrum_bytes(p, basis, batch);
  const size_t out_bytes = (size_t)B * p->nx * p->ny * p->nz * sizeof(float);
  if (overlap(in, in_bytes, out, out_bytes)) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const bool zf = basis[2] == FFTK_FOURIER;
  const long long qy = zf ? p->hz : p->nz / 2, qx = (long long)p->ny * qy;
  const float2* src = static_cast<const float2*>(in);
  cudaError_t e = cudaSuccess;
  // the x and y passes run in the plan's workspace (Fourier z) or in `out`
  // (all-real spectra have the size of the field); `in` is not modified
  float2* w = reinterpret_cast<float2*>(out);
  if (zf && (p->nx > 1 || p->ny > 1)) {
    void* wv = nullptr;
    fftk_status s = ensure_ws(p, in_bytes, &wv);
    if (s != FFTK_OK) return s;
    if (overlap(wv, in_bytes, in, in_bytes) || overlap(wv, in_bytes, out, out_bytes)) return FFTK_ERR_INVALID_ARG;
    w = static_cast<float2*>(wv);
  }
  if (p->nx > 1) {
    e = axis_pass(p, basis[0], p->nx, +1, src, w, B, qx, 1.f, KK_X_INV, st);
    src = w;
  }
  if (e == cudaSuccess && p->ny > 1) {
    e = axis_pass(p, basis[1], p->ny, +1, src, w, B * p->nx, qy, 1.f, KK_Y_INV, st);
    src = w;
  }
  if (e == cudaSuccess) {
    if (zf)
      e = launch_z_c2r(p, src, out, B * p->nx * p->ny, st);
    else
      e = launch_scz(p, basis[2] == FFTK_SINE, +1, reinterpret_cast<const float*>(src), out, B * p->nx * p->ny,
                     1.f, KK_SC_INV, st);
  }
  return from_cuda(e);
}

extern "C" fftk_status fftk_sync(fftk_plan p, void* cuda_stream) {
  if (!p) return FFTK_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return from_cuda(e);
  int err = 0;
  e = cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  if (err) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return FFTK_ERR_TIMEOUT;
  }
  return FFTK_OK;
}

extern "C" long long fftk_launch_count(fftk_plan p) {
  return p ? p->launches.load(std::memory_order_relaxed) : -1;
}

extern "C" fftk_status fftk_profile_enable(fftk_plan p, int on) {
  if (!p) return FFTK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(p->mu);
  p->prof.clear();
  p->prof.on = on != 0;
  return FFTK_OK;
}

extern "C" fftk_status fftk_profile_read(fftk_plan p, int kind, double* total_ms,
                                         long long* launches) {
  if (!p || kind < 0 || kind >= KK_COUNT || !total_ms || !launches) return FFTK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(p->mu);
  double t = 0.0;
  long long n = 0;
  for (const auto& r : p->prof.recs) {
    if (r.kind != kind) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return from_cuda(e);
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return from_cuda(e);
    t += ms;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  return FFTK_OK;
}

extern "C" int fftk_kernel_kinds(void) { return KK_COUNT; }

extern "C" const char* fftk_kernel_name(int kind) {
  return (kind >= 0 && kind < KK_COUNT) ? kKernelNames[kind] : nullptr;
}
