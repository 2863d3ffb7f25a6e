// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/fftk.h"

namespace fftk {

// Kernel kinds, for launch counting and event-based profiling.
enum KernelKind : int {
  KK_Z_R2C = 0,
  KK_Y_FWD,
  KK_X_FWD,
  KK_X_INV,
  KK_Y_INV,
  KK_Z_C2R,
  KK_NS_INVX,
  KK_NS_INVY,
  KK_NS_Z,
  KK_NS_FWDY,
  KK_NS_FWDX,
  KK_NS_REDUCE,
  KK_AUX,
  KK_SC_FWD,
  KK_SC_INV,
  KK_RBC_PREP,
  KK_RBC_Z,
  KK_RBC_UPDATE,
  KK_COUNT
};
extern const char* const kKernelNames[KK_COUNT];

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  size_t next = 0;
  cudaEvent_t take();
  void clear();
  ~Profiler();
};

struct NSWork;  // solver workspace, ns.cu

}  // namespace fftk

struct fftk_plan_s {
  int nx, ny, nz, hz;  // hz = nz/2 + 1
  fftk_dtype dtype;
  int device;
  int twlog;                 // LT = 2^twlog = max(nx, ny, nz)
  float2* d_tw_alloc = nullptr;  // per-stage twiddle tables (kStageTwiddles entries), then the pyramid
  float2* d_tw = nullptr;    // twiddle tables: at offset L (L = 1, 2, 4, ..., 4 LT), exp(-2 pi i m / L), m < L
  float2* d_tw3 = nullptr;   // the same for L = 3, 6, 12, ... up to the largest 3 * 2^m dimension
  __half* d_dft16 = nullptr; // split-FP16 DFT-16 operands (FFTK_R32_SPLIT16): forward, inverse
  int* d_err = nullptr;      // device error word (bounded waits that expired)
  // c2r workspace (one complex field per batch element)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  // solver state
  fftk::NSWork* ns = nullptr;
  // bookkeeping
  std::atomic<long long> launches{0};
  fftk::Profiler prof;
  std::mutex mu;
};

namespace fftk {

// The table of size L = 3 * 2^m (a dimension of the plan or a divisor of one).
inline const float2* twiddles3(const fftk_plan_s* p, int L) { return p->d_tw3 + L; }

// The plan's twiddle table of size L (a power of two <= 4 LT): exp(-2 pi i m / L), m < L.
// Tables beyond LT serve the quarter-wave factors of the sine/cosine passes.
inline const float2* twiddles(const fftk_plan_s* p, int L) { return p->d_tw + L; }

// One-time set-up for each device.  Kernel attributes (the dynamic
// shared-memory limit) and occupancy figures belong to a function on the
// device that is current when they are set or queried, so a process that
// drives several devices repeats them on each.  run(f) calls f(dev) once per
// device (the current one) and returns that status on every later call.
constexpr int kMaxDevices = 64;
struct PerDevice {
  std::mutex mu;
  bool done[kMaxDevices] = {};
  cudaError_t err[kMaxDevices] = {};
  template <class F>
  cudaError_t run(F&& f, int* dev_out = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (dev_out) *dev_out = dev;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
      err[dev] = f(dev);
      done[dev] = true;
    }
    return err[dev];
  }
};

// Launch bracketing: counts the launch and records profiling events.
struct LaunchScope {
  fftk_plan p;
  int kind;
  cudaStream_t st;
  cudaEvent_t b = nullptr;
  LaunchScope(fftk_plan p_, int kind_, cudaStream_t st_);
  ~LaunchScope();
};

// ---------------------------------------------------------- FFT passes -----
// z pass, real -> half complex, lines of nz reals -> nz/2+1 complex (scale applied).
cudaError_t launch_z_r2c(fftk_plan p, const float* in, float2* out, long long nlines, float scale,
                         cudaStream_t st);
// z pass, half complex -> real (unnormalised); Im of the k=0 and k=nz/2 terms ignored.
cudaError_t launch_z_c2r(fftk_plan p, const float2* in, float* out, long long nlines,
                         cudaStream_t st);
// strided c2c pass: array [P][L][Q], transform along L (element stride Q),
// in may equal out.  sign = -1 forward, +1 inverse; output multiplied by scale.
cudaError_t launch_scpass(fftk_plan p, int L, bool sine, int dir, const float2* in, float2* out, long long P,
                          long long Q, float scale, int kind, cudaStream_t st);
cudaError_t launch_scz(fftk_plan p, bool sine, int dir, const float* in, float* out, long long nlines,
                       float scale, int kind, cudaStream_t st);
// lines of length 3 * 2^m (fft_radix3.cu)
cudaError_t launch_cpass3(fftk_plan p, int L, int sign, const float2* in, float2* out, long long B, long long Q,
                          float scale, int kind, cudaStream_t st);
cudaError_t launch_z3(fftk_plan p, bool fwd, const void* in, void* out, long long nlines, float scale,
                      cudaStream_t st);
bool is_pow2_or_3x(long long v);
// strided passes restricted to the 2/3-rule set of an n^3 cube (fft_pruned.cu):
// the inverse x pass reads the kept k_x rows of the kept (k_y, k_z) columns
// and writes whole lines; the inverse y pass reads kept k_y rows of the kept
// k_z columns of every x; the forward passes mirror them and write only kept
// rows.  B batch elements of [n][n][n/2+1].
cudaError_t launch_pruned_x(fftk_plan p, int sign, const float2* in, float2* out, long long B, float scale,
                            cudaStream_t st);
cudaError_t launch_pruned_y(fftk_plan p, int sign, const float2* in, float2* out, long long B, float scale,
                            cudaStream_t st);
// the sine/cosine x pass restricted to the same set (3 k_x < 2n on the x axis)
cudaError_t launch_scpass_pruned(fftk_plan p, bool sine, int dir, const float2* in, float2* out, long long B,
                                 float scale, cudaStream_t st);
cudaError_t launch_cpass(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P,
                         long long Q, float scale, int kind, cudaStream_t st);

// split-FP16 tensor-core strided pass (FFTK_R32_SPLIT16), L in {256, 512, 1024, 2048}
bool cpass_tc_supported(int L);
// strided c2c pass with TMA tile loads for lines of 512 points: false
// (nothing launched) where the layout does not allow TMA (row stride Q odd,
// base not 16-byte aligned); otherwise true with the launch status in *e
bool launch_cpass_tma(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P, long long Q,
                      float scale, int kind, cudaStream_t st, cudaError_t* e);
// the split-FP16 pass restricted to the 2/3-rule set of an n^3 spectrum
// (axis 0: x lines, 1: y lines; n of 256, 512 or 1024), as launch_pruned_x/y
cudaError_t launch_cpass_tc_pruned(fftk_plan p, int axis, int sign, const float2* in, float2* out, long long B,
                                   float scale, int kind, cudaStream_t st);
cudaError_t launch_cpass_tc(fftk_plan p, int L, int sign, const float2* in, float2* out, long long P,
                            long long Q, float scale, int kind, cudaStream_t st);
cudaError_t upload_dft16_operands(fftk_plan p);
// The plan's forward transform of B real fields without argument checks
// (scale applied in the last pass), and its inverse of B spectra whose x and y
// passes run in place (the spectra are overwritten) before the z pass into out.
// (scratch: optional array of the spectrum's size; given, the strided passes
// run out of place through it)
cudaError_t r2c_scaled(fftk_plan p, const float* in, float2* out, long long B, float scale, cudaStream_t st,
                       float2* scratch = nullptr);
cudaError_t c2r_overwrite(fftk_plan p, float2* spec, float* out, long long B, cudaStream_t st,
                          float2* scratch = nullptr);
// A tiled FP32 tensor map for TMA loads: dims[0] innermost (in floats),
// strides[i] the byte stride of dimension i + 1 (a multiple of 16), box the
// box extents (box[0] * 4 bytes a multiple of 16); out-of-range elements of a
// box read as zero.  False (nothing encoded) where the driver entry point is
// missing or a rule is broken.
bool encode_f32_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                    const uint32_t* box);
}  // namespace fftk

struct fftk_sgs_work;
namespace fftk {
// subgrid force of a learned model for the state u: points *out at P[-i k_j tau_hat_ij]
cudaError_t sgs_term(fftk_plan p, fftk_sgs_work** w, const float2* u, const tarang_sgs_model* model,
                     cudaStream_t st, const float2** out);
void sgs_free(fftk_sgs_work* w);

bool is_pow2(long long v);
int ilog2(long long v);

}  // namespace fftk
