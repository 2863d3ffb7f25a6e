// Shared by the Tarang solver's translation units: ns.cu (the fused
// Navier-Stokes passes and the time steppers), ns_diag.cu (diagnostics and
// the scale-by-scale energy transfer) and rbc.cu (convection).  Geometry of
// the 2/3-truncated spectrum, the update modes and the plan-owned workspace.
#pragma once

#include <cstdint>

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

enum NSMode : int {
  NS_RHS = 0,
  NS_STAGE1 = 1,
  NS_STAGE2 = 2,
  NS_RK4_1 = 3,
  NS_RK4_2 = 4,
  NS_RK4_3 = 5,
  NS_RK4_4 = 6
};

constexpr int DIAG_WARPS = 8;
constexpr size_t kNoAllocScratchDoubles = 262144;  // 2 MiB of partials for tarang_diag_noalloc

// ------------------------------------------------------------ workspace ----
struct RBCWork;  // Rayleigh-Benard scratch, below

struct NSWork {
  NSGeom g;
  float2* w = nullptr;     // 6 fields
  float2* w2 = nullptr;    // 6 more fields: the fused passes alternate between w and w2
  float2* u1 = nullptr;    // 3 fields
  float2* etab = nullptr;  // exp(-nu k^2 dt) as hi + lo, k^2 in [0, 3 kd^2]
  int etab_len = 0;
  double etab_nu = -1.0, etab_dt = -1.0;
  double* ef = nullptr;    // forced energy
  double* part = nullptr;  // diag partials
  double* dout = nullptr;  // diag result (device)
  double* hout = nullptr;  // diag result (pinned host)
  fftk_sgs_work* sgs = nullptr;  // learned-closure scratch
  float* r6 = nullptr;     // 6 real fields (shell-to-shell transfer)
  float* r3 = nullptr;     // 3 real fields (shell-to-shell transfer: the advection term)
  float2* acc = nullptr;   // 3 fields (RK4 accumulator)
  RBCWork* rbc = nullptr;  // Rayleigh-Benard scratch (allocated on first use)
  double* sout = nullptr;  // per-giver shell sums of the shell-to-shell transfer
  int sout_rows = 0;
  int kmax = 0;
  int diag_smem = 0;
};

int ns_kmax(int n);
// Cubes the solver accepts: n a power of two in [8, 1024] (the fused passes),
// or n = 3 * 2^m in [12, 768] (the paper's 768^3 runs; the right-hand side
// runs through the plan's transforms with the radix-3 step, unfused).
inline bool ns_size_ok(int n) {
  if (n >= 8 && n <= 1024 && (n & (n - 1)) == 0) return true;
  return n >= 12 && n <= 768 && n % 3 == 0 && ((n / 3) & (n / 3 - 1)) == 0;
}
NSGeom make_geom(int n);
fftk_status ns_ensure(fftk_plan p);
fftk_status ns_check(fftk_plan p, const tarang_params* prm, bool need_dt);
void rbc_free(RBCWork* r);

// diagnostics (ns_diag.cu)
int diag_blocks(int width);
cudaError_t diag_attr();
cudaError_t diag_launch(fftk_plan p, const float2* u, const float2* nh, double nu, cudaStream_t st, int nf = 3);

inline bool misaligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0; }

}  // namespace fftk
