// Rayleigh-Benard convection through the plan's transforms: the periodic
// cube (FFF basis) and free-slip, isothermal plates (SFF basis).
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "fft_engine.cuh"
#include "ns_common.cuh"

// ------------------------------------------------ Rayleigh-Benard (FFF) ---
// Sec. 2.2, Eqs. (12)-(13), non-dimensional, on the 2 pi-periodic cube with
// gravity along z; state float2 [4][n][n][n/2+1] = (u_x, u_y, u_z, theta).
//   N_u = P[F(u x omega) + theta z],   N_theta = -i k . F(u theta) + u_z,
// evaluated with seven inverse transforms (u, omega, theta) and six forward
// ones (u x omega, u theta) per right-hand side, 13 per stage and 52 per RK4
// step as counted in the paper's Sec. 7: x and y passes restricted to the
// 2/3 set (fft_pruned.cu, fft_sc.cu) and one fused z pass per stage that
// forms the products in registers.
namespace fftk {

struct RBCWork {
  float2* w7 = nullptr;   // 7 spectra: u, omega, theta; then n (u x omega), u theta, in place
  float* r7 = nullptr;    // 7 real fields (3 * 2^m cubes: the unfused right-hand side)
  float2* s1 = nullptr;   // stage state (4 fields)
  float2* acc = nullptr;  // RK4 accumulator (4 fields)
  float2* tab = nullptr;  // integrating factors, hi + lo by integer k^2: E_nu, E_kappa, H_nu, H_kappa
  int tab_len = 0;
  double Ra = -1.0, Pr = -1.0, dt = -1.0;
};

void rbc_free(RBCWork* r) {
  if (!r) return;
  cudaFree(r->w7);
  cudaFree(r->r7);
  cudaFree(r->s1);
  cudaFree(r->acc);
  cudaFree(r->tab);
  delete r;
}

static fftk_status rbc_ensure(fftk_plan p) {
  fftk_status st = ns_ensure(p);
  if (st != FFTK_OK) return st;
  NSWork* s = p->ns;
  std::lock_guard<std::mutex> lk(p->mu);
  if (s->rbc) return FFTK_OK;
  RBCWork* r = new (std::nothrow) RBCWork;
  if (!r) return FFTK_ERR_OOM;
  const NSGeom g = s->g;
  const size_t fb = sizeof(float2) * (size_t)g.M;
  // |k|^2 up to 3 kd^2 on the cube, (2n-1)/3 squared + 2 kd^2 between plates
  const int kxs = (2 * g.n - 1) / 3;
  r->tab_len = kxs * kxs + 2 * g.kd * g.kd + 1;
  cudaError_t e = cudaMalloc(&r->w7, 7 * fb);
  if (e == cudaSuccess) e = cudaMalloc(&r->s1, 4 * fb);
  if (e == cudaSuccess) e = cudaMemset(r->s1, 0, 4 * fb);
  if (e == cudaSuccess) e = cudaMalloc(&r->acc, 4 * fb);
  if (e == cudaSuccess) e = cudaMemset(r->acc, 0, 4 * fb);
  if (e == cudaSuccess) e = cudaMalloc(&r->tab, sizeof(float2) * 4 * (size_t)r->tab_len);
  if (e != cudaSuccess) {
    cudaGetLastError();
    rbc_free(r);
    return e == cudaErrorMemoryAllocation ? FFTK_ERR_OOM : FFTK_ERR_CUDA;
  }
  s->rbc = r;
  return FFTK_OK;
}

static fftk_status rbc_tables(fftk_plan p, double Ra, double Pr, double dt) {
  RBCWork* r = p->ns->rbc;
  if (r->Ra == Ra && r->Pr == Pr && r->dt == dt) return FFTK_OK;
  const double nu = std::sqrt(Pr / Ra), kappa = 1.0 / std::sqrt(Ra * Pr);
  const double coef[4] = {nu * dt, kappa * dt, 0.5 * nu * dt, 0.5 * kappa * dt};
  std::vector<float2> h(4 * (size_t)r->tab_len);
  for (int t = 0; t < 4; ++t)
    for (int k2 = 0; k2 < r->tab_len; ++k2) {
      const double E = std::exp(-coef[t] * (double)k2);
      const float hi = (float)E;
      h[(size_t)t * r->tab_len + k2] = make_float2(hi, (float)(E - (double)hi));
    }
  cudaError_t e = cudaMemcpy(r->tab, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return from_cuda(e);
  r->Ra = Ra;
  r->Pr = Pr;
  r->dt = dt;
  return FFTK_OK;
}

// w7 = (u, i k x u, theta) of the stage input x; the Nyquist derivative is 0
__global__ void k_rbc_prep(const float2* __restrict__ x, float2* __restrict__ w7, NSGeom g) {
  // the kept modes only (the pruned inverse passes read nothing else),
  // k_z fastest so that neighbouring threads touch neighbouring entries
  const long long items = (long long)g.nk * g.nk * g.kc;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % g.kc);
    const long long ab = it / g.kc;
    const int a = dense_to_a((int)(ab / g.nk), g.n, g.kd), b = dense_to_a((int)(ab % g.nk), g.n, g.kd);
    const long long idx = ((long long)a * g.n + b) * g.h1 + c;
    const int ka = kwav(a, g.n), kb = kwav(b, g.n);
    const float kx = (2 * abs(ka) == g.n) ? 0.f : (float)ka, ky = (2 * abs(kb) == g.n) ? 0.f : (float)kb;
    const float kz = (2 * c == g.n) ? 0.f : (float)c;
    const float2 ux = x[idx], uy = x[idx + g.M], uz = x[idx + 2 * g.M];
    w7[idx] = ux;
    w7[idx + g.M] = uy;
    w7[idx + 2 * g.M] = uz;
    w7[idx + 3 * g.M] = csub(mul_i(uz, ky), mul_i(uy, kz));
    w7[idx + 4 * g.M] = csub(mul_i(ux, kz), mul_i(uz, kx));
    w7[idx + 5 * g.M] = csub(mul_i(uy, kx), mul_i(ux, ky));
    w7[idx + 6 * g.M] = x[idx + 3 * g.M];
  }
}

struct RBCUpdate {
  const float2* tab;  // E_nu, E_kappa, H_nu, H_kappa at offsets 0, L, 2L, 3L
  int tab_len;
  float dt;
};

__device__ __forceinline__ float2 mul_pair(float2 v, float2 E) {  // v * (hi + lo), one rounding
  return make_float2(fmaf(v.x, E.x, v.x * E.y), fmaf(v.y, E.x, v.y * E.y));
}

// Every kept mode: N from w7 (n and u theta spectra) and the stage input x,
// then the update of the selected mode (the NS modes, four fields, the
// temperature with its own factors).  Outside the kept set nothing is written.
__global__ void k_rbc_update(const float2* __restrict__ w7, const float2* x, const float2* u0, float2* s1,
                             float2* acc, float2* out, NSGeom g, RBCUpdate upd, int mode) {
  const long long items = (long long)g.nk * g.nk * g.kc;  // the kept modes, k_z fastest
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % g.kc);
    const long long ab = it / g.kc;
    const int a = dense_to_a((int)(ab / g.nk), g.n, g.kd), b = dense_to_a((int)(ab % g.nk), g.n, g.kd);
    const long long idx = ((long long)a * g.n + b) * g.h1 + c;
    const int kx = kwav(a, g.n), ky = kwav(b, g.n), kz = c;
    const int k2 = kx * kx + ky * ky + kz * kz;
    const long long M = g.M;
    float2 nv[4];
    const float2 th = x[idx + 3 * M];
    if (k2 == 0) {
      nv[0] = nv[1] = nv[2] = nv[3] = make_float2(0.f, 0.f);
    } else {
      const float fkx = (float)kx, fky = (float)ky, fkz = (float)kz;
      // n + theta z, then the projection
      float2 px = w7[idx], py = w7[idx + M], pz = cadd(w7[idx + 2 * M], th);
      const float inv = 1.f / (float)k2;
      const float2 kn = make_float2((fkx * px.x + fky * py.x + fkz * pz.x) * inv,
                                    (fkx * px.y + fky * py.y + fkz * pz.y) * inv);
      nv[0] = csub(px, cscale(kn, fkx));
      nv[1] = csub(py, cscale(kn, fky));
      nv[2] = csub(pz, cscale(kn, fkz));
      // -i k . F(u theta) + u_z
      const float2 qx = w7[idx + 3 * M], qy = w7[idx + 4 * M], qz = w7[idx + 5 * M];
      const float2 dv = make_float2(fkx * qx.x + fky * qy.x + fkz * qz.x, fkx * qx.y + fky * qy.y + fkz * qz.y);
      const float2 uz = x[idx + 2 * M];
      nv[3] = make_float2(dv.y + uz.x, -dv.x + uz.y);
    }
    const float dt = upd.dt;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const long long i = idx + f * M;
      const float2 n = nv[f];
      if (mode == NS_RHS) {
        out[i] = n;
        continue;
      }
      const int t = f == 3 ? 1 : 0;
      const float2 E = __ldg(&upd.tab[t * upd.tab_len + k2]);
      const float2 H = __ldg(&upd.tab[(2 + t) * upd.tab_len + k2]);
      if (mode == NS_STAGE1) {
        const float2 v = u0[i];
        out[i] = mul_pair(make_float2(v.x + dt * n.x, v.y + dt * n.y), E);
      } else if (mode == NS_STAGE2) {
        const float2 ea = mul_pair(u0[i], E), b1 = s1[i];
        out[i] = make_float2(0.5f * (ea.x + (b1.x + dt * n.x)), 0.5f * (ea.y + (b1.y + dt * n.y)));
      } else if (mode == NS_RK4_4) {
        const float2 ac = acc[i];
        out[i] = make_float2(fmaf(dt / 6.f, n.x, ac.x), fmaf(dt / 6.f, n.y, ac.y));
      } else {
        const float2 v = u0[i];
        const float2 ea = mul_pair(v, E), ha = mul_pair(v, H), hn = mul_pair(n, H);
        if (mode == NS_RK4_1) {
          const float2 en = mul_pair(n, E);
          acc[i] = make_float2(fmaf(dt / 6.f, en.x, ea.x), fmaf(dt / 6.f, en.y, ea.y));
          out[i] = mul_pair(make_float2(v.x + 0.5f * dt * n.x, v.y + 0.5f * dt * n.y), H);
        } else {
          const float2 ac = acc[i];
          acc[i] = make_float2(fmaf(dt / 3.f, hn.x, ac.x), fmaf(dt / 3.f, hn.y, ac.y));
          out[i] = (mode == NS_RK4_2) ? make_float2(fmaf(0.5f * dt, n.x, ha.x), fmaf(0.5f * dt, n.y, ha.y))
                                      : make_float2(fmaf(dt, hn.x, ea.x), fmaf(dt, hn.y, ea.y));
        }
      }
    }
  }
}

// ---- free-slip plates (SFF): wall-normal axis x on [0, pi], gravity along x.
// u_x and theta are sine series along x (storage index a is k_x = a + 1),
// u_y and u_z cosine series (index a is k_x = a); y and z Fourier.  d_x of a
// sine coefficient s_k is the cosine coefficient k s_k, d_x of a cosine
// coefficient c_k the sine coefficient -k c_k.  Kept: 3 k_x < 2n, 3|k_y| < n,
// 3 k_z < n.  A thread owns the wavenumber triple (k_x = a, k_y, k_z): the
// cosine entry at index a and the sine entry at index a - 1.

// w7 = [u_x, omega_y, omega_z, theta | u_y, u_z, omega_x]: sine group, then
// cosine group (each contiguous, for one batched transform per group)
__global__ void k_rbc_sff_prep(const float2* __restrict__ x, float2* __restrict__ w7, NSGeom g) {
  const long long M = g.M, rowa = (long long)g.n * g.h1;  // one step of the x index
  // the kept modes only (the pruned inverse passes read nothing else; the
  // sine entry of k_x = a is kept with the cosine one, k_x = n never is)
  const int nx = (2 * g.n - 1) / 3 + 1;  // k_x = 0 .. nx - 1 (3 k_x < 2n)
  const long long items = (long long)nx * g.nk * g.kc;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % g.kc);
    const long long ab = it / g.kc;
    const int a = (int)(ab / g.nk), b = dense_to_a((int)(ab % g.nk), g.n, g.kd);
    const long long idx = ((long long)a * g.n + b) * g.h1 + c;
    const int kb = kwav(b, g.n);
    const float ky = (2 * abs(kb) == g.n) ? 0.f : (float)kb, kz = (2 * c == g.n) ? 0.f : (float)c;
    const float2 uy = x[idx + M], uz = x[idx + 2 * M];
    // cosine entries at index a
    w7[idx + 4 * M] = uy;
    w7[idx + 5 * M] = uz;
    w7[idx + 6 * M] = csub(mul_i(uz, ky), mul_i(uy, kz));  // omega_x = d_y u_z - d_z u_y
    // sine entries of k_x = a at index a - 1
    if (a == 0) continue;
    const long long sidx = idx - rowa;
    const float kx = (float)a;
    const float2 ux = x[sidx], th = x[sidx + 3 * M];
    const float2 uyc = uy, uzc = uz;
    w7[sidx] = ux;
    w7[sidx + M] = cadd(mul_i(ux, kz), cscale(uzc, kx));      // omega_y = d_z u_x - d_x u_z
    w7[sidx + 2 * M] = csub(cscale(uyc, -kx), mul_i(ux, ky));  // omega_z = d_x u_y - d_y u_x
    w7[sidx + 3 * M] = th;
  }
}

// the stage update of one field entry i (the modes of ns_mode_update)
__device__ __forceinline__ void rbc_entry_update(long long i, float2 n, float2 E, float2 H, float dt, int mode,
                                                 const float2* u0, const float2* s1, float2* acc, float2* out) {
  if (mode == NS_RHS) {
    out[i] = n;
  } else if (mode == NS_STAGE1) {
    const float2 v = u0[i];
    out[i] = mul_pair(make_float2(v.x + dt * n.x, v.y + dt * n.y), E);
  } else if (mode == NS_STAGE2) {
    const float2 ea = mul_pair(u0[i], E), b1 = s1[i];
    out[i] = make_float2(0.5f * (ea.x + (b1.x + dt * n.x)), 0.5f * (ea.y + (b1.y + dt * n.y)));
  } else if (mode == NS_RK4_4) {
    const float2 ac = acc[i];
    out[i] = make_float2(fmaf(dt / 6.f, n.x, ac.x), fmaf(dt / 6.f, n.y, ac.y));
  } else {
    const float2 v = u0[i];
    const float2 ea = mul_pair(v, E), ha = mul_pair(v, H), hn = mul_pair(n, H);
    if (mode == NS_RK4_1) {
      const float2 en = mul_pair(n, E);
      acc[i] = make_float2(fmaf(dt / 6.f, en.x, ea.x), fmaf(dt / 6.f, en.y, ea.y));
      out[i] = mul_pair(make_float2(v.x + 0.5f * dt * n.x, v.y + 0.5f * dt * n.y), H);
    } else {
      const float2 ac = acc[i];
      acc[i] = make_float2(fmaf(dt / 3.f, hn.x, ac.x), fmaf(dt / 3.f, hn.y, ac.y));
      out[i] = (mode == NS_RK4_2) ? make_float2(fmaf(0.5f * dt, n.x, ha.x), fmaf(0.5f * dt, n.y, ha.y))
                                  : make_float2(fmaf(dt, hn.x, ea.x), fmaf(dt, hn.y, ea.y));
    }
  }
}

// w7 (spectra): [(u x omega)_x, (u_y theta), (u_z theta) in sine | (u x omega)_y,
// (u x omega)_z, (u_x theta) in cosine].  v = u x omega + theta x, minus the
// gradient of the cosine pressure p = -div v / k^2; N_theta = -div(u theta) + u_x.
__global__ void k_rbc_sff_update(const float2* __restrict__ w7, const float2* x, const float2* u0, float2* s1,
                                 float2* acc, float2* out, NSGeom g, RBCUpdate upd, int mode) {
  const long long M = g.M, rowa = (long long)g.n * g.h1;
  const int nx = (2 * g.n - 1) / 3 + 1;  // the kept modes, k_z fastest
  const long long items = (long long)nx * g.nk * g.kc;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % g.kc);
    const long long ab = it / g.kc;
    const int a = (int)(ab / g.nk), b = dense_to_a((int)(ab % g.nk), g.n, g.kd);
    const long long idx = ((long long)a * g.n + b) * g.h1 + c;
    const int ky = kwav(b, g.n), kz = c, kx = a;
    const int k2 = kx * kx + ky * ky + kz * kz;
    const float fkx = (float)kx, fky = (float)ky, fkz = (float)kz;
    const bool has_s = a >= 1;  // the sine entry of k_x = a (index a - 1)
    const long long sidx = idx - rowa;
    // velocity
    float2 vx = make_float2(0.f, 0.f);
    if (has_s) vx = cadd(w7[sidx], x[sidx + 3 * M]);  // (u x omega)_x + theta
    float2 vy = w7[idx + 3 * M], vz = w7[idx + 4 * M];
    // k = 0 (cosine k_x = 0, k_y = k_z = 0): a uniform flow along the plates,
    // with no pressure gradient to remove
    if (k2 != 0) {
      const float inv = 1.f / (float)k2;
      // div v = k_x v_x + i k_y v_y + i k_z v_z (cosine); p = -div / k^2
      const float2 dv = make_float2(fkx * vx.x - fky * vy.y - fkz * vz.y, fkx * vx.y + fky * vy.x + fkz * vz.x);
      const float2 pc = make_float2(-dv.x * inv, -dv.y * inv);
      vy = csub(vy, mul_i(pc, fky));
      vz = csub(vz, mul_i(pc, fkz));
      vx = cadd(vx, cscale(pc, fkx));
    }
    float2 nt = make_float2(0.f, 0.f);
    if (has_s) {
      // -(d_x (u_x theta) + d_y (u_y theta) + d_z (u_z theta)) + u_x
      const float2 cx = w7[idx + 5 * M], sy = w7[sidx + M], sz = w7[sidx + 2 * M];
      const float2 ux = x[sidx];
      const float2 d = csub(cadd(mul_i(sy, fky), mul_i(sz, fkz)), cscale(cx, fkx));
      nt = cadd(make_float2(-d.x, -d.y), ux);
    }
    const float dt = upd.dt;
    const float2 Eu = __ldg(&upd.tab[k2]), Et = __ldg(&upd.tab[upd.tab_len + k2]);
    const float2 Hu = __ldg(&upd.tab[2 * upd.tab_len + k2]), Ht = __ldg(&upd.tab[3 * upd.tab_len + k2]);
    rbc_entry_update(idx + M, vy, Eu, Hu, dt, mode, u0, s1, acc, out);
    rbc_entry_update(idx + 2 * M, vz, Eu, Hu, dt, mode, u0, s1, acc, out);
    if (has_s) {
      rbc_entry_update(sidx, vx, Eu, Hu, dt, mode, u0, s1, acc, out);
      rbc_entry_update(sidx + 3 * M, nt, Et, Ht, dt, mode, u0, s1, acc, out);
    }
  }
}

// ---- fused z pass (both bases: z is Fourier in each) ----------------------
// Per (x, y) line: c2r of u, theta (parked in shared memory) and of the three
// vorticity components (folded into the accumulators of n = u x omega), then
// r2c of n and of u theta.  Reads k_z < kc of the seven input slots, writes
// k_z < kc of the six output slots, in place (every input of a line is read
// before the line's first output is written).  Slot maps: in[7] = u_x, u_y,
// u_z, omega_x, omega_y, omega_z, theta; out[6] = n_x, n_y, n_z, u_x theta,
// u_y theta, u_z theta.
struct RBCSlots {
  int in[7];
  int out[6];
};

template <int N>
struct RZCfg {
  static constexpr int H = N / 2;
  static constexpr int G = H < 8 ? H : 8;
  static constexpr int S = H / G;
  static constexpr int LPC = S >= 128 ? 1 : 128 / S;
  static constexpr int THREADS = LPC * S;
  static constexpr bool WARP = S <= 32;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)LPC * H * 5;  // exchange + 4 parked fields
};

template <int N>
__global__ void __launch_bounds__(RZCfg<N>::THREADS, 3)
    k_rbc_z(float2* w, RBCSlots sl, const float2* __restrict__ tw) {
  constexpr long long H1 = N / 2 + 1, MM = (long long)N * N * H1;
  constexpr int KC = (N - 1) / 3 + 1;
  using C = RZCfg<N>;
  constexpr int H = C::H, G = C::G, S = C::S;
  constexpr int LOGN = Log2<N>::value;
  extern __shared__ float2 smr[];
  const int li = threadIdx.x / S, j = threadIdx.x % S;
  const long long line = (long long)blockIdx.x * C::LPC + li;
  const bool valid = line < (long long)N * N;
  const LineX<C::WARP> xc{smr + li * H};
  float2* park = smr + C::LPC * H + li * 4 * H + j;  // [4][G][S]: u_x, u_y, u_z, theta

  auto c2r = [&](int slot, float2(&U)[G]) {
    const float2* src = w + slot * MM + line * H1;
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
      const float2 O = cmulc(csub(A, Bc), __ldg(&tw[k]));
      U[m] = make_float2(E.x - O.y, E.y + O.x);
    }
    fft_line<H, G, +1, LOGN>(U, j, xc, tw);
  };
  auto r2c = [&](int slot, float2(&U)[G]) {
    fft_line<H, G, -1, LOGN>(U, j, xc, tw);
#pragma unroll
    for (int m = 0; m < G; ++m) xc.st(j + m * S, U[m]);
    xc.sync();
    float2* dst = w + slot * MM + line * H1;
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const int k = j + m * S;
      const float2 Bc = cconj(xc.ld((H - k) & (H - 1)));
      const float2 E = cscale(cadd(U[m], Bc), 0.5f);
      const float2 D = csub(U[m], Bc);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
      if (valid && k < KC) dst[k] = cadd(E, cmul(__ldg(&tw[k]), O));
    }
    xc.sync();
  };
  auto pk = [&](int f, int m) -> float2& { return park[(f * G + m) * S]; };
  {
    float2 U[G];
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      c2r(sl.in[q < 3 ? q : 6], U);
#pragma unroll
      for (int m = 0; m < G; ++m) pk(q, m) = U[m];
    }
  }
  // n = u x omega, two real points per slot
  float2 Nx[G], Ny[G], Nz[G];
  {
    float2 W[G];
    c2r(sl.in[3], W);  // omega_x
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const float2 uy = pk(1, m), uz = pk(2, m);
      Ny[m] = make_float2(uz.x * W[m].x, uz.y * W[m].y);
      Nz[m] = make_float2(-uy.x * W[m].x, -uy.y * W[m].y);
    }
    c2r(sl.in[4], W);  // omega_y
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const float2 ux = pk(0, m), uz = pk(2, m);
      Nx[m] = make_float2(-uz.x * W[m].x, -uz.y * W[m].y);
      Nz[m] = make_float2(fmaf(ux.x, W[m].x, Nz[m].x), fmaf(ux.y, W[m].y, Nz[m].y));
    }
    c2r(sl.in[5], W);  // omega_z
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const float2 ux = pk(0, m), uy = pk(1, m);
      Nx[m] = make_float2(fmaf(uy.x, W[m].x, Nx[m].x), fmaf(uy.y, W[m].y, Nx[m].y));
      Ny[m] = make_float2(fmaf(-ux.x, W[m].x, Ny[m].x), fmaf(-ux.y, W[m].y, Ny[m].y));
    }
  }
  // every input slot of this line has been read: the outputs may overwrite them
  __syncthreads();
  r2c(sl.out[0], Nx);
  r2c(sl.out[1], Ny);
  r2c(sl.out[2], Nz);
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    float2 P[G];
#pragma unroll
    for (int m = 0; m < G; ++m) {
      const float2 ui = pk(i, m), th = pk(3, m);
      P[m] = make_float2(ui.x * th.x, ui.y * th.y);
    }
    r2c(sl.out[3 + i], P);
  }
}

template <int N>
static cudaError_t rbc_z_n(fftk_plan p, float2* w, const RBCSlots& sl, cudaStream_t st) {
  using C = RZCfg<N>;
  static PerDevice once;
  const cudaError_t attr_err = once.run([](int) {
    return cudaFuncSetAttribute(k_rbc_z<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const long long lines = (long long)N * N;
  LaunchScope ls(p, KK_RBC_Z, st);
  k_rbc_z<N><<<(unsigned)((lines + C::LPC - 1) / C::LPC), C::THREADS, C::SMEM, st>>>(w, sl, twiddles(p, N));
  return cudaGetLastError();
}

static cudaError_t rbc_z(fftk_plan p, float2* w, const RBCSlots& sl, cudaStream_t st) {
  switch (p->nz) {
#define CASE(n) \
  case n:       \
    return rbc_z_n<n>(p, w, sl, st);
    CASE(8) CASE(16) CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

// Pointwise products of the unfused right-hand side, in place over the seven
// real fields (u, omega, theta): n = u x omega into 0..2, u theta into 3..5.
__global__ void k_rbc_products(float* __restrict__ r, long long R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += (long long)gridDim.x * blockDim.x) {
    const float ux = r[i], uy = r[i + R], uz = r[i + 2 * R];
    const float wx = r[i + 3 * R], wy = r[i + 4 * R], wz = r[i + 5 * R];
    const float th = r[i + 6 * R];
    r[i] = fmaf(uy, wz, -uz * wy);
    r[i + R] = fmaf(uz, wx, -ux * wz);
    r[i + 2 * R] = fmaf(ux, wy, -uy * wx);
    r[i + 3 * R] = ux * th;
    r[i + 4 * R] = uy * th;
    r[i + 5 * R] = uz * th;
  }
}

// The periodic right-hand side on 3 * 2^m cubes, through the plan's full
// transforms (one radix-3 step per 1D pass): (u, omega, theta) on the kept
// modes into a cleared workspace, inverse transforms of the seven fields,
// the products in real space, forward transforms of the six products, then
// the update of the fused path (which reads only the kept modes).
static cudaError_t rbc_stage_unfused(fftk_plan p, const float2* x, const float2* u0, float2* out,
                                     const RBCUpdate& upd, int mode, cudaStream_t st) {
  NSWork* s = p->ns;
  RBCWork* r = s->rbc;
  const NSGeom g = s->g;
  const long long R = (long long)g.n * g.n * g.n;
  if (!r->r7) {
    cudaError_t ea = cudaMalloc(&r->r7, sizeof(float) * 7 * (size_t)R);
    if (ea != cudaSuccess) {
      cudaGetLastError();
      r->r7 = nullptr;
      return ea;
    }
  }
  const unsigned grid = 152 * 8;
  float2* w = r->w7;
  cudaError_t e = cudaMemsetAsync(w, 0, sizeof(float2) * 7 * (size_t)g.M, st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_RBC_PREP, st);
    k_rbc_prep<<<grid, 256, 0, st>>>(x, w, g);
  }
  e = c2r_overwrite(p, w, r->r7, 7, st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_rbc_products<<<grid, 256, 0, st>>>(r->r7, R);
  }
  e = r2c_scaled(p, r->r7, w, 6, (float)(1.0 / (double)R), st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_RBC_UPDATE, st);
    k_rbc_update<<<grid, 256, 0, st>>>(w, x, u0, r->s1, r->acc, out, g, upd, mode);
  }
  return cudaGetLastError();
}

// One right-hand side of the stage input x and the update of `mode`:
// spectral preparation, inverse x and y passes restricted to the kept set,
// the fused z pass (products in registers), forward y and x passes, update.
static cudaError_t rbc_stage(fftk_plan p, const float2* x, const float2* u0, float2* out, const RBCUpdate& upd,
                             int mode, int basis, cudaStream_t st) {
  NSWork* s = p->ns;
  RBCWork* r = s->rbc;
  const NSGeom g = s->g;
  const long long R = (long long)g.n * g.n * g.n;
  const float scale = (float)(1.0 / (double)R);
  const unsigned grid = 152 * 8;
  float2* w = r->w7;
  cudaError_t e = cudaSuccess;
  if (basis == TARANG_RBC_SFF) {
    // w7 = [u_x, omega_y, omega_z, theta | u_y, u_z, omega_x]: sine group, cosine group
    {
      LaunchScope ls(p, KK_RBC_PREP, st);
      k_rbc_sff_prep<<<grid, 256, 0, st>>>(x, w, g);
    }
    e = launch_scpass_pruned(p, true, +1, w, w, 4, 1.f, st);
    if (e == cudaSuccess) e = launch_scpass_pruned(p, false, +1, w + 4 * g.M, w + 4 * g.M, 3, 1.f, st);
    if (e == cudaSuccess) e = launch_pruned_y(p, +1, w, w, 7, 1.f, st);
    // products: [(u x omega)_x, u_y theta, u_z theta | (u x omega)_y, (u x omega)_z, u_x theta]
    const RBCSlots sl{{0, 4, 5, 6, 1, 2, 3}, {0, 3, 4, 5, 1, 2}};
    if (e == cudaSuccess) e = rbc_z(p, w, sl, st);
    if (e == cudaSuccess) e = launch_pruned_y(p, -1, w, w, 6, 1.f, st);
    if (e == cudaSuccess) e = launch_scpass_pruned(p, true, -1, w, w, 3, scale, st);
    if (e == cudaSuccess) e = launch_scpass_pruned(p, false, -1, w + 3 * g.M, w + 3 * g.M, 3, scale, st);
    if (e != cudaSuccess) return e;
    {
      LaunchScope ls(p, KK_RBC_UPDATE, st);
      k_rbc_sff_update<<<grid, 256, 0, st>>>(w, x, u0, r->s1, r->acc, out, g, upd, mode);
    }
    return cudaGetLastError();
  }
  if (!is_pow2(g.n)) return rbc_stage_unfused(p, x, u0, out, upd, mode, st);
  // w7 = [u_x, u_y, u_z, omega_x, omega_y, omega_z, theta] -> [n_x, n_y, n_z, u_x theta, ...]
  {
    LaunchScope ls(p, KK_RBC_PREP, st);
    k_rbc_prep<<<grid, 256, 0, st>>>(x, w, g);
  }
  e = launch_pruned_x(p, +1, w, w, 7, 1.f, st);
  if (e == cudaSuccess) e = launch_pruned_y(p, +1, w, w, 7, 1.f, st);
  const RBCSlots sl{{0, 1, 2, 3, 4, 5, 6}, {0, 1, 2, 3, 4, 5}};
  if (e == cudaSuccess) e = rbc_z(p, w, sl, st);
  if (e == cudaSuccess) e = launch_pruned_y(p, -1, w, w, 6, 1.f, st);
  if (e == cudaSuccess) e = launch_pruned_x(p, -1, w, w, 6, scale, st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_RBC_UPDATE, st);
    k_rbc_update<<<grid, 256, 0, st>>>(w, x, u0, r->s1, r->acc, out, g, upd, mode);
  }
  return cudaGetLastError();
}

// Cubes as for the Navier-Stokes solver (powers of two in [8, 1024], 3 * 2^m
// in [12, 768]); the plates (SFF) need power-of-two axes for their sine and
// cosine transforms.
static fftk_status rbc_check(fftk_plan p, const void* state, int basis = TARANG_RBC_FFF) {
  if (!p || !state || misaligned16(state)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (!ns_size_ok(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (basis == TARANG_RBC_SFF && !is_pow2(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  return FFTK_OK;
}

}  // namespace fftk

using namespace fftk;

extern "C" fftk_status tarang_rbc_rhs(fftk_plan p, int basis, const void* state, void* out, void* cuda_stream) {
  if (basis != TARANG_RBC_FFF && basis != TARANG_RBC_SFF) return FFTK_ERR_INVALID_ARG;
  fftk_status s = rbc_check(p, state, basis);
  if (s != FFTK_OK) return s;
  if (!out || out == state || misaligned16(out)) return FFTK_ERR_INVALID_ARG;
  s = rbc_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const NSGeom g = p->ns->g;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float2) * 4 * (size_t)g.M, st);
  RBCUpdate upd{p->ns->rbc->tab, p->ns->rbc->tab_len, 0.f};
  if (e == cudaSuccess)
    e = rbc_stage(p, static_cast<const float2*>(state), static_cast<const float2*>(state),
                  static_cast<float2*>(out), upd, NS_RHS, basis, st);
  return from_cuda(e);
}

extern "C" fftk_status tarang_rbc_step(fftk_plan p, void* state, const tarang_rbc_params* prm, int nsteps,
                                       void* cuda_stream) {
  fftk_status s = rbc_check(p, state, prm ? prm->basis : TARANG_RBC_FFF);
  if (s != FFTK_OK) return s;
  if (!prm || nsteps < 0 || !(prm->Ra > 0.0) || !(prm->Pr > 0.0) || !(prm->dt > 0.0) || !std::isfinite(prm->Ra) ||
      !std::isfinite(prm->Pr) || !std::isfinite(prm->dt) || (prm->scheme != TARANG_RK2 && prm->scheme != TARANG_RK4) ||
      (prm->basis != TARANG_RBC_FFF && prm->basis != TARANG_RBC_SFF))
    return FFTK_ERR_INVALID_ARG;
  s = rbc_ensure(p);
  if (s != FFTK_OK) return s;
  s = rbc_tables(p, prm->Ra, prm->Pr, prm->dt);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  RBCWork* r = p->ns->rbc;
  float2* u = static_cast<float2*>(state);
  const RBCUpdate upd{r->tab, r->tab_len, (float)prm->dt};
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < nsteps && e == cudaSuccess; ++it) {
    if (prm->scheme == TARANG_RK2) {
      e = rbc_stage(p, u, u, r->s1, upd, NS_STAGE1, prm->basis, st);
      if (e == cudaSuccess) e = rbc_stage(p, r->s1, u, u, upd, NS_STAGE2, prm->basis, st);
    } else {
      for (int stage = 0; stage < 4 && e == cudaSuccess; ++stage)
        e = rbc_stage(p, stage == 0 ? u : r->s1, u, stage == 3 ? u : r->s1, upd, NS_RK4_1 + stage, prm->basis,
                      st);
    }
  }
  return from_cuda(e);
}

// Kinetic and thermal energy transfer of the periodic convection (the flux
// computation of the paper's Sec. 7, Pi_u(k) and Pi_theta(k)): with N the
// right-hand side of tarang_rbc_rhs,
//   T_u(K) = sum_shell w Re(conj(u) . N_u) - sum_shell w Re(conj(u_z) theta),
//   T_theta(K) = sum_shell w Re(conj(theta) N_theta) - sum_shell w Re(conj(theta) u_z)
// (the buoyancy and conduction-source exchanges removed, advection left),
// Pi(K) = -sum_{K' <= K} T(K').
extern "C" fftk_status tarang_rbc_transfer(fftk_plan p, const void* state, double* out_host, void* cuda_stream) {
  fftk_status s = rbc_check(p, state);
  if (s != FFTK_OK) return s;
  if (!out_host) return FFTK_ERR_INVALID_ARG;
  s = rbc_ensure(p);
  if (s != FFTK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NSWork* w = p->ns;
  RBCWork* r = w->rbc;
  const NSGeom g = w->g;
  const float2* x = static_cast<const float2*>(state);
  float2* nh = r->acc;  // free between steps
  cudaError_t e = cudaMemsetAsync(nh, 0, sizeof(float2) * 4 * (size_t)g.M, st);
  const RBCUpdate upd{r->tab, r->tab_len, 0.f};
  if (e == cudaSuccess) e = rbc_stage(p, x, x, nh, upd, NS_RHS, TARANG_RBC_FFF, st);
  const int nb = w->kmax + 1, width = 2 + nb;
  // three reductions: u . N_u (3 components), u_z theta, theta N_theta
  const float2* ua[3] = {x, x + 2 * g.M, x + 3 * g.M};
  const float2* na[3] = {nh, x + 3 * g.M, nh + 3 * g.M};
  const int nfs[3] = {3, 1, 1};
  std::vector<double> h(3 * (size_t)width);
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
    e = diag_launch(p, ua[q], na[q], 0.0, st, nfs[q]);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data() + (size_t)q * width, w->dout, sizeof(double) * width, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return from_cuda(e);
  // out: sum T_u, T_u(0..kmax), Pi_u(0..kmax), sum T_theta, T_theta(...), Pi_theta(...)
  bool finite = true;
  for (int fld = 0; fld < 2; ++fld) {
    double* o = out_host + (size_t)fld * (1 + 2 * nb);
    const double* adv = h.data() + (size_t)(fld == 0 ? 0 : 2) * width;
    const double* buoy = h.data() + (size_t)width;
    double pi = 0.0, tot = 0.0;
    for (int K = 0; K < nb; ++K) {
      const double t = adv[2 + K] - buoy[2 + K];
      o[1 + K] = t;
      pi -= t;
      o[1 + nb + K] = pi;
      tot += t;
    }
    o[0] = tot;
    finite = finite && std::isfinite(tot);
  }
  return finite ? FFTK_OK : FFTK_ERR_NONFINITE;
}
