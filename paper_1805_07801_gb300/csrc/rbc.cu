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
// evaluated through the plan's transforms: seven inverse (u, omega, theta),
// six forward (u x omega, u theta) per right-hand side, 13 per stage and 52
// per RK4 step as counted in the paper's Sec. 7.
namespace fftk {

struct RBCWork {
  float2* w7 = nullptr;   // spectra: u, omega, theta; then n (u x omega), u theta
  float* r7 = nullptr;    // the same seven fields in real space
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
  const size_t fb = sizeof(float2) * (size_t)g.M, rb = sizeof(float) * (size_t)g.n * g.n * g.n;
  // |k|^2 up to 3 kd^2 on the cube, (2n-1)/3 squared + 2 kd^2 between plates
  const int kxs = (2 * g.n - 1) / 3;
  r->tab_len = kxs * kxs + 2 * g.kd * g.kd + 1;
  cudaError_t e = cudaMalloc(&r->w7, 7 * fb);
  if (e == cudaSuccess) e = cudaMalloc(&r->r7, 7 * rb);
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
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    // the pruned inverse passes read only the kept modes
    if (!(kept_xy(a, g.n, g.kd) && kept_xy(b, g.n, g.kd) && c < g.kc)) continue;
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

// r7[0..2] = u x omega, r7[3..5] = u theta (in place, point by point)
__global__ void k_rbc_products(float* __restrict__ r7, long long R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R;
       i += (long long)gridDim.x * blockDim.x) {
    const float ux = r7[i], uy = r7[R + i], uz = r7[2 * R + i];
    const float wx = r7[3 * R + i], wy = r7[4 * R + i], wz = r7[5 * R + i], th = r7[6 * R + i];
    r7[i] = uy * wz - uz * wy;
    r7[R + i] = uz * wx - ux * wz;
    r7[2 * R + i] = ux * wy - uy * wx;
    r7[3 * R + i] = ux * th;
    r7[4 * R + i] = uy * th;
    r7[5 * R + i] = uz * th;
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
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    if (!(kept_xy(a, g.n, g.kd) && kept_xy(b, g.n, g.kd) && c < g.kc)) continue;
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

__device__ __forceinline__ bool sff_kept(int kx, int b, int c, const NSGeom& g) {
  return 3 * kx < 2 * g.n && kept_xy(b, g.n, g.kd) && c < g.kc;
}

// w7 = [u_x, omega_y, omega_z, theta | u_y, u_z, omega_x]: sine group, then
// cosine group (each contiguous, for one batched transform per group)
__global__ void k_rbc_sff_prep(const float2* __restrict__ x, float2* __restrict__ w7, NSGeom g) {
  const long long M = g.M, rowa = (long long)g.n * g.h1;  // one step of the x index
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    // the pruned inverse passes read only the kept modes (the sine entry of
    // k_x = a is kept with the cosine one; k_x = n never is)
    if (!sff_kept(a, b, c, g)) continue;
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

// r7 = [u_x, omega_y, omega_z, theta, u_y, u_z, omega_x] -> in place
// [(u x omega)_x, u_y theta, u_z theta | (u x omega)_y, (u x omega)_z, u_x theta]:
// the sine-parity products first, then the cosine-parity ones
__global__ void k_rbc_sff_products(float* __restrict__ r7, long long R) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R;
       i += (long long)gridDim.x * blockDim.x) {
    const float ux = r7[i], wy = r7[R + i], wz = r7[2 * R + i], th = r7[3 * R + i];
    const float uy = r7[4 * R + i], uz = r7[5 * R + i], wx = r7[6 * R + i];
    r7[i] = uy * wz - uz * wy;
    r7[R + i] = uy * th;
    r7[2 * R + i] = uz * th;
    r7[3 * R + i] = uz * wx - ux * wz;
    r7[4 * R + i] = ux * wy - uy * wx;
    r7[5 * R + i] = ux * th;
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
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.h1);
    const long long ab = idx / g.h1;
    const int b = (int)(ab % g.n), a = (int)(ab / g.n);
    if (!sff_kept(a, b, c, g)) continue;
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

// One right-hand side of the stage input x and the update of `mode`.
static cudaError_t rbc_stage(fftk_plan p, const float2* x, const float2* u0, float2* out, const RBCUpdate& upd,
                             int mode, int basis, cudaStream_t st) {
  NSWork* s = p->ns;
  RBCWork* r = s->rbc;
  const NSGeom g = s->g;
  const long long R = (long long)g.n * g.n * g.n;
  const unsigned grid = 152 * 8;
  if (basis == TARANG_RBC_SFF) {
    {
      LaunchScope ls(p, KK_AUX, st);
      k_rbc_sff_prep<<<grid, 256, 0, st>>>(x, r->w7, g);
    }
    // inverse transforms restricted to the kept set, in place in w7: the sine
    // group (4 fields), then the cosine group (3)
    cudaError_t e = cudaSuccess;
    for (int grp = 0; grp < 2 && e == cudaSuccess; ++grp) {
      const int nf = grp == 0 ? 4 : 3;
      float2* w = r->w7 + (grp == 0 ? 0 : 4 * g.M);
      e = launch_scpass_pruned(p, grp == 0, +1, w, w, nf, 1.f, st);
      if (e == cudaSuccess) e = launch_pruned_y(p, +1, w, w, nf, 1.f, st);
      if (e == cudaSuccess) e = launch_z_c2r(p, w, r->r7 + (grp == 0 ? 0 : 4 * R), (long long)nf * g.n * g.n, st, g.kc);
    }
    if (e != cudaSuccess) return e;
    {
      LaunchScope ls(p, KK_AUX, st);
      k_rbc_sff_products<<<grid, 256, 0, st>>>(r->r7, R);
    }
    // forward transforms of the sine-parity products, then the cosine-parity ones
    const float sc = (float)(1.0 / (double)R);
    for (int grp = 0; grp < 2 && e == cudaSuccess; ++grp) {
      float2* w = r->w7 + (grp == 0 ? 0 : 3 * g.M);
      e = launch_z_r2c(p, r->r7 + (grp == 0 ? 0 : 3 * R), w, 3LL * g.n * g.n, 1.f, st, g.kc);
      if (e == cudaSuccess) e = launch_pruned_y(p, -1, w, w, 3, 1.f, st);
      if (e == cudaSuccess) e = launch_scpass_pruned(p, grp == 0, -1, w, w, 3, sc, st);
    }
    if (e != cudaSuccess) return e;
    {
      LaunchScope ls(p, KK_AUX, st);
      k_rbc_sff_update<<<grid, 256, 0, st>>>(r->w7, x, u0, r->s1, r->acc, out, g, upd, mode);
    }
    return cudaGetLastError();
  }
  {
    LaunchScope ls(p, KK_AUX, st);
    k_rbc_prep<<<grid, 256, 0, st>>>(x, r->w7, g);
  }
  // inverse transforms restricted to the 2/3 set, in place in w7, then the z c2r
  cudaError_t e = launch_pruned_x(p, +1, r->w7, r->w7, 7, 1.f, st);
  if (e == cudaSuccess) e = launch_pruned_y(p, +1, r->w7, r->w7, 7, 1.f, st);
  if (e == cudaSuccess) e = launch_z_c2r(p, r->w7, r->r7, 7LL * g.n * g.n, st, g.kc);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_rbc_products<<<grid, 256, 0, st>>>(r->r7, R);
  }
  e = launch_z_r2c(p, r->r7, r->w7, 6LL * g.n * g.n, 1.f, st, g.kc);
  if (e == cudaSuccess) e = launch_pruned_y(p, -1, r->w7, r->w7, 6, 1.f, st);
  if (e == cudaSuccess) e = launch_pruned_x(p, -1, r->w7, r->w7, 6, (float)(1.0 / ((double)R)), st);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_rbc_update<<<grid, 256, 0, st>>>(r->w7, x, u0, r->s1, r->acc, out, g, upd, mode);
  }
  return cudaGetLastError();
}

static fftk_status rbc_check(fftk_plan p, const void* state) {
  if (!p || !state || misaligned16(state)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz) return FFTK_ERR_UNSUPPORTED_SIZE;
  if (p->nx < 8 || p->nx > 1024 || !is_pow2(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  return FFTK_OK;
}

}  // namespace fftk

using namespace fftk;

extern "C" fftk_status tarang_rbc_rhs(fftk_plan p, int basis, const void* state, void* out, void* cuda_stream) {
  fftk_status s = rbc_check(p, state);
  if (s != FFTK_OK) return s;
  if (!out || out == state || misaligned16(out)) return FFTK_ERR_INVALID_ARG;
  if (basis != TARANG_RBC_FFF && basis != TARANG_RBC_SFF) return FFTK_ERR_INVALID_ARG;
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
  fftk_status s = rbc_check(p, state);
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
