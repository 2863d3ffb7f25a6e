// Learned subgrid-stress closure (not in the paper; the task's closure
// workload): closure data from a resolved field, the MLP training kernels,
// and the per-point inference used inside the right-hand side.
//
// Reading of "5 invariants in, 6 stresses out": the network predicts tau in
// the eigenframe of the filtered strain rate S (eigenvalues descending, each
// eigenvector's largest-magnitude component positive), tau = Q tau' Q^T,
// which makes the closure covariant under rotations.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft_engine.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace fftk {

fftk_status from_cuda(cudaError_t e);

// ------------------------------------------------------------ box filter ---
// One CTA per coarse (X, Y) column: the factor^2 fine z lines of the column
// are read with consecutive threads on consecutive z; every thread sums its
// z positions over the column in FP64, then groups of `factor` lanes reduce
// over z with shuffles (fixed order) to the coarse cells.
__global__ void k_box_filter(const float* __restrict__ u, int n, int factor, double* __restrict__ out9) {
  const int m = n / factor;
  const int X = blockIdx.x / m, Y = blockIdx.x % m;
  const long long R = (long long)n * n * n, Mc = (long long)m * m * m;
  for (int z0 = 0; z0 < n; z0 += blockDim.x) {
    const int z = z0 + threadIdx.x;
    double s[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) s[q] = 0.0;
    if (z < n) {
      for (int a = 0; a < factor; ++a)
        for (int b = 0; b < factor; ++b) {
          const long long idx = ((long long)(X * factor + a) * n + (Y * factor + b)) * n + z;
          const double ux = u[idx], uy = u[R + idx], uz = u[2 * R + idx];
          s[0] += ux;
          s[1] += uy;
          s[2] += uz;
          s[3] += ux * ux;
          s[4] += uy * uy;
          s[5] += uz * uz;
          s[6] += ux * uy;
          s[7] += ux * uz;
          s[8] += uy * uz;
        }
    }
    // reduce over the `factor` consecutive z of each coarse cell
    for (int o = 1; o < factor; o <<= 1)
#pragma unroll
      for (int q = 0; q < 9; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (z < n && (z % factor) == 0) {
      const double inv = 1.0 / ((double)factor * factor * factor);
      const long long cell = ((long long)X * m + Y) * m + z / factor;
#pragma unroll
      for (int q = 0; q < 9; ++q) out9[q * Mc + cell] = s[q] * inv;
    }
  }
}

// ubar_i and tau_ij = <u_i u_j> - ubar_i ubar_j from the block means
__global__ void k_box_finish(const double* __restrict__ m9, long long Mc, float* __restrict__ ubar,
                             float* __restrict__ tau) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < Mc;
       c += (long long)gridDim.x * blockDim.x) {
    const double ux = m9[c], uy = m9[Mc + c], uz = m9[2 * Mc + c];
    ubar[c] = (float)ux;
    ubar[Mc + c] = (float)uy;
    ubar[2 * Mc + c] = (float)uz;
    tau[c] = (float)(m9[3 * Mc + c] - ux * ux);
    tau[Mc + c] = (float)(m9[4 * Mc + c] - uy * uy);
    tau[2 * Mc + c] = (float)(m9[5 * Mc + c] - uz * uz);
    tau[3 * Mc + c] = (float)(m9[6 * Mc + c] - ux * uy);
    tau[4 * Mc + c] = (float)(m9[7 * Mc + c] - ux * uz);
    tau[5 * Mc + c] = (float)(m9[8 * Mc + c] - uy * uz);
  }
}

// ---------------------------------------------------------- point algebra --
__device__ __forceinline__ bool kept_mode(int a, int b, int c, int n) {
  const int kd = (n - 1) / 3;
  return (a <= kd || a >= n - kd) && (b <= kd || b >= n - kd) && c <= kd;
}
__device__ __forceinline__ int kw(int a, int n) { return 2 * a < n ? a : a - n; }
__device__ __forceinline__ int kdv(int k, int n) { return 2 * (k < 0 ? -k : k) == n ? 0 : k; }

// spectra of the 9 gradient components i k_j u_i from a 2/3-truncated copy of u
// zero every mode outside the 2/3 set (3|k_i| < m on every axis) of nf
// spectra [nf][m][m][m/2+1]
__global__ void k_truncate(float2* __restrict__ f, int m, int nf) {
  const int h1 = m / 2 + 1;
  const long long M = (long long)m * m * h1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)nf * M;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i % M;
    const int c = (int)(r % h1);
    const long long ab = r / h1;
    const int b = (int)(ab % m), a = (int)(ab / m);
    const int ka = 2 * a < m ? a : a - m, kb = 2 * b < m ? b : b - m;
    if (!(3 * abs(ka) < m && 3 * abs(kb) < m && 3 * c < m)) f[i] = make_float2(0.f, 0.f);
  }
}

// P_p = tau_p + ubar_i ubar_j - ut_i ut_j for the six pairs (i, j) of
// xx, yy, zz, xy, xz, yz (FP32 products of FP32 fields)
__global__ void k_les_products(const float* __restrict__ ubar, const float* __restrict__ tau,
                               const float* __restrict__ ut, float* __restrict__ P, long long R) {
  const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < R; x += (long long)gridDim.x * blockDim.x) {
    float ub[3], tt[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ub[q] = ubar[q * R + x];
      tt[q] = ut[q * R + x];
    }
#pragma unroll
    for (int p = 0; p < 6; ++p)
      P[p * R + x] = fmaf(ub[pi[p]], ub[pj[p]], tau[p * R + x]) - tt[pi[p]] * tt[pj[p]];
  }
}

__global__ void k_grad_spectra(const float2* __restrict__ uh, float2* __restrict__ gh, int n) {
  const int h1 = n / 2 + 1;
  const long long M = (long long)n * n * h1;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % h1);
    const int b = (int)((idx / h1) % n), a = (int)(idx / ((long long)h1 * n));
    const bool keep = kept_mode(a, b, c, n);
    const float k[3] = {(float)kdv(kw(a, n), n), (float)kdv(kw(b, n), n), (float)kdv(c, n)};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float2 v = keep ? uh[i * M + idx] : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j) gh[(i * 3 + j) * M + idx] = make_float2(-k[j] * v.y, k[j] * v.x);
    }
  }
}

__device__ __forceinline__ void m3mul(const float* a, const float* b, float* c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c[i * 3 + j] = a[i * 3] * b[j] + a[i * 3 + 1] * b[3 + j] + a[i * 3 + 2] * b[6 + j];
}

// invariants tr S^2, tr R^2, tr S^3, tr R^2 S, tr R^2 S^2 and the symmetric S
__device__ __forceinline__ void point_invariants(const float A[9], float S[9], float inv[5]) {
  float R[9], S2[9], R2[9], t[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S[i * 3 + j] = 0.5f * (A[i * 3 + j] + A[j * 3 + i]);
      R[i * 3 + j] = 0.5f * (A[i * 3 + j] - A[j * 3 + i]);
    }
  m3mul(S, S, S2);
  m3mul(R, R, R2);
  inv[0] = S2[0] + S2[4] + S2[8];
  inv[1] = R2[0] + R2[4] + R2[8];
  m3mul(S2, S, t);
  inv[2] = t[0] + t[4] + t[8];
  m3mul(R2, S, t);
  inv[3] = t[0] + t[4] + t[8];
  m3mul(R2, S2, t);
  inv[4] = t[0] + t[4] + t[8];
}

// cyclic Jacobi (fixed sweep cap), eigenvalues descending, eigenvector
// columns Q[row*3+k] with their largest-magnitude component positive
__device__ void point_eig3(const float S[9], float Q[9]) {
  float a[9], v[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
#pragma unroll
  for (int i = 0; i < 9; ++i) a[i] = S[i];
  for (int sweep = 0; sweep < 12; ++sweep) {
    // converged to FP32 resolution: off-diagonal mass below 1e-7 of the diagonal's
    if (fabsf(a[1]) + fabsf(a[2]) + fabsf(a[5]) <= 1e-7f * (fabsf(a[0]) + fabsf(a[4]) + fabsf(a[8]))) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
      const float apq = a[p * 3 + q];
      if (apq == 0.f) continue;
      const float theta = (a[q * 3 + q] - a[p * 3 + p]) / (2.f * apq);
      const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(1.f + theta * theta));
      const float c = rsqrtf(1.f + t * t), s = t * c;
      // a <- J^T a J, v <- v J  (J: identity with c, s / -s, c in rows and columns p, q)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float akp = a[k * 3 + p], akq = a[k * 3 + q];
        a[k * 3 + p] = c * akp - s * akq;
        a[k * 3 + q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float apk = a[p * 3 + k], aqk = a[q * 3 + k];
        a[p * 3 + k] = c * apk - s * aqk;
        a[q * 3 + k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float vkp = v[k * 3 + p], vkq = v[k * 3 + q];
        v[k * 3 + p] = c * vkp - s * vkq;
        v[k * 3 + q] = s * vkp + c * vkq;
      }
    }
  }
  int o0 = 0, o1 = 1, o2 = 2, tmp;
  if (a[o1 * 4] > a[o0 * 4]) { tmp = o0; o0 = o1; o1 = tmp; }
  if (a[o2 * 4] > a[o0 * 4]) { tmp = o0; o0 = o2; o2 = tmp; }
  if (a[o2 * 4] > a[o1 * 4]) { tmp = o1; o1 = o2; o2 = tmp; }
  const int ord[3] = {o0, o1, o2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int src = ord[k];
    int big = 0;
    if (fabsf(v[3 + src]) > fabsf(v[src])) big = 1;
    if (fabsf(v[6 + src]) > fabsf(v[big * 3 + src])) big = 2;
    const float sg = v[big * 3 + src] < 0.f ? -1.f : 1.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) Q[i * 3 + k] = sg * v[i * 3 + src];
  }
}

// symmetric 3x3 from the 6 components (xx, yy, zz, xy, xz, yz) and back
__device__ __forceinline__ void sym_from6(const float t6[6], float T[9]) {
  T[0] = t6[0]; T[4] = t6[1]; T[8] = t6[2];
  T[1] = T[3] = t6[3];
  T[2] = T[6] = t6[4];
  T[5] = T[7] = t6[5];
}
__device__ __forceinline__ void sym_to6(const float T[9], float t6[6]) {
  t6[0] = T[0]; t6[1] = T[4]; t6[2] = T[8];
  t6[3] = T[1]; t6[4] = T[2]; t6[5] = T[5];
}

// features at each coarse point: invariants, frame Q, and tau' = Q^T tau Q
__global__ void k_closure_features(const float* __restrict__ A9, const float* __restrict__ tau6, long long Mc,
                                   float* __restrict__ inv5, float* __restrict__ Q9,
                                   float* __restrict__ taup6) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < Mc;
       c += (long long)gridDim.x * blockDim.x) {
    float A[9], S[9], inv[5], Q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) A[i] = A9[i * Mc + c];
    point_invariants(A, S, inv);
    point_eig3(S, Q);
#pragma unroll
    for (int i = 0; i < 5; ++i) inv5[i * Mc + c] = inv[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) Q9[i * Mc + c] = Q[i];
    if (tau6 && taup6) {
      float t6[6], T[9], QT[9], tmp[9], out[9];
#pragma unroll
      for (int i = 0; i < 6; ++i) t6[i] = tau6[i * Mc + c];
      sym_from6(t6, T);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) QT[i * 3 + j] = Q[j * 3 + i];
      m3mul(QT, T, tmp);
      m3mul(tmp, Q, out);
      sym_to6(out, t6);
#pragma unroll
      for (int i = 0; i < 6; ++i) taup6[i * Mc + c] = t6[i];
    }
  }
}

// ------------------------------------------------------------------- MLP ---
// 5 -> 64 -> 64 -> 64 -> 6, tanh on the hidden layers; parameters (FP32):
// W1[64][5] b1 W2[64][64] b2 W3[64][64] b3 W4[6][64] b4 (9094 values).
// Each layer's input (x, h1, h2, h3) is rounded to bfloat16; products and
// sums are FP32.
constexpr int kNP = 9094;
constexpr int kChunk = 128;   // samples per CTA
constexpr int kAStride = kChunk + 1;
__device__ __constant__ int kDims[5] = {5, 64, 64, 64, 6};
__device__ __constant__ int kWOff[4] = {0, 384, 4544, 8704};
__device__ __constant__ int kBOff[4] = {320, 4480, 8640, 9088};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// a layer input as the network defines it (BF16), or unrounded in the FP32
// test mode that isolates the kernels' arithmetic from the BF16 rounding
template <bool BF16>
__device__ __forceinline__ float act_round(float x) {
  return BF16 ? bf16r(x) : x;
}

struct MLPSmem {
  float w[kNP];
  float act0[5 * kAStride];        // input of layer 0, [feature][sample]
  float act123[3][64 * kAStride];  // inputs of layers 1..3
  float d0[64 * kAStride];         // deltas
  float d1[64 * kAStride];
  __device__ __forceinline__ float* act(int l) { return l == 0 ? act0 : act123[l - 1]; }
};

// forward of the chunk; y written for samples < nb; returns nothing
template <bool BF16>
__device__ void mlp_chunk_forward(MLPSmem& s, const float* __restrict__ x, int nb, int base, float* y6) {
  const int b = threadIdx.x;
  if (b < kChunk) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
      s.act(0)[i * kAStride + b] = b < nb ? act_round<BF16>(x[(long long)(base + b) * 5 + i]) : 0.f;
  }
  __syncthreads();
  for (int l = 0; l < 4; ++l) {
    const int din = kDims[l], dout = kDims[l + 1];
    const float* W = s.w + kWOff[l];
    const float* bias = s.w + kBOff[l];
    for (int o = 0; o < dout; ++o) {
      float z = bias[o];
      for (int i = 0; i < din; ++i) z = fmaf(W[o * din + i], s.act(l)[i * kAStride + b], z);
      if (l < 3)
        s.act(l + 1)[o * kAStride + b] = act_round<BF16>(tanhf(z));
      else
        y6[o] = z;
    }
    __syncthreads();
  }
}

// one CTA: forward + backward of 128 samples; writes its gradient partial and
// its loss partial (sum of squared errors).  BF16: layer inputs rounded to
// bfloat16 (the network's definition); false in the FP32 test mode.
template <bool BF16>
__global__ void __launch_bounds__(kChunk) k_mlp_grad(const float* __restrict__ params, const float* __restrict__ x,
                                                     const float* __restrict__ t, int B, float* __restrict__ part,
                                                     double* __restrict__ loss_part) {
  extern __shared__ float smem_mlp[];
  MLPSmem& s = *reinterpret_cast<MLPSmem*>(smem_mlp);
  const int b = threadIdx.x;
  const int base = blockIdx.x * kChunk;
  const int nb = min(kChunk, B - base);
  for (int i = b; i < kNP; i += kChunk) s.w[i] = params[i];
  __syncthreads();
  float y[6];
  mlp_chunk_forward<BF16>(s, x, nb, base, y);
  // output error: dL/dz4 = 2 (y - t) / (6 B)
  __shared__ double lsum[kChunk];
  double l2 = 0.0;
  const float g = 2.f / (6.f * (float)B);
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    float e = 0.f;
    if (b < nb) e = y[o] - t[(long long)(base + b) * 6 + o];
    l2 += (double)e * e;
    s.d0[o * kAStride + b] = e * g;
  }
  lsum[b] = l2;
  __syncthreads();
  float* dcur = s.d0;
  float* dnext = s.d1;
  float* out = part + (long long)blockIdx.x * kNP;
  for (int l = 3; l >= 0; --l) {
    const int din = kDims[l], dout = kDims[l + 1];
    // weight and bias gradients of layer l: sums over the chunk's samples
    for (int pr = b; pr < dout * din; pr += kChunk) {
      const int o = pr / din, i = pr % din;
      float acc = 0.f;
      for (int k = 0; k < kChunk; ++k) acc = fmaf(dcur[o * kAStride + k], s.act(l)[i * kAStride + k], acc);
      out[kWOff[l] + pr] = acc;
    }
    for (int o = b; o < dout; o += kChunk) {
      float acc = 0.f;
      for (int k = 0; k < kChunk; ++k) acc += dcur[o * kAStride + k];
      out[kBOff[l] + o] = acc;
    }
    if (l > 0) {
      const float* W = s.w + kWOff[l];
      for (int i = 0; i < din; ++i) {
        float acc = 0.f;
        for (int o = 0; o < dout; ++o) acc = fmaf(W[o * din + i], dcur[o * kAStride + b], acc);
        const float a = s.act(l)[i * kAStride + b];
        dnext[i * kAStride + b] = acc * (1.f - a * a);
      }
    }
    __syncthreads();
    float* t2 = dcur;
    dcur = dnext;
    dnext = t2;
  }
  if (b == 0) {
    double acc = 0.0;
    for (int k = 0; k < kChunk; ++k) acc += lsum[k];
    loss_part[blockIdx.x] = acc;
  }
}

// the forward pass alone on the CUDA cores (128 samples per CTA), the
// arithmetic of k_mlp_grad's forward: y[B][6]
template <bool BF16>
__global__ void __launch_bounds__(kChunk) k_mlp_forward_cc(const float* __restrict__ params,
                                                           const float* __restrict__ x, float* __restrict__ y, int B) {
  extern __shared__ float smem_mlp[];
  MLPSmem& s = *reinterpret_cast<MLPSmem*>(smem_mlp);
  const int b = threadIdx.x;
  const int base = blockIdx.x * kChunk;
  const int nb = min(kChunk, B - base);
  for (int i = b; i < kNP; i += kChunk) s.w[i] = params[i];
  __syncthreads();
  float y6[6];
  mlp_chunk_forward<BF16>(s, x, nb, base, y6);
  if (b < nb) {
#pragma unroll
    for (int o = 0; o < 6; ++o) y[(long long)(base + b) * 6 + o] = y6[o];
  }
}

// fixed-order sums of the per-CTA partials
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad,
                             const double* __restrict__ loss_part, double* __restrict__ loss, double inv_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNP) {
    double acc = 0.0;
    for (int k = 0; k < nblk; ++k) acc += part[(long long)k * kNP + i];
    grad[i] = (float)acc;
  }
  if (i == 0 && loss) {
    double acc = 0.0;
    for (int k = 0; k < nblk; ++k) acc += loss_part[k];
    *loss = acc * inv_count;
  }
}

// Adam (Kingma and Ba 2015) with bias corrections; step counted from 1
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Constants of the learned model (normalisation of inputs and outputs).
struct SGSConst {
  float in_shift[5], in_scale[5], out_scale[6];
};

// --------------------------------------------- MLP on the tensor cores ---
// Inference of the 5-64-64-64-6 network for 256 points per CTA pass (two
// M = 128 blocks, one point per thread).  Every layer is one tcgen05 MMA chain
// D = H W_hi^T + H W_lo^T: H is the layer's input in BF16 (the rounding the
// network is defined with), W = W_hi + W_lo its FP32 weights split into two
// BF16 parts (16 significant bits), FP32 accumulation in TMEM.  Bias, tanh and
// the BF16 rounding of the next layer's input run on the CUDA cores (tanh as
// a rational function accurate to the BF16 rounding, tanh_to_bf16); the input
// x is padded to K = 16, the output layer to N = 16 (6 used).  Operands are
// K-major without swizzle (B rows = output units).
namespace mlptc {
constexpr int kThreads = 256;
constexpr int kBlocks = 2;
constexpr int kW1 = 64 * 16 * 2;  // bytes of one BF16 part of W1 as B [64 x 16]
constexpr int kW2 = 64 * 64 * 2;  // W2, W3 as B [64 x 64]
constexpr int kW4 = 16 * 64 * 2;  // W4 as B [16 x 64]
constexpr int kX = 128 * 16 * 2;  // one block of inputs as A [128 x 16]
constexpr int kH = 128 * 64 * 2;  // one block of a hidden layer as A [128 x 64]
constexpr int oW1 = 0, oW2 = oW1 + 2 * kW1, oW3 = oW2 + 2 * kW2, oW4 = oW3 + 2 * kW2;
constexpr int oBias = oW4 + 2 * kW4;  // b1, b2, b3 (64 each), b4 (6): FP32
constexpr int oX = oBias + 1024;
constexpr int oH = oX + kBlocks * kX;
constexpr int oBar = oH + kBlocks * kH;
constexpr int kSmem = 1024 + oBar + 64;
constexpr int kCols = 128;  // TMEM: 64 FP32 columns per block
constexpr uint32_t kIdN64 = tcg::idesc_f16(128, 64, true);
constexpr uint32_t kIdN16 = tcg::idesc_f16(128, 16, true);

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// tanh x for a value that is rounded to BF16 next: the convergent of Lambert's
// continued fraction tanh x = x / (1 + x^2 / (3 + x^2 / (5 + ...))) through the
// term 17, x P(y) / Q(y) with y = x^2,
//   P = 34459425 + 4729725 y + 135135 y^2 + 990 y^3 + y^4,
//   Q = 34459425 + 16216200 y + 945945 y^2 + 13860 y^3 + 45 y^4
// (both divided by 34459425 below); relative error below 3e-7 in FP32 for
// |x| < 3.5.  For |x| >= 3.5 the BF16 rounding of tanh x is exactly +-1.
__device__ __forceinline__ float tanh_to_bf16(float x) {
  const float y = x * x;
  const float p = fmaf(fmaf(fmaf(fmaf(1.f / 34459425.f, y, 2.f / 69615.f), y, 1.f / 255.f), y, 7.f / 51.f), y, 1.f);
  const float q = fmaf(fmaf(fmaf(fmaf(1.f / 765765.f, y, 4.f / 9945.f), y, 7.f / 255.f), y, 8.f / 17.f), y, 1.f);
  return fabsf(x) >= 3.5f ? copysignf(1.f, x) : x * __fdividef(p, q);
}

__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, int off, float w) {
  const __nv_bfloat16 h = __float2bfloat16_rn(w);
  const __nv_bfloat16 l = __float2bfloat16_rn(w - __bfloat162float(h));
  *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
}

// weights as BF16 hi/lo B operands and biases, from the FP32 parameters
__device__ void load_weights(unsigned char* base, const float* __restrict__ params) {
  for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
    const int o = e >> 4, i = e & 15;
    store_split(base + oW1, base + oW1 + kW1, tcg::kmajor_off<16>(o, i), i < 5 ? params[o * 5 + i] : 0.f);
  }
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int off = tcg::kmajor_off<64>(e >> 6, e & 63);
    store_split(base + oW2, base + oW2 + kW2, off, params[384 + e]);
    store_split(base + oW3, base + oW3 + kW2, off, params[4544 + e]);
  }
  for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
    const int o = e >> 6, i = e & 63;
    store_split(base + oW4, base + oW4 + kW4, tcg::kmajor_off<64>(o, i), o < 6 ? params[8704 + o * 64 + i] : 0.f);
  }
  float* bias = reinterpret_cast<float*>(base + oBias);
  for (int e = threadIdx.x; e < 198; e += blockDim.x)
    bias[e] = e < 64 ? params[320 + e] : e < 128 ? params[4480 + e - 64] : e < 192 ? params[8640 + e - 128]
                                                                                  : params[9088 + e - 192];
}

// the network input of thread t's point (row t & 127 of block t >> 7), rounded to BF16
__device__ __forceinline__ void write_x(unsigned char* base, int t, const float x[5]) {
  unsigned char* X = base + oX + (t >> 7) * kX;
  const int r = t & 127;
  *reinterpret_cast<uint4*>(X + tcg::kmajor_off<16>(r, 0)) =
      make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], 0.f), 0u);
  *reinterpret_cast<uint4*>(X + tcg::kmajor_off<16>(r, 8)) = make_uint4(0u, 0u, 0u, 0u);
}

// the four layers for the CTA's 256 points (after write_x by every thread);
// y = this thread's 6 outputs.  False if an MMA wait expired (uniform over the CTA).
__device__ bool forward(unsigned char* base, uint32_t tmem, uint64_t* bar, uint32_t& phase, float y[6]) {
  const int t = threadIdx.x, warp = t >> 5, blk = t >> 7, r = t & 127;
  const uint32_t row_addr = tmem + (((uint32_t)(warp & 3) * 32u) << 16) + 64u * (uint32_t)blk;
  const uint32_t sb = tcg::su32(base);
  const float* bias = reinterpret_cast<const float*>(base + oBias);
  unsigned char* H = base + oH + blk * kH;
#pragma unroll 1
  for (int l = 0; l < 4; ++l) {
    tcg::fence_smem_async();
    tcg::fence_before_sync();
    __syncthreads();
    tcg::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int b = 0; b < kBlocks; ++b) {
        const uint32_t d = tmem + 64u * b;
        if (l == 0) {
          const uint32_t a = sb + oX + b * kX;
          tcg::mma_f16(d, tcg::desc(a, 128, 256), tcg::desc(sb + oW1, 128, 256), kIdN64, 0);
          tcg::mma_f16(d, tcg::desc(a, 128, 256), tcg::desc(sb + oW1 + kW1, 128, 256), kIdN64, 1);
        } else {
          const uint32_t a = sb + oH + b * kH;
          const uint32_t whi = sb + (l == 1 ? oW2 : l == 2 ? oW3 : oW4);
          const uint32_t wlo = whi + (l == 3 ? kW4 : kW2);
          const uint32_t id = l == 3 ? kIdN16 : kIdN64;
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            tcg::mma_f16(d, tcg::desc(a + 256 * s, 128, 1024), tcg::desc(whi + 256 * s, 128, 1024), id, s > 0);
            tcg::mma_f16(d, tcg::desc(a + 256 * s, 128, 1024), tcg::desc(wlo + 256 * s, 128, 1024), id, 1);
          }
        }
      }
      tcg::commit(bar);
    }
    bool ok = true;
    if (t == 0) {
      ok = tcg::mbar_wait(bar, phase);
      tcg::fence_after_sync();
      tcg::fence_before_sync();
    }
    phase ^= 1;
    const bool all = __syncthreads_and(ok) != 0;
    tcg::fence_after_sync();
    if (!all) return false;
    if (l < 3) {
      // next layer's input, over this layer's (whose MMAs have completed)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float d[32];
        tcg::ld32(row_addr + 32u * hh, d);
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          const float* bl = bias + 64 * l + 32 * hh + j;
          pk[j / 2] = pack_bf16(tanh_to_bf16(d[j] + bl[0]), tanh_to_bf16(d[j + 1] + bl[1]));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(H + tcg::kmajor_off<64>(r, 32 * hh + 8 * q)) =
              make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
      }
    } else {
      float d[8];
      tcg::ld8(row_addr, d);
#pragma unroll
      for (int o = 0; o < 6; ++o) y[o] = d[o] + bias[192 + o];
    }
  }
  return true;
}

__device__ __forceinline__ unsigned char* aligned_base(unsigned char* raw) {
  return raw + ((1024 - (tcg::su32(raw) & 1023)) & 1023);
}

// CTA setup: weights, TMEM, mbarrier
__device__ __forceinline__ uint32_t setup(unsigned char* base, const float* __restrict__ params) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + oBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  load_weights(base, params);
  if ((threadIdx.x >> 5) == 0) tcg::tmem_alloc(tslot, kCols);
  if (threadIdx.x == 0) tcg::mbar_init(bar);
  tcg::fence_smem_async();
  tcg::fence_before_sync();
  __syncthreads();
  tcg::fence_after_sync();
  return *tslot;
}

// CTA teardown; on failure flags `err` and lets the pending MMAs drain (bounded)
__device__ __forceinline__ void finish(unsigned char* base, uint32_t tmem, uint32_t phase, bool failed, int* err) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + oBar);
  if (failed && threadIdx.x == 0) {
    atomicOr(err, 1);
    tcg::mbar_wait(bar, phase ^ 1);
  }
  tcg::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tcg::tmem_dealloc(tmem, kCols);
}
}  // namespace mlptc

// Fused SGS inference with the network on the tensor cores: per point the
// gradient A -> invariants and strain eigenframe -> normalised input -> MLP
// -> tau' -> tau = Q tau' Q^T.  Writes tau[6][n^3].
__global__ void __launch_bounds__(mlptc::kThreads, 2)
    k_sgs_pointwise_tc(const float* __restrict__ A9, long long R, const float* __restrict__ params, SGSConst cst,
                       float* __restrict__ tau6, int* err) {
  extern __shared__ __align__(1024) unsigned char smraw_tc[];
  unsigned char* base = mlptc::aligned_base(smraw_tc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + mlptc::oBar);
  const uint32_t tmem = mlptc::setup(base, params);
  const int t = threadIdx.x;
  uint32_t phase = 0;
  bool failed = false;
  for (long long c0 = (long long)blockIdx.x * mlptc::kThreads; c0 < R; c0 += (long long)gridDim.x * mlptc::kThreads) {
    const long long c = c0 + t;
    const bool valid = c < R;
    float A[9], S[9], inv[5], Q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) A[i] = valid ? A9[i * R + c] : 0.f;
    point_invariants(A, S, inv);
    point_eig3(S, Q);
    float x[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) x[i] = (inv[i] - cst.in_shift[i]) * cst.in_scale[i];
    mlptc::write_x(base, t, x);
    float t6[6];
    if (!mlptc::forward(base, tmem, bar, phase, t6)) {
      failed = true;
      break;
    }
    if (valid) {
#pragma unroll
      for (int o = 0; o < 6; ++o) t6[o] *= cst.out_scale[o];
      float T[9], tmp[9], out[9], QT[9];
      sym_from6(t6, T);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) QT[i * 3 + j] = Q[j * 3 + i];
      m3mul(Q, T, tmp);
      m3mul(tmp, QT, out);
      sym_to6(out, t6);
#pragma unroll
      for (int i = 0; i < 6; ++i) tau6[i * R + c] = t6[i];
    }
  }
  mlptc::finish(base, tmem, phase, failed, err);
}

// Plain inference y[B][6] = MLP(x[B][5]) with the network on the tensor cores.
__global__ void __launch_bounds__(mlptc::kThreads, 2)
    k_mlp_forward_tc(const float* __restrict__ params, const float* __restrict__ x, float* __restrict__ y,
                     long long B, int* err) {
  extern __shared__ __align__(1024) unsigned char smraw_tc[];
  unsigned char* base = mlptc::aligned_base(smraw_tc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + mlptc::oBar);
  const uint32_t tmem = mlptc::setup(base, params);
  const int t = threadIdx.x;
  uint32_t phase = 0;
  bool failed = false;
  for (long long c0 = (long long)blockIdx.x * mlptc::kThreads; c0 < B; c0 += (long long)gridDim.x * mlptc::kThreads) {
    const long long c = c0 + t;
    const bool valid = c < B;
    float xi[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) xi[i] = valid ? x[c * 5 + i] : 0.f;
    mlptc::write_x(base, t, xi);
    float out[6];
    if (!mlptc::forward(base, tmem, bar, phase, out)) {
      failed = true;
      break;
    }
    if (valid)
#pragma unroll
      for (int o = 0; o < 6; ++o) y[c * 6 + o] = out[o];
  }
  mlptc::finish(base, tmem, phase, failed, err);
}

// SGS force s_i = -i k_j tau_hat_ij on the 2/3 set, projected; written to s (3 fields)
__global__ void k_sgs_divergence(const float2* __restrict__ th, float2* __restrict__ s, int n) {
  const int h1 = n / 2 + 1;
  const long long M = (long long)n * n * h1;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % h1);
    const int b = (int)((idx / h1) % n), a = (int)(idx / ((long long)h1 * n));
    float2 f[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const float kx = (float)kw(a, n), ky = (float)kw(b, n), kz = (float)c;
    const float k2 = kx * kx + ky * ky + kz * kz;
    if (kept_mode(a, b, c, n) && k2 > 0.f) {
      const float k[3] = {kx, ky, kz};
      const int pid[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float2 v = th[pid[i][j] * M + idx];
          acc.x += k[j] * v.x;
          acc.y += k[j] * v.y;
        }
        f[i] = make_float2(acc.y, -acc.x);  // -i * acc
      }
      const float2 kf = make_float2((kx * f[0].x + ky * f[1].x + kz * f[2].x) / k2,
                                    (kx * f[0].y + ky * f[1].y + kz * f[2].y) / k2);
      f[0] = csub(f[0], cscale(kf, kx));
      f[1] = csub(f[1], cscale(kf, ky));
      f[2] = csub(f[2], cscale(kf, kz));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i * M + idx] = f[i];
  }
}

// ------------------------------------------------------------ host side ----
static int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)(b < 152 * 16 ? b : 152 * 16);
}

static size_t mlp_smem() { return sizeof(MLPSmem); }

static cudaError_t mlp_attrs() {
  static PerDevice once;
  return once.run([](int) {
    cudaError_t err = cudaFuncSetAttribute(k_mlp_grad<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)mlp_smem());
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_mlp_grad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem());
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_mlp_forward_cc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_smem());
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_mlp_forward_cc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_smem());
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, mlptc::kSmem);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_sgs_pointwise_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, mlptc::kSmem);
    return err;
  });
}

// persistent grid of the tensor-core inference kernels: two CTAs per SM
static int mlptc_grid(long long points) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long need = (points + mlptc::kThreads - 1) / mlptc::kThreads;
  const long long cap = 2LL * sms;
  return (int)(need < cap ? need : cap);
}

}  // namespace fftk

struct tarang_mlp_s {
  int max_batch = 0;
  int* err = nullptr;           // device word: a tensor-core wait expired
  float* part = nullptr;        // [blocks][9094]
  double* loss_part = nullptr;  // [blocks]
  float* grad = nullptr;        // [9094]
};

struct fftk_sgs_work {
  int n = 0;
  float* A = nullptr;       // [9][n^3]
  float* tau = nullptr;     // [6][n^3]
  float2* gh = nullptr;     // [9][M]
  float2* th = nullptr;     // [6][M]
  float2* s = nullptr;      // [3][M]
};

using namespace fftk;

static bool mis16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

extern "C" fftk_status tarang_box_filter(fftk_plan p, const void* uhat, int factor, float* ubar, float* tau,
                                         void* cuda_stream) {
  if (!p || !uhat || !ubar || !tau || mis16(uhat)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz) return FFTK_ERR_UNSUPPORTED_SIZE;
  const int n = p->nx;
  if (factor < 1 || factor > 32 || (factor & (factor - 1)) || n % factor || n < 32)
    return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const long long R = (long long)n * n * n;
  const int m = n / factor;
  const long long Mc = (long long)m * m * m;
  float* ureal = nullptr;
  double* m9 = nullptr;
  cudaError_t e = cudaMalloc(&ureal, sizeof(float) * 3 * (size_t)R);
  if (e == cudaSuccess) e = cudaMalloc(&m9, sizeof(double) * 9 * (size_t)Mc);
  if (e != cudaSuccess) {
    cudaFree(ureal);
    cudaFree(m9);
    cudaGetLastError();
    return FFTK_ERR_OOM;
  }
  fftk_status s = fftk_c2r(p, uhat, ureal, 3, cuda_stream);
  if (s == FFTK_OK) {
    {
      LaunchScope ls(p, KK_AUX, st);
      const int threads = n < 256 ? n : 256;
      k_box_filter<<<m * m, threads, 0, st>>>(ureal, n, factor, m9);
    }
    {
      LaunchScope ls(p, KK_AUX, st);
      k_box_finish<<<grid_for(Mc, 256), 256, 0, st>>>(m9, Mc, ubar, tau);
    }
    e = cudaStreamSynchronize(st);
    s = from_cuda(e == cudaSuccess ? cudaGetLastError() : e);
  }
  cudaFree(ureal);
  cudaFree(m9);
  return s;
}

extern "C" fftk_status tarang_closure_features(fftk_plan p, const float* ubar, const float* tau, float* inv,
                                               float* frame, float* tau_frame, void* cuda_stream) {
  if (!p || !ubar || !inv || !frame || mis16(ubar) || ((tau == nullptr) != (tau_frame == nullptr)))
    return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || !is_pow2(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  const int n = p->nx;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const long long R = (long long)n * n * n, M = (long long)n * n * (n / 2 + 1);
  float2* uh = nullptr;
  float2* gh = nullptr;
  float* A = nullptr;
  cudaError_t e = cudaMalloc(&uh, sizeof(float2) * 3 * (size_t)M);
  if (e == cudaSuccess) e = cudaMalloc(&gh, sizeof(float2) * 9 * (size_t)M);
  if (e == cudaSuccess) e = cudaMalloc(&A, sizeof(float) * 9 * (size_t)R);
  fftk_status s = e == cudaSuccess ? FFTK_OK : FFTK_ERR_OOM;
  if (s == FFTK_OK) s = fftk_r2c(p, ubar, uh, 3, cuda_stream);
  if (s == FFTK_OK) {
    LaunchScope ls(p, KK_AUX, st);
    k_grad_spectra<<<grid_for(M, 256), 256, 0, st>>>(uh, gh, n);
  }
  if (s == FFTK_OK) s = fftk_c2r(p, gh, A, 9, cuda_stream);
  if (s == FFTK_OK) {
    LaunchScope ls(p, KK_AUX, st);
    k_closure_features<<<grid_for(R, 128), 128, 0, st>>>(A, tau, R, inv, frame, tau_frame);
    e = cudaStreamSynchronize(st);
    s = from_cuda(e == cudaSuccess ? cudaGetLastError() : e);
  }
  cudaGetLastError();
  cudaFree(uh);
  cudaFree(gh);
  cudaFree(A);
  return s;
}

extern "C" fftk_status tarang_les_stress(fftk_plan p, const float* ubar, const float* tau, float* out,
                                         void* cuda_stream) {
  if (!p || !ubar || !tau || !out || mis16(ubar) || mis16(tau) || mis16(out)) return FFTK_ERR_INVALID_ARG;
  if (p->nx != p->ny || p->nx != p->nz || p->nx < 8 || !is_pow2(p->nx)) return FFTK_ERR_UNSUPPORTED_SIZE;
  const int m = p->nx;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const long long R = (long long)m * m * m, M = (long long)m * m * (m / 2 + 1);
  float2* sp = nullptr;
  float* ut = nullptr;
  float* P = nullptr;
  cudaError_t e = cudaMalloc(&sp, sizeof(float2) * 6 * (size_t)M);
  if (e == cudaSuccess) e = cudaMalloc(&ut, sizeof(float) * 3 * (size_t)R);
  if (e == cudaSuccess) e = cudaMalloc(&P, sizeof(float) * 6 * (size_t)R);
  fftk_status s = e == cudaSuccess ? FFTK_OK : FFTK_ERR_OOM;
  // ubar_T = T ubar
  if (s == FFTK_OK) s = fftk_r2c(p, ubar, sp, 3, cuda_stream);
  if (s == FFTK_OK) {
    LaunchScope ls(p, KK_AUX, st);
    k_truncate<<<grid_for(3 * M, 256), 256, 0, st>>>(sp, m, 3);
    s = from_cuda(cudaGetLastError());
  }
  if (s == FFTK_OK) s = fftk_c2r(p, sp, ut, 3, cuda_stream);
  // T[tau + ubar_i ubar_j - ubar_T,i ubar_T,j]
  if (s == FFTK_OK) {
    LaunchScope ls(p, KK_AUX, st);
    k_les_products<<<grid_for(R, 256), 256, 0, st>>>(ubar, tau, ut, P, R);
    s = from_cuda(cudaGetLastError());
  }
  if (s == FFTK_OK) s = fftk_r2c(p, P, sp, 6, cuda_stream);
  if (s == FFTK_OK) {
    LaunchScope ls(p, KK_AUX, st);
    k_truncate<<<grid_for(6 * M, 256), 256, 0, st>>>(sp, m, 6);
    s = from_cuda(cudaGetLastError());
  }
  if (s == FFTK_OK) s = fftk_c2r(p, sp, out, 6, cuda_stream);
  if (s == FFTK_OK) s = from_cuda(cudaStreamSynchronize(st));
  cudaGetLastError();
  cudaFree(sp);
  cudaFree(ut);
  cudaFree(P);
  return s;
}

extern "C" fftk_status tarang_mlp_create(int max_batch, tarang_mlp* out) {
  if (!out || max_batch < 1) return FFTK_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return FFTK_ERR_NO_DEVICE;
  }
  tarang_mlp m = new (std::nothrow) tarang_mlp_s;
  if (!m) return FFTK_ERR_OOM;
  m->max_batch = max_batch;
  const int nblk = (max_batch + kChunk - 1) / kChunk;
  cudaError_t e = cudaMalloc(&m->part, sizeof(float) * (size_t)nblk * kNP);
  if (e == cudaSuccess) e = cudaMalloc(&m->loss_part, sizeof(double) * (size_t)nblk);
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc(&m->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
  if (e == cudaSuccess) e = mlp_attrs();
  if (e != cudaSuccess) {
    cudaFree(m->part);
    cudaFree(m->loss_part);
    cudaFree(m->grad);
    cudaFree(m->err);
    delete m;
    cudaGetLastError();
    return FFTK_ERR_OOM;
  }
  *out = m;
  return FFTK_OK;
}

extern "C" fftk_status tarang_mlp_destroy(tarang_mlp m) {
  if (!m) return FFTK_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  cudaFree(m->part);
  cudaFree(m->loss_part);
  cudaFree(m->grad);
  cudaFree(m->err);
  delete m;
  return FFTK_OK;
}

extern "C" fftk_status tarang_mlp_forward(tarang_mlp m, const float* params, const float* x, float* y, int B,
                                          void* cuda_stream) {
  if (!m || !params || !x || !y || B < 1) return FFTK_ERR_INVALID_ARG;
  k_mlp_forward_tc<<<mlptc_grid(B), mlptc::kThreads, mlptc::kSmem, static_cast<cudaStream_t>(cuda_stream)>>>(
      params, x, y, B, m->err);
  return from_cuda(cudaGetLastError());
}

extern "C" fftk_status tarang_mlp_sync(tarang_mlp m, void* cuda_stream) {
  if (!m) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  if (h) {
    e = cudaMemsetAsync(m->err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? FFTK_ERR_TIMEOUT : from_cuda(e);
  }
  return FFTK_OK;
}

extern "C" fftk_status tarang_mlp_loss_grad_mode(tarang_mlp m, const float* params, const float* x, const float* t,
                                                 int B, float* grad, double* loss, int act_mode, void* cuda_stream) {
  if (!m || !params || !x || !t || !grad || B < 1 || B > m->max_batch) return FFTK_ERR_INVALID_ARG;
  if (act_mode != TARANG_ACT_BF16 && act_mode != TARANG_ACT_FP32) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblk = (B + kChunk - 1) / kChunk;
  if (act_mode == TARANG_ACT_BF16)
    k_mlp_grad<true><<<nblk, kChunk, mlp_smem(), st>>>(params, x, t, B, m->part, m->loss_part);
  else
    k_mlp_grad<false><<<nblk, kChunk, mlp_smem(), st>>>(params, x, t, B, m->part, m->loss_part);
  k_mlp_reduce<<<(kNP + 255) / 256, 256, 0, st>>>(m->part, nblk, grad, m->loss_part, loss,
                                                 1.0 / (6.0 * (double)B));
  return from_cuda(cudaGetLastError());
}

extern "C" fftk_status tarang_mlp_loss_grad(tarang_mlp m, const float* params, const float* x, const float* t,
                                            int B, float* grad, double* loss, void* cuda_stream) {
  return tarang_mlp_loss_grad_mode(m, params, x, t, B, grad, loss, TARANG_ACT_BF16, cuda_stream);
}

extern "C" fftk_status tarang_mlp_forward_mode(tarang_mlp m, const float* params, const float* x, float* y, int B,
                                               int act_mode, void* cuda_stream) {
  if (!m || !params || !x || !y || B < 1) return FFTK_ERR_INVALID_ARG;
  if (act_mode != TARANG_ACT_BF16 && act_mode != TARANG_ACT_FP32) return FFTK_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblk = (B + kChunk - 1) / kChunk;
  if (act_mode == TARANG_ACT_BF16)
    k_mlp_forward_cc<true><<<nblk, kChunk, mlp_smem(), st>>>(params, x, y, B);
  else
    k_mlp_forward_cc<false><<<nblk, kChunk, mlp_smem(), st>>>(params, x, y, B);
  return from_cuda(cudaGetLastError());
}

extern "C" fftk_status tarang_mlp_adam(float* params, float* mom, float* var, const float* grad, int step,
                                       float lr, float beta1, float beta2, float eps, void* cuda_stream) {
  if (!params || !mom || !var || !grad || step < 1) return FFTK_ERR_INVALID_ARG;
  const float c1 = (float)(1.0 - std::pow((double)beta1, step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, step));
  k_adam<<<(kNP + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(params, mom, var, grad, kNP, lr,
                                                                                beta1, beta2, eps, c1, c2);
  return from_cuda(cudaGetLastError());
}

extern "C" fftk_status tarang_mlp_train_step(tarang_mlp m, float* params, float* mom, float* var, int step,
                                             const float* x, const float* t, int B, float lr, double* loss,
                                             void* cuda_stream) {
  fftk_status s = tarang_mlp_loss_grad(m, params, x, t, B, m ? m->grad : nullptr, loss, cuda_stream);
  if (s != FFTK_OK) return s;
  return tarang_mlp_adam(params, mom, var, m->grad, step, lr, 0.9f, 0.999f, 1e-8f, cuda_stream);
}

// SplitMix64 (Steele, Lea & Flood 2014): output number c of the stream that
// starts from state 0
static uint64_t splitmix64_at(uint64_t c) {
  uint64_t z = (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" fftk_status tarang_sgs_train(tarang_mlp m, float* params, float* mom, float* var, int first_step,
                                        int steps, const float* x, const float* t, long long nsamples, int batch,
                                        float lr, unsigned long long seed, double* loss_log, int log_every,
                                        void* cuda_stream) {
  if (!m || !params || !mom || !var || !x || !t || first_step < 1 || steps < 0 || batch < 1 ||
      batch > m->max_batch || nsamples < batch || (loss_log && log_every < 1) || !(lr > 0.f))
    return FFTK_ERR_INVALID_ARG;
  const unsigned long long windows = (unsigned long long)(nsamples - batch + 1);
  for (int k = 0; k < steps; ++k) {
    const int step = first_step + k;
    const long long off = (long long)(splitmix64_at((seed << 32) + (unsigned long long)step) % windows);
    double* lp = (loss_log && (k + 1) % log_every == 0) ? loss_log + ((k + 1) / log_every - 1) : nullptr;
    const fftk_status s =
        tarang_mlp_train_step(m, params, mom, var, step, x + off * 5, t + off * 6, batch, lr, lp, cuda_stream);
    if (s != FFTK_OK) return s;
  }
  return FFTK_OK;
}

// -------------------------------------------- SGS term for the solver ------
namespace fftk {

void sgs_free(fftk_sgs_work* w) {
  if (!w) return;
  cudaFree(w->A);
  cudaFree(w->tau);
  cudaFree(w->gh);
  cudaFree(w->th);
  cudaFree(w->s);
  delete w;
}

// s = P[-i k_j tau_hat_ij] of the network's stress for the state u (2/3-truncated)
cudaError_t sgs_term(fftk_plan p, fftk_sgs_work** wp, const float2* u, const tarang_sgs_model* model,
                     cudaStream_t st, const float2** out) {
  const int n = p->nx;
  const long long R = (long long)n * n * n, M = (long long)n * n * (n / 2 + 1);
  const cudaError_t ea = mlp_attrs();
  if (ea != cudaSuccess) return ea;
  if (!*wp) {
    fftk_sgs_work* w = new (std::nothrow) fftk_sgs_work;
    if (!w) return cudaErrorMemoryAllocation;
    w->n = n;
    cudaError_t e = cudaMalloc(&w->A, sizeof(float) * 9 * (size_t)R);
    if (e == cudaSuccess) e = cudaMalloc(&w->tau, sizeof(float) * 6 * (size_t)R);
    if (e == cudaSuccess) e = cudaMalloc(&w->gh, sizeof(float2) * 9 * (size_t)M);
    if (e == cudaSuccess) e = cudaMalloc(&w->th, sizeof(float2) * 6 * (size_t)M);
    if (e == cudaSuccess) e = cudaMalloc(&w->s, sizeof(float2) * 3 * (size_t)M);
    if (e != cudaSuccess) {
      sgs_free(w);
      return e;
    }
    *wp = w;
  }
  fftk_sgs_work* w = *wp;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_grad_spectra<<<grid_for(M, 256), 256, 0, st>>>(u, w->gh, n);
  }
  if (fftk_c2r(p, w->gh, w->A, 9, st) != FFTK_OK) return cudaErrorLaunchFailure;
  SGSConst c;
  std::memcpy(c.in_shift, model->in_shift, sizeof(c.in_shift));
  std::memcpy(c.in_scale, model->in_scale, sizeof(c.in_scale));
  std::memcpy(c.out_scale, model->out_scale, sizeof(c.out_scale));
  {
    LaunchScope ls(p, KK_AUX, st);
    k_sgs_pointwise_tc<<<mlptc_grid(R), mlptc::kThreads, mlptc::kSmem, st>>>(w->A, R, model->params, c, w->tau,
                                                                            p->d_err);
  }
  if (fftk_r2c(p, w->tau, w->th, 6, st) != FFTK_OK) return cudaErrorLaunchFailure;
  {
    LaunchScope ls(p, KK_AUX, st);
    k_sgs_divergence<<<grid_for(M, 256), 256, 0, st>>>(w->th, w->s, n);
  }
  *out = w->s;
  return cudaGetLastError();
}

}  // namespace fftk
