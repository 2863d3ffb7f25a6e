/* Plain, slow FP64 CPU oracle for the FFTK/Tarang hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product library.  It shares no
 * code with the CUDA path.  Every routine is written for readability: a
 * textbook recursive radix-2 FFT, line-by-line 3D passes in the order of the
 * paper's Sec. 3, and pointwise loops for the solver.  OpenMP only splits
 * independent lines / points across threads; it changes no arithmetic order
 * within a line.
 *
 * Parity status: every function here is pinned by the CPU tests against closed
 * forms, brute-force sums, invariants or numpy's FFT (see the test files);
 * the turbulent 512^3 run after many steps is checked only through those pins.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559005768

typedef ocplx cplx;

static int is_pow2(long n) { return n >= 1 && (n & (n - 1)) == 0; }

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* tw[m] = exp(sign * 2 pi i m / n) for m < max(n/2, 1), FP64 host libm. */
static cplx *make_twiddles(long n, int sign) {
  long h = n / 2 > 0 ? n / 2 : 1;
  cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)h);
  if (!tw) return NULL;
  for (long m = 0; m < h; m++) {
    double ang = TWO_PI * (double)m / (double)n;
    tw[m] = cos(ang) + (double)sign * sin(ang) * I;
  }
  return tw;
}

/* Recursive radix-2 decimation in time (Cooley and Tukey, 1965):
 *   out[k] = sum_{j<n} in[j*stride] exp(sign 2 pi i j k / n).
 * The sub-transform of length n uses tw[k * twstep], twstep = n_top / n. */
static void fft_rec(const cplx *in, long stride, cplx *out, long n,
                    const cplx *tw, long twstep) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  long h = n / 2;
  fft_rec(in, 2 * stride, out, h, tw, 2 * twstep);          /* even samples */
  fft_rec(in + stride, 2 * stride, out + h, h, tw, 2 * twstep); /* odd samples */
  for (long k = 0; k < h; k++) {
    cplx e = out[k];
    cplx o = tw[k * twstep] * out[k + h];
    out[k] = e + o;
    out[k + h] = e - o;
  }
}

int oracle_fft1d(const cplx *in, cplx *out, long n, int sign) {
  if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
  cplx *tw = make_twiddles(n, sign);
  if (!tw) return -2;
  fft_rec(in, 1, out, n, tw, 1);
  free(tw);
  return 0;
}

/* The DFT by its definition, O(n^2); the phase j*k is reduced mod n first. */
int oracle_dft1d(const cplx *in, cplx *out, long n, int sign) {
  if (n < 1 || (sign != 1 && sign != -1)) return -1;
  for (long k = 0; k < n; k++) {
    cplx s = 0;
    for (long j = 0; j < n; j++) {
      long m = (j * k) % n;
      double ang = TWO_PI * (double)m / (double)n;
      s += in[j] * (cos(ang) + (double)sign * sin(ang) * I);
    }
    out[k] = s;
  }
  return 0;
}

/* Lines of a 3D transform: n = 2^m by the recursive radix-2 FFT above, or
 * n = 3 * 2^m (the paper's 768, 1536, 3072 grids) by the DFT's definition,
 * O(n^2), with the phase j k reduced mod n. */
static int ok_len(long n) { return is_pow2(n) || (n % 3 == 0 && is_pow2(n / 3)); }
/* Cubic grids of the solver: an even length the 1D transforms take (2^m, or
 * 3 * 2^m as in the paper's 768^3 - 3072^3 runs of Sec. 6-7). */
static int ok_grid(long n) { return n >= 2 && n % 2 == 0 && ok_len(n); }

static cplx *make_line_table(long n, int sign) {
  if (is_pow2(n)) return make_twiddles(n, sign);
  cplx *t = (cplx *)malloc(sizeof(cplx) * (size_t)n);
  if (!t) return NULL;
  for (long m = 0; m < n; m++) {
    double ang = TWO_PI * (double)m / (double)n;
    t[m] = cos(ang) + (double)sign * sin(ang) * I;
  }
  return t;
}

static void line_transform(const cplx *in, cplx *out, long n, const cplx *tab) {
  if (is_pow2(n)) {
    fft_rec(in, 1, out, n, tab, 1);
    return;
  }
  for (long k = 0; k < n; k++) {
    cplx acc = 0;
    for (long j = 0; j < n; j++) acc += in[j] * tab[(j * k) % n];
    out[k] = acc;
  }
}

/* ---------------------------------------------------------------- 3D ---- */

static long maxl3(long a, long b, long c) {
  long m = a > b ? a : b;
  return m > c ? m : c;
}

/* Forward: Sec. 3 steps 1 (r2c along z), 3 (c2c along y), 5 (c2c along x);
 * the 1/(Nx Ny Nz) factor makes Eq. (1) its inverse. */
int oracle_rfft3(const double *in, cplx *out, int nx, int ny, int nz) {
  if (!ok_len(nx) || !ok_len(ny) || !ok_len(nz) || nz < 2) return -1;
  const long NX = nx, NY = ny, NZ = nz, HZ = nz / 2 + 1;
  cplx *twz = make_line_table(NZ, -1), *twy = make_line_table(NY, -1),
       *twx = make_line_table(NX, -1);
  const long LMAX = maxl3(NX, NY, NZ);
  int rc = 0;
#pragma omp parallel
  {
    cplx *lin = (cplx *)malloc(sizeof(cplx) * (size_t)LMAX);
    cplx *lout = (cplx *)malloc(sizeof(cplx) * (size_t)LMAX);
    /* step 1: real-to-complex along z for every (i, j) column */
#pragma omp for schedule(static)
    for (long ij = 0; ij < NX * NY; ij++) {
      for (long l = 0; l < NZ; l++) lin[l] = in[ij * NZ + l];
      line_transform(lin, lout, NZ, twz);
      for (long c = 0; c < HZ; c++) out[ij * HZ + c] = lout[c];
    }
    /* step 3: complex-to-complex along y for every (i, k_z) */
#pragma omp for schedule(static)
    for (long ic = 0; ic < NX * HZ; ic++) {
      long i = ic / HZ, c = ic % HZ;
      for (long j = 0; j < NY; j++) lin[j] = out[(i * NY + j) * HZ + c];
      line_transform(lin, lout, NY, twy);
      for (long j = 0; j < NY; j++) out[(i * NY + j) * HZ + c] = lout[j];
    }
    /* step 5: complex-to-complex along x for every (k_y, k_z) */
#pragma omp for schedule(static)
    for (long jc = 0; jc < NY * HZ; jc++) {
      for (long i = 0; i < NX; i++) lin[i] = out[i * NY * HZ + jc];
      line_transform(lin, lout, NX, twx);
      for (long i = 0; i < NX; i++) out[i * NY * HZ + jc] = lout[i];
    }
    free(lin);
    free(lout);
  }
  const double scale = 1.0 / ((double)NX * (double)NY * (double)NZ);
  const long M = NX * NY * HZ;
#pragma omp parallel for schedule(static)
  for (long m = 0; m < M; m++) out[m] *= scale;
  free(twz);
  free(twy);
  free(twx);
  return rc;
}

/* Inverse: the reverse of the forward passes (Sec. 3): x, y, then z c2r.  The
 * z line is extended by f(N-c) = conj(f(c)) and the real part is kept. */
int oracle_irfft3(const cplx *in, double *out, int nx, int ny, int nz) {
  if (!ok_len(nx) || !ok_len(ny) || !ok_len(nz) || nz < 2) return -1;
  const long NX = nx, NY = ny, NZ = nz, HZ = nz / 2 + 1;
  const long M = NX * NY * HZ;
  cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)M);
  if (!work) return -2;
  memcpy(work, in, sizeof(cplx) * (size_t)M);
  cplx *twz = make_line_table(NZ, +1), *twy = make_line_table(NY, +1),
       *twx = make_line_table(NX, +1);
  const long LMAX = maxl3(NX, NY, NZ);
#pragma omp parallel
  {
    cplx *lin = (cplx *)malloc(sizeof(cplx) * (size_t)LMAX);
    cplx *lout = (cplx *)malloc(sizeof(cplx) * (size_t)LMAX);
#pragma omp for schedule(static)
    for (long jc = 0; jc < NY * HZ; jc++) {
      for (long i = 0; i < NX; i++) lin[i] = work[i * NY * HZ + jc];
      line_transform(lin, lout, NX, twx);
      for (long i = 0; i < NX; i++) work[i * NY * HZ + jc] = lout[i];
    }
#pragma omp for schedule(static)
    for (long ic = 0; ic < NX * HZ; ic++) {
      long i = ic / HZ, c = ic % HZ;
      for (long j = 0; j < NY; j++) lin[j] = work[(i * NY + j) * HZ + c];
      line_transform(lin, lout, NY, twy);
      for (long j = 0; j < NY; j++) work[(i * NY + j) * HZ + c] = lout[j];
    }
#pragma omp for schedule(static)
    for (long ij = 0; ij < NX * NY; ij++) {
      for (long c = 0; c < NZ; c++)
        lin[c] = (c < HZ) ? work[ij * HZ + c] : conj(work[ij * HZ + (NZ - c)]);
      line_transform(lin, lout, NZ, twz);
      for (long l = 0; l < NZ; l++) out[ij * NZ + l] = creal(lout[l]);
    }
    free(lin);
    free(lout);
  }
  free(twz);
  free(twy);
  free(twx);
  free(work);
  return 0;
}

/* ------------------------------------------------ sine / cosine bases ---- */
/* Sec. 2.1, Eq. (2b, 2c): along a free-slip axis the inverse transform is
 *   f(s_j) = sum_k fhat_k 2 sin(k s_j)   (sine, k = 1..n, fhat_k stored at k-1)
 *   f(s_j) = sum_k fhat_k 2 cos(k s_j)   (cosine, k = 0..n-1, stored at k)
 * on the n points s_j = (j + 1/2) pi / n of [0, pi], and the forward
 * transform is its inverse:  fhat_k = (c_k / n) sum_j f(s_j) sin(k s_j)
 * (cos(k s_j) for the cosine), c_k = 1/2 for the cosine k = 0 and the sine
 * k = n, 1 otherwise.  Both by their definitions, O(n^2), complex-linear. */

/* cos(pi m / (2n)) and sin(pi m / (2n)) for an integer m reduced mod 4n */
static double cos_q(long m, long n) {
  m %= 4 * n;
  if (m < 0) m += 4 * n;
  return cos(TWO_PI * (double)m / (double)(4 * n));
}
static double sin_q(long m, long n) {
  m %= 4 * n;
  if (m < 0) m += 4 * n;
  return sin(TWO_PI * (double)m / (double)(4 * n));
}

/* table[k][j] = phi_k(s_j) / 2 for the n modes of the basis (k index of storage) */
static double *sc_table(long n, int kind) {
  double *t = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!t) return NULL;
  for (long i = 0; i < n; i++) {
    long k = (kind == ORACLE_SINE) ? i + 1 : i;
    for (long j = 0; j < n; j++) {
      long m = k * (2 * j + 1); /* k s_j = pi m / (2n) */
      t[i * n + j] = (kind == ORACLE_SINE) ? sin_q(m, n) : cos_q(m, n);
    }
  }
  return t;
}

static void sc_line(const cplx *in, cplx *out, long n, int kind, int dir, const double *t) {
  if (dir < 0) {
    for (long i = 0; i < n; i++) {
      cplx acc = 0;
      for (long j = 0; j < n; j++) acc += in[j] * t[i * n + j];
      int edge = (kind == ORACLE_SINE) ? (i == n - 1) : (i == 0);
      out[i] = acc * ((edge ? 0.5 : 1.0) / (double)n);
    }
  } else {
    for (long j = 0; j < n; j++) {
      cplx acc = 0;
      for (long i = 0; i < n; i++) acc += in[i] * t[i * n + j];
      out[j] = 2.0 * acc;
    }
  }
}

int oracle_sc1d(const cplx *in, cplx *out, long n, int kind, int dir) {
  if (n < 1 || (kind != ORACLE_SINE && kind != ORACLE_COSINE) || (dir != 1 && dir != -1)) return -1;
  double *t = sc_table(n, kind);
  if (!t) return -2;
  sc_line(in, out, n, kind, dir, t);
  free(t);
  return 0;
}

/* One axis of a 3D array a[n0][n1][n2] (complex): every line along `axis`
 * goes through the Fourier transform (kind ORACLE_FOURIER, sign = dir, factor
 * 1/n when forward) or the sine/cosine transform above. */
static int axis_pass(cplx *a, const long dims[3], int axis, int kind, int dir) {
  const long n = dims[axis];
  long stride = 1;
  for (int d = axis + 1; d < 3; d++) stride *= dims[d];
  const long nlines = dims[0] * dims[1] * dims[2] / n;
  double *t = NULL;
  cplx *tw = NULL;
  if (kind == ORACLE_FOURIER) {
    if (!is_pow2(n)) return -1;
    tw = make_twiddles(n, dir);
  } else {
    t = sc_table(n, kind);
  }
  if (!tw && !t) return -2;
#pragma omp parallel
  {
    cplx *lin = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *lout = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
    for (long l = 0; l < nlines; l++) {
      long outer = l / stride, inner = l % stride;
      cplx *base = a + outer * n * stride + inner;
      for (long i = 0; i < n; i++) lin[i] = base[i * stride];
      if (kind == ORACLE_FOURIER) {
        fft_rec(lin, 1, lout, n, tw, 1);
        if (dir < 0)
          for (long i = 0; i < n; i++) lout[i] /= (double)n;
      } else {
        sc_line(lin, lout, n, kind, dir, t);
      }
      for (long i = 0; i < n; i++) base[i * stride] = lout[i];
    }
    free(lin);
    free(lout);
  }
  free(t);
  free(tw);
  return 0;
}

static int basis_ok(const int kind[3]) {
  for (int d = 0; d < 3; d++)
    if (kind[d] != ORACLE_FOURIER && kind[d] != ORACLE_SINE && kind[d] != ORACLE_COSINE) return 0;
  /* Fourier axes are the trailing ones: FFF, SFF, SSF, SSS (Sec. 2.1) */
  if (kind[0] == ORACLE_FOURIER && (kind[1] != ORACLE_FOURIER || kind[2] != ORACLE_FOURIER)) return 0;
  if (kind[1] == ORACLE_FOURIER && kind[2] != ORACLE_FOURIER) return 0;
  return 1;
}

/* Forward 3D transform in the paper's pass order (z, then y, then x) with a
 * basis per axis.  in: real [nx][ny][nz].  out: complex [nx][ny][hz] with
 * hz = nz/2 + 1 when z is Fourier (real-to-complex half spectrum), else
 * hz = nz (the coefficients are real; imaginary parts 0). */
int oracle_transform3(const double *in, cplx *out, int nx, int ny, int nz, const int kind[3]) {
  if (!basis_ok(kind) || nx < 1 || ny < 1 || nz < 2) return -1;
  const long NX = nx, NY = ny, NZ = nz;
  const int zf = kind[2] == ORACLE_FOURIER;
  const long HZ = zf ? NZ / 2 + 1 : NZ;
  cplx *full = (cplx *)malloc(sizeof(cplx) * (size_t)(NX * NY * NZ));
  if (!full) return -2;
  for (long i = 0; i < NX * NY * NZ; i++) full[i] = in[i];
  const long dfull[3] = {NX, NY, NZ};
  int rc = axis_pass(full, dfull, 2, kind[2], -1);
  const long dh[3] = {NX, NY, HZ};
  for (long l = 0; l < NX * NY; l++)
    for (long c = 0; c < HZ; c++) out[l * HZ + c] = full[l * NZ + c];
  free(full);
  if (!rc && NY > 1) rc = axis_pass(out, dh, 1, kind[1], -1);
  if (!rc && NX > 1) rc = axis_pass(out, dh, 0, kind[0], -1);
  return rc;
}

/* Inverse in the reverse order (x, y, then z).  A Fourier z axis is extended
 * by conjugation per line and the real part kept (as oracle_irfft3). */
int oracle_itransform3(const cplx *in, double *out, int nx, int ny, int nz, const int kind[3]) {
  if (!basis_ok(kind) || nx < 1 || ny < 1 || nz < 2) return -1;
  const long NX = nx, NY = ny, NZ = nz;
  const int zf = kind[2] == ORACLE_FOURIER;
  const long HZ = zf ? NZ / 2 + 1 : NZ;
  cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)(NX * NY * HZ));
  cplx *full = (cplx *)malloc(sizeof(cplx) * (size_t)(NX * NY * NZ));
  if (!w || !full) return -2;
  memcpy(w, in, sizeof(cplx) * (size_t)(NX * NY * HZ));
  const long dh[3] = {NX, NY, HZ};
  int rc = 0;
  if (NX > 1) rc = axis_pass(w, dh, 0, kind[0], +1);
  if (!rc && NY > 1) rc = axis_pass(w, dh, 1, kind[1], +1);
  for (long l = 0; l < NX * NY; l++)
    for (long c = 0; c < NZ; c++) {
      if (zf)
        full[l * NZ + c] = (c < HZ) ? w[l * HZ + c] : conj(w[l * HZ + (NZ - c)]);
      else
        full[l * NZ + c] = w[l * NZ + c];
    }
  const long dfull[3] = {NX, NY, NZ};
  if (!rc) rc = axis_pass(full, dfull, 2, kind[2], +1);
  for (long i = 0; i < NX * NY * NZ; i++) out[i] = creal(full[i]);
  free(w);
  free(full);
  return rc;
}

/* One coefficient of oracle_transform3 straight from its definition, for
 * FP32 input too large for the full transform: the sum over all points of
 * f times the product of the three axis factors (exp(-i k s)/n on a Fourier
 * axis, c_k sin(k s_j)/n or c_k cos(k s_j)/n on a sine/cosine axis). */
static cplx axis_factor(int kind, long idx, long j, long n) {
  if (kind == ORACLE_FOURIER) {
    long m = (idx * j) % n;
    double ang = TWO_PI * (double)m / (double)n;
    return (cos(ang) - sin(ang) * I) / (double)n;
  }
  long k = (kind == ORACLE_SINE) ? idx + 1 : idx;
  int edge = (kind == ORACLE_SINE) ? (k == n) : (k == 0);
  double c = (edge ? 0.5 : 1.0) / (double)n;
  long m = k * (2 * j + 1);
  return c * ((kind == ORACLE_SINE) ? sin_q(m, n) : cos_q(m, n));
}

int oracle_transform3_coeff_f32(const float *in, int nx, int ny, int nz, const int kind[3], int a, int b,
                                int c, double *out) {
  if (!basis_ok(kind)) return -1;
  const long NX = nx, NY = ny, NZ = nz;
  cplx *fy = (cplx *)malloc(sizeof(cplx) * (size_t)NY);
  cplx *fz = (cplx *)malloc(sizeof(cplx) * (size_t)NZ);
  if (!fy || !fz) return -2;
  for (long j = 0; j < NY; j++) fy[j] = axis_factor(kind[1], b, j, NY);
  for (long l = 0; l < NZ; l++) fz[l] = axis_factor(kind[2], c, l, NZ);
  double re = 0.0, im = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : re, im)
  for (long i = 0; i < NX; i++) {
    cplx row = 0;
    for (long j = 0; j < NY; j++) {
      cplx acc = 0;
      const float *line = in + (i * NY + j) * NZ;
      for (long l = 0; l < NZ; l++) acc += (double)line[l] * fz[l];
      row += acc * fy[j];
    }
    cplx t = row * axis_factor(kind[0], a, i, NX);
    re += creal(t);
    im += cimag(t);
  }
  free(fy);
  free(fz);
  out[0] = re;
  out[1] = im;
  return 0;
}

/* exp(sign 2 pi i m / n) for m reduced mod n. */
static cplx phase(long m, long n, int sign) {
  m %= n;
  if (m < 0) m += n;
  double ang = TWO_PI * (double)m / (double)n;
  return cos(ang) + (double)sign * sin(ang) * I;
}

void oracle_rfft3_coeff_f32(const float *in, int nx, int ny, int nz, int a, int b, int c,
                            double *re_im) {
  const long NX = nx, NY = ny, NZ = nz;
  cplx *ex = (cplx *)malloc(sizeof(cplx) * (size_t)NX);
  cplx *ey = (cplx *)malloc(sizeof(cplx) * (size_t)NY);
  cplx *ez = (cplx *)malloc(sizeof(cplx) * (size_t)NZ);
  for (long i = 0; i < NX; i++) ex[i] = phase((long)a * i, NX, -1);
  for (long j = 0; j < NY; j++) ey[j] = phase((long)b * j, NY, -1);
  for (long l = 0; l < NZ; l++) ez[l] = phase((long)c * l, NZ, -1);
  double sre = 0.0, sim = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sre, sim)
  for (long i = 0; i < NX; i++) {
    cplx si = 0;
    for (long j = 0; j < NY; j++) {
      cplx sj = 0;
      const float *line = in + (i * NY + j) * NZ;
      for (long l = 0; l < NZ; l++) sj += (double)line[l] * ez[l];
      si += ey[j] * sj;
    }
    cplx t = ex[i] * si;
    sre += creal(t);
    sim += cimag(t);
  }
  free(ex);
  free(ey);
  free(ez);
  const double scale = 1.0 / ((double)NX * (double)NY * (double)NZ);
  re_im[0] = sre * scale;
  re_im[1] = sim * scale;
}

double oracle_irfft3_point_c64(const float *in, int nx, int ny, int nz, int i, int j, int l) {
  const long NX = nx, NY = ny, NZ = nz, HZ = nz / 2 + 1;
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (long a = 0; a < NX; a++) {
    cplx pa = phase(a * i, NX, +1);
    double sa = 0.0;
    for (long b = 0; b < NY; b++) {
      cplx pab = pa * phase(b * j, NY, +1);
      for (long c = 0; c < HZ; c++) {
        const float *v = in + 2 * ((a * NY + b) * HZ + c);
        cplx f = (double)v[0] + (double)v[1] * I;
        double w = (c == 0 || 2 * c == NZ) ? 1.0 : 2.0;
        sa += w * creal(f * pab * phase(c * l, NZ, +1));
      }
    }
    s += sa;
  }
  return s;
}

/* --------------------------------------------------------- wavenumbers ---- */

/* Wavenumber of index a on an x or y axis: a if a < n/2, else a - n
 * (the Nyquist index n/2 stands for -n/2); on z the index is the wavenumber. */
static long kxy(long a, long n) { return (2 * a < n) ? a : a - n; }
/* Wavenumber used inside derivatives: the Nyquist mode gets i k := 0. */
static long kder(long k, long n) { return (2 * labs(k) == n) ? 0 : k; }
/* 2/3 rule (Sec. 2.2): keep the mode only if 3|k| < N along every axis. */
static int kept(long kx, long ky, long kz, long n) {
  return 3 * labs(kx) < n && 3 * labs(ky) < n && 3 * labs(kz) < n;
}

int oracle_dealias(cplx *f, int nfields, int n) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  for (int fld = 0; fld < nfields; fld++)
    for (long a = 0; a < N; a++)
      for (long b = 0; b < N; b++)
        for (long c = 0; c < HZ; c++)
          if (!kept(kxy(a, N), kxy(b, N), c, N)) f[fld * M + (a * N + b) * HZ + c] = 0;
  return 0;
}

/* Projection onto divergence-free fields, Eq. (8): u <- u - k (k.u)/|k|^2,
 * with u(0) = 0. */
int oracle_project(cplx *u, int n) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        double kx = (double)kxy(a, N), ky = (double)kxy(b, N), kz = (double)c;
        double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0.0) {
          u[idx] = u[M + idx] = u[2 * M + idx] = 0;
          continue;
        }
        cplx kdotu = kx * u[idx] + ky * u[M + idx] + kz * u[2 * M + idx];
        u[idx] -= kx * kdotu / k2;
        u[M + idx] -= ky * kdotu / k2;
        u[2 * M + idx] -= kz * kdotu / k2;
      }
  return 0;
}

static double mode_weight(long c, long nz) { return (c == 0 || 2 * c == nz) ? 1.0 : 2.0; }

static double sq(cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* ------------------------------------------------------ Navier-Stokes ---- */

/* Sum over forced modes of 1/2 w |u|^2. */
static double forced_energy(const cplx *u, int n, const oracle_ns_params *p) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  double e = 0.0;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long kx = kxy(a, N), ky = kxy(b, N), k2 = kx * kx + ky * ky + c * c;
        if (k2 < p->force_k2min || k2 > p->force_k2max) continue;
        long idx = (a * N + b) * HZ + c;
        e += 0.5 * mode_weight(c, N) * (sq(u[idx]) + sq(u[M + idx]) + sq(u[2 * M + idx]));
      }
  return e;
}

int oracle_ns_rhs(const cplx *uhat, cplx *nhat, int n, const oracle_ns_params *p) {
  if (!ok_grid(n)) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  cplx *what = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  double *ur = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  double *wr = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  double *nr = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  if (!what || !ur || !wr || !nr) return -2;
  /* 1. vorticity omega = curl u, in Fourier space i k x u */
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        double kx = (double)kder(kxy(a, N), N), ky = (double)kder(kxy(b, N), N),
               kz = (double)kder(c, N);
        cplx ux = uhat[idx], uy = uhat[M + idx], uz = uhat[2 * M + idx];
        what[idx] = I * (ky * uz - kz * uy);
        what[M + idx] = I * (kz * ux - kx * uz);
        what[2 * M + idx] = I * (kx * uy - ky * ux);
      }
  /* 2. velocity and vorticity in real space */
  for (int f = 0; f < 3; f++) {
    oracle_irfft3(uhat + f * M, ur + f * R, n, n, n);
    oracle_irfft3(what + f * M, wr + f * R, n, n, n);
  }
  /* 3. pointwise product u x omega (the pseudo-spectral step of Sec. 2.2) */
#pragma omp parallel for schedule(static)
  for (long x = 0; x < R; x++) {
    double ux = ur[x], uy = ur[R + x], uz = ur[2 * R + x];
    double wx = wr[x], wy = wr[R + x], wz = wr[2 * R + x];
    nr[x] = uy * wz - uz * wy;
    nr[R + x] = uz * wx - ux * wz;
    nr[2 * R + x] = ux * wy - uy * wx;
  }
  /* 4. back to Fourier space, 5. dealias, 6. project */
  for (int f = 0; f < 3; f++) oracle_rfft3(nr + f * R, nhat + f * M, n, n, n);
  oracle_dealias(nhat, 3, n);
  oracle_project(nhat, n);
  /* 7. constant-power forcing: f = eps u / (2 E_f) on the forced modes */
  if (p && p->force_eps > 0.0) {
    double ef = forced_energy(uhat, n, p);
    if (ef > 0.0) {
      double g = p->force_eps / (2.0 * ef);
      for (long a = 0; a < N; a++)
        for (long b = 0; b < N; b++)
          for (long c = 0; c < HZ; c++) {
            long kx = kxy(a, N), ky = kxy(b, N), k2 = kx * kx + ky * ky + c * c;
            if (k2 < p->force_k2min || k2 > p->force_k2max) continue;
            long idx = (a * N + b) * HZ + c;
            for (int f = 0; f < 3; f++) nhat[f * M + idx] += g * uhat[f * M + idx];
          }
    }
  }
  free(what);
  free(ur);
  free(wr);
  free(nr);
  return 0;
}

int oracle_ns_rhs_divergence(const cplx *uhat, cplx *nhat, int n) {
  if (!ok_grid(n)) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  double *ur = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  double *pr = (double *)malloc(sizeof(double) * (size_t)R);
  cplx *th = (cplx *)malloc(sizeof(cplx) * 9 * (size_t)M); /* T_lj, full 3x3 */
  if (!ur || !pr || !th) return -2;
  for (int f = 0; f < 3; f++) oracle_irfft3(uhat + f * M, ur + f * R, n, n, n);
  for (int l = 0; l < 3; l++)
    for (int j = 0; j < 3; j++) {
      for (long x = 0; x < R; x++) pr[x] = ur[l * R + x] * ur[j * R + x];
      oracle_rfft3(pr, th + (l * 3 + j) * M, n, n, n);
    }
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        double k[3] = {(double)kder(kxy(a, N), N), (double)kder(kxy(b, N), N),
                       (double)kder(c, N)};
        for (int j = 0; j < 3; j++) {
          cplx s = 0;
          for (int l = 0; l < 3; l++) s += k[l] * th[(l * 3 + j) * M + idx];
          nhat[j * M + idx] = -I * s;
        }
      }
  oracle_dealias(nhat, 3, n);
  oracle_project(nhat, n);
  free(ur);
  free(pr);
  free(th);
  return 0;
}

/* RK2 (Heun) with integrating factor E = exp(-nu |k|^2 dt):
 *   u1 = E (u + dt N(u)),   u_new = 1/2 E u + 1/2 (u1 + dt N(u1)). */
int oracle_ns_step(cplx *uhat, int n, const oracle_ns_params *p, int nsteps) {
  if (!ok_grid(n) || !p) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  cplx *u1 = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  cplx *nh = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  double *E = (double *)malloc(sizeof(double) * (size_t)M);
  if (!u1 || !nh || !E) return -2;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        double kx = (double)kxy(a, N), ky = (double)kxy(b, N), kz = (double)c;
        E[(a * N + b) * HZ + c] = exp(-p->nu * (kx * kx + ky * ky + kz * kz) * p->dt);
      }
  for (int s = 0; s < nsteps; s++) {
    int rc = oracle_ns_rhs(uhat, nh, n, p);
    if (rc) return rc;
    for (int f = 0; f < 3; f++)
      for (long m = 0; m < M; m++)
        u1[f * M + m] = E[m] * (uhat[f * M + m] + p->dt * nh[f * M + m]);
    oracle_dealias(u1, 3, n);
    rc = oracle_ns_rhs(u1, nh, n, p);
    if (rc) return rc;
    for (int f = 0; f < 3; f++)
      for (long m = 0; m < M; m++)
        uhat[f * M + m] = 0.5 * E[m] * uhat[f * M + m] +
                          0.5 * (u1[f * M + m] + p->dt * nh[f * M + m]);
    oracle_dealias(uhat, 3, n);
  }
  free(u1);
  free(nh);
  free(E);
  return 0;
}

/* The paper's Runge-Kutta scheme of fourth order (Sec. 2.2; RK4, 36
 * transforms per step in Sec. 6) with the viscous integrating factor
 * (Lawson's form): with E = exp(-nu k^2 dt), H = exp(-nu k^2 dt/2),
 *   N1 = N(u),                 ua = H (u + dt/2 N1),
 *   N2 = N(ua),                ub = H u + dt/2 N2,
 *   N3 = N(ub),                uc = E u + dt H N3,
 *   N4 = N(uc),
 *   u <- E u + dt/6 (E N1 + 2 H N2 + 2 H N3 + N4). */
int oracle_ns_step_rk4(cplx *uhat, int n, const oracle_ns_params *p, int nsteps) {
  if (!ok_grid(n) || !p) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  cplx *us = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  cplx *nh = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  cplx *acc = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  double *E = (double *)malloc(sizeof(double) * (size_t)M);
  double *H = (double *)malloc(sizeof(double) * (size_t)M);
  if (!us || !nh || !acc || !E || !H) return -2;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        double kx = (double)kxy(a, N), ky = (double)kxy(b, N), kz = (double)c;
        double k2 = kx * kx + ky * ky + kz * kz;
        E[(a * N + b) * HZ + c] = exp(-p->nu * k2 * p->dt);
        H[(a * N + b) * HZ + c] = exp(-p->nu * k2 * p->dt * 0.5);
      }
  const double dt = p->dt;
  for (int s = 0; s < nsteps; s++) {
    int rc = oracle_ns_rhs(uhat, nh, n, p); /* N1 */
    if (rc) return rc;
    for (int f = 0; f < 3; f++)
      for (long m = 0; m < M; m++) {
        long i = f * M + m;
        acc[i] = E[m] * uhat[i] + dt / 6.0 * E[m] * nh[i];
        us[i] = H[m] * (uhat[i] + 0.5 * dt * nh[i]);
      }
    oracle_dealias(us, 3, n);
    rc = oracle_ns_rhs(us, nh, n, p); /* N2 */
    if (rc) return rc;
    for (int f = 0; f < 3; f++)
      for (long m = 0; m < M; m++) {
        long i = f * M + m;
        acc[i] += dt / 3.0 * H[m] * nh[i];
        us[i] = H[m] * uhat[i] + 0.5 * dt * nh[i];
      }
    oracle_dealias(us, 3, n);
    rc = oracle_ns_rhs(us, nh, n, p); /* N3 */
    if (rc) return rc;
    for (int f = 0; f < 3; f++)
      for (long m = 0; m < M; m++) {
        long i = f * M + m;
        acc[i] += dt / 3.0 * H[m] * nh[i];
        us[i] = E[m] * uhat[i] + dt * H[m] * nh[i];
      }
    oracle_dealias(us, 3, n);
    rc = oracle_ns_rhs(us, nh, n, p); /* N4 */
    if (rc) return rc;
    for (long i = 0; i < 3 * M; i++) uhat[i] = acc[i] + dt / 6.0 * nh[i];
    oracle_dealias(uhat, 3, n);
  }
  free(us);
  free(nh);
  free(acc);
  free(E);
  free(H);
  return 0;
}

/* ------------------------------------------------ Rayleigh-Benard (FFF) -- */
/* Sec. 2.2, Eqs. (12)-(13) in the non-dimensional form, on the 2 pi-periodic
 * cube with gravity along z: state s[4][n][n][n/2+1] = (u_x, u_y, u_z, theta),
 *   d_t u + (u.grad) u = -grad sigma + theta z + nu lap u,      nu = sqrt(Pr/Ra),
 *   d_t theta + (u.grad) theta = u_z + kappa lap theta,        kappa = 1/sqrt(Ra Pr).
 * Right-hand side without the diffusive terms (u solenoidal):
 *   N_u = P[F(u x omega) + theta z],  N_theta = -i k . F(u theta) + u_z,
 * both 2/3-truncated. */
int oracle_rbc_rhs(const cplx *st, cplx *out, int n) {
  if (!ok_grid(n)) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  int rc = oracle_ns_rhs(st, out, n, NULL); /* P[F(u x omega)] */
  if (rc) return rc;
  /* + P[theta z]: theta z - k k_z theta / |k|^2 */
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        double kx = (double)kxy(a, N), ky = (double)kxy(b, N), kz = (double)c;
        double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0.0 || !kept(kxy(a, N), kxy(b, N), c, N)) continue;
        cplx th = st[3 * M + idx];
        out[idx] += -kx * kz * th / k2;
        out[M + idx] += -ky * kz * th / k2;
        out[2 * M + idx] += th - kz * kz * th / k2;
      }
  /* N_theta = -i k . F(u theta) + u_z */
  double *ur = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  double *tr = (double *)malloc(sizeof(double) * (size_t)R);
  double *pr = (double *)malloc(sizeof(double) * (size_t)R);
  cplx *ph = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  if (!ur || !tr || !pr || !ph) return -2;
  for (int f = 0; f < 3; f++) oracle_irfft3(st + f * M, ur + f * R, n, n, n);
  oracle_irfft3(st + 3 * M, tr, n, n, n);
  for (int f = 0; f < 3; f++) {
    for (long x = 0; x < R; x++) pr[x] = ur[f * R + x] * tr[x];
    oracle_rfft3(pr, ph + f * M, n, n, n);
  }
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        double kx = (double)kder(kxy(a, N), N), ky = (double)kder(kxy(b, N), N), kz = (double)kder(c, N);
        cplx div = kx * ph[idx] + ky * ph[M + idx] + kz * ph[2 * M + idx];
        out[3 * M + idx] = -I * div + st[2 * M + idx];
      }
  oracle_dealias(out + 3 * M, 1, n);
  free(ur);
  free(tr);
  free(pr);
  free(ph);
  return 0;
}

/* nsteps of RK2 (Heun, scheme 0) or RK4 (Lawson, scheme 1) with the
 * integrating factors exp(-nu k^2 dt) for u and exp(-kappa k^2 dt) for theta,
 * in the forms of oracle_ns_step and oracle_ns_step_rk4. */
int oracle_rbc_step(cplx *st, int n, double Ra, double Pr, double dt, int nsteps, int scheme) {
  if (!ok_grid(n) || Ra <= 0.0 || Pr <= 0.0 || (scheme != 0 && scheme != 1)) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  const double nu = sqrt(Pr / Ra), kappa = 1.0 / sqrt(Ra * Pr);
  cplx *us = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)M);
  cplx *nh = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)M);
  cplx *acc = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)M);
  double *E = (double *)malloc(sizeof(double) * 2 * (size_t)M); /* [u or theta][mode] */
  double *H = (double *)malloc(sizeof(double) * 2 * (size_t)M);
  if (!us || !nh || !acc || !E || !H) return -2;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long m = (a * N + b) * HZ + c;
        double kx = (double)kxy(a, N), ky = (double)kxy(b, N), kz = (double)c;
        double k2 = kx * kx + ky * ky + kz * kz;
        E[m] = exp(-nu * k2 * dt);
        E[M + m] = exp(-kappa * k2 * dt);
        H[m] = exp(-nu * k2 * dt * 0.5);
        H[M + m] = exp(-kappa * k2 * dt * 0.5);
      }
  for (int s = 0; s < nsteps; s++) {
    int rc = oracle_rbc_rhs(st, nh, n);
    if (rc) return rc;
    if (scheme == 0) {
      for (int f = 0; f < 4; f++)
        for (long m = 0; m < M; m++) {
          long i = f * M + m, e = (f == 3 ? M : 0) + m;
          us[i] = E[e] * (st[i] + dt * nh[i]);
        }
      oracle_dealias(us, 4, n);
      rc = oracle_rbc_rhs(us, nh, n);
      if (rc) return rc;
      for (int f = 0; f < 4; f++)
        for (long m = 0; m < M; m++) {
          long i = f * M + m, e = (f == 3 ? M : 0) + m;
          st[i] = 0.5 * E[e] * st[i] + 0.5 * (us[i] + dt * nh[i]);
        }
      oracle_dealias(st, 4, n);
      continue;
    }
    for (int f = 0; f < 4; f++)
      for (long m = 0; m < M; m++) {
        long i = f * M + m, e = (f == 3 ? M : 0) + m;
        acc[i] = E[e] * st[i] + dt / 6.0 * E[e] * nh[i];
        us[i] = H[e] * (st[i] + 0.5 * dt * nh[i]);
      }
    oracle_dealias(us, 4, n);
    rc = oracle_rbc_rhs(us, nh, n);
    if (rc) return rc;
    for (int f = 0; f < 4; f++)
      for (long m = 0; m < M; m++) {
        long i = f * M + m, e = (f == 3 ? M : 0) + m;
        acc[i] += dt / 3.0 * H[e] * nh[i];
        us[i] = H[e] * st[i] + 0.5 * dt * nh[i];
      }
    oracle_dealias(us, 4, n);
    rc = oracle_rbc_rhs(us, nh, n);
    if (rc) return rc;
    for (int f = 0; f < 4; f++)
      for (long m = 0; m < M; m++) {
        long i = f * M + m, e = (f == 3 ? M : 0) + m;
        acc[i] += dt / 3.0 * H[e] * nh[i];
        us[i] = E[e] * st[i] + dt * H[e] * nh[i];
      }
    oracle_dealias(us, 4, n);
    rc = oracle_rbc_rhs(us, nh, n);
    if (rc) return rc;
    for (long i = 0; i < 4 * M; i++) st[i] = acc[i] + dt / 6.0 * nh[i];
    oracle_dealias(st, 4, n);
  }
  free(us);
  free(nh);
  free(acc);
  free(E);
  free(H);
  return 0;
}

/* ------------------------------------------ Rayleigh-Benard (SFF plates) -- */
/* Eqs. (12)-(14) between free-slip, isothermal plates (the SFF basis,
 * Sec. 2.2): the wall-normal axis is x on [0, pi] (the n points of the sine
 * and cosine bases), y and z are 2 pi-periodic, gravity along x.  State
 * s[4][n][n][n/2+1]: u_x and theta in the sine basis along x (index a is
 * k_x = a + 1: u_x = theta = 0 on the plates), u_y, u_z in the cosine basis
 * (index a is k_x = a: d_x u_y = d_x u_z = 0 on the plates); Fourier along
 * y and z as everywhere.  Right-hand side without diffusion:
 *   N_u = P[u x omega + theta x],  N_theta = -div(u theta) + u_x,
 * 2/3-truncated (3 k_x < 2n on the wall-normal axis, 3|k| < n on the
 * periodic ones); P subtracts the gradient of a cosine-basis pressure. */
static const int kSFF_S[3] = {ORACLE_SINE, ORACLE_FOURIER, ORACLE_FOURIER};
static const int kSFF_C[3] = {ORACLE_COSINE, ORACLE_FOURIER, ORACLE_FOURIER};

static int sff_kept(long kx, long ky, long kz, long n) { return 3 * kx < 2 * n && 3 * labs(ky) < n && 3 * kz < n; }

/* zero the modes outside the truncated set; sine fields index a is k_x = a + 1 */
static void sff_dealias(cplx *f, int sine, int n) {
  const long N = n, HZ = n / 2 + 1;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++)
        if (!sff_kept(sine ? a + 1 : a, kxy(b, N), c, N)) f[(a * N + b) * HZ + c] = 0;
}

int oracle_rbc_sff_rhs(const cplx *st, cplx *out, int n) {
  if (!is_pow2(n) || n < 2) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  const cplx *ux = st, *uy = st + M, *uz = st + 2 * M, *th = st + 3 * M;
  cplx *w = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M); /* omega_x (cos), omega_y, omega_z (sin) */
  double *r = (double *)malloc(sizeof(double) * 7 * (size_t)R);
  double *pr = (double *)malloc(sizeof(double) * (size_t)R);
  cplx *ph = (cplx *)malloc(sizeof(cplx) * 6 * (size_t)M);
  if (!w || !r || !pr || !ph) return -2;
  /* omega = curl u in the mixed basis: d_x of a sine coefficient s_k is the
   * cosine coefficient k s_k, d_x of a cosine coefficient c_k the sine
   * coefficient -k c_k */
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c, up = ((a + 1) * N + b) * HZ + c;
        double ky = (double)kder(kxy(b, N), N), kz = (double)kder(c, N), kxs = (double)(a + 1);
        w[idx] = I * ky * uz[idx] - I * kz * uy[idx];                       /* cos: d_y u_z - d_z u_y */
        cplx uzc = (a + 1 < N) ? uz[up] : 0, uyc = (a + 1 < N) ? uy[up] : 0; /* cosine mode k_x = a + 1 */
        w[M + idx] = I * kz * ux[idx] + kxs * uzc;                          /* sin: d_z u_x - d_x u_z */
        w[2 * M + idx] = -kxs * uyc - I * ky * ux[idx];                     /* sin: d_x u_y - d_y u_x */
      }
  /* real space: r = u_x, u_y, u_z, omega_x, omega_y, omega_z, theta */
  oracle_itransform3(ux, r, n, n, n, kSFF_S);
  oracle_itransform3(uy, r + R, n, n, n, kSFF_C);
  oracle_itransform3(uz, r + 2 * R, n, n, n, kSFF_C);
  oracle_itransform3(w, r + 3 * R, n, n, n, kSFF_C);
  oracle_itransform3(w + M, r + 4 * R, n, n, n, kSFF_S);
  oracle_itransform3(w + 2 * M, r + 5 * R, n, n, n, kSFF_S);
  oracle_itransform3(th, r + 6 * R, n, n, n, kSFF_S);
  /* products back to the mixed basis: (u x omega)_x, u_y theta, u_z theta in
   * sine; (u x omega)_y, (u x omega)_z, u_x theta in cosine */
  const double *rx = r, *ry = r + R, *rz = r + 2 * R, *wx = r + 3 * R, *wy = r + 4 * R, *wz = r + 5 * R,
               *tt = r + 6 * R;
  for (int q = 0; q < 6; q++) {
    for (long x = 0; x < R; x++) {
      double v = 0.0;
      switch (q) {
        case 0: v = ry[x] * wz[x] - rz[x] * wy[x]; break;
        case 1: v = rz[x] * wx[x] - rx[x] * wz[x]; break;
        case 2: v = rx[x] * wy[x] - ry[x] * wx[x]; break;
        case 3: v = rx[x] * tt[x]; break;
        case 4: v = ry[x] * tt[x]; break;
        default: v = rz[x] * tt[x]; break;
      }
      pr[x] = v;
    }
    const int sine = (q == 0 || q == 4 || q == 5);
    oracle_transform3(pr, ph + q * M, n, n, n, sine ? kSFF_S : kSFF_C);
  }
  /* v = u x omega + theta x, then v - grad p with the cosine pressure
   * p = -div v / k^2 (div v in the cosine basis: k_x v_x + i k_y v_y + i k_z v_z) */
  cplx *vx = out, *vy = out + M, *vz = out + 2 * M;
  for (long i = 0; i < M; i++) {
    vx[i] = ph[i] + th[i];
    vy[i] = ph[M + i];
    vz[i] = ph[2 * M + i];
  }
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        double kx = (double)a, ky = (double)kxy(b, N), kz = (double)c;
        double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0.0) continue;
        long sidx = ((a - 1) * N + b) * HZ + c; /* sine index of k_x = a */
        cplx vxs = (a >= 1) ? vx[sidx] : 0;
        cplx div = kx * vxs + I * ky * vy[idx] + I * kz * vz[idx];
        cplx pc = -div / k2;
        vy[idx] -= I * ky * pc;
        vz[idx] -= I * kz * pc;
        if (a >= 1) vx[sidx] += kx * pc; /* d_x p has the sine coefficient -k_x p */
      }
  /* the sine mode k_x = n has no cosine partner: it is outside the kept set */
  /* N_theta = -(d_x(u_x theta) + d_y(u_y theta) + d_z(u_z theta)) + u_x */
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c, up = ((a + 1) * N + b) * HZ + c;
        double ky = (double)kder(kxy(b, N), N), kz = (double)kder(c, N), kxs = (double)(a + 1);
        cplx cxt = (a + 1 < N) ? ph[3 * M + up] : 0;
        cplx div = -kxs * cxt + I * ky * ph[4 * M + idx] + I * kz * ph[5 * M + idx];
        out[3 * M + idx] = -div + ux[idx];
      }
  sff_dealias(vx, 1, n);
  sff_dealias(vy, 0, n);
  sff_dealias(vz, 0, n);
  sff_dealias(out + 3 * M, 1, n);
  free(w);
  free(r);
  free(pr);
  free(ph);
  return 0;
}

/* nsteps of RK2 (scheme 0) or RK4 (scheme 1) for the SFF state, as
 * oracle_rbc_step, with k^2 = k_x^2 + k_y^2 + k_z^2 and k_x per field's basis. */
int oracle_rbc_sff_step(cplx *st, int n, double Ra, double Pr, double dt, int nsteps, int scheme) {
  if (!is_pow2(n) || n < 2 || Ra <= 0.0 || Pr <= 0.0 || (scheme != 0 && scheme != 1)) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  const double nu = sqrt(Pr / Ra), kappa = 1.0 / sqrt(Ra * Pr);
  cplx *us = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)M);
  cplx *nh = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)M);
  cplx *acc = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)M);
  double *E = (double *)malloc(sizeof(double) * 4 * (size_t)M);
  double *H = (double *)malloc(sizeof(double) * 4 * (size_t)M);
  if (!us || !nh || !acc || !E || !H) return -2;
  for (int f = 0; f < 4; f++) {
    const int sine = (f == 0 || f == 3);
    const double d = (f == 3) ? kappa : nu;
    for (long a = 0; a < N; a++)
      for (long b = 0; b < N; b++)
        for (long c = 0; c < HZ; c++) {
          double kx = (double)(sine ? a + 1 : a), ky = (double)kxy(b, N), kz = (double)c;
          double k2 = kx * kx + ky * ky + kz * kz;
          long i = f * M + (a * N + b) * HZ + c;
          E[i] = exp(-d * k2 * dt);
          H[i] = exp(-d * k2 * dt * 0.5);
        }
  }
  for (int s = 0; s < nsteps; s++) {
    int rc = oracle_rbc_sff_rhs(st, nh, n);
    if (rc) return rc;
    if (scheme == 0) {
      for (long i = 0; i < 4 * M; i++) us[i] = E[i] * (st[i] + dt * nh[i]);
      rc = oracle_rbc_sff_rhs(us, nh, n);
      if (rc) return rc;
      for (long i = 0; i < 4 * M; i++) st[i] = 0.5 * E[i] * st[i] + 0.5 * (us[i] + dt * nh[i]);
      continue;
    }
    for (long i = 0; i < 4 * M; i++) {
      acc[i] = E[i] * st[i] + dt / 6.0 * E[i] * nh[i];
      us[i] = H[i] * (st[i] + 0.5 * dt * nh[i]);
    }
    rc = oracle_rbc_sff_rhs(us, nh, n);
    if (rc) return rc;
    for (long i = 0; i < 4 * M; i++) {
      acc[i] += dt / 3.0 * H[i] * nh[i];
      us[i] = H[i] * st[i] + 0.5 * dt * nh[i];
    }
    rc = oracle_rbc_sff_rhs(us, nh, n);
    if (rc) return rc;
    for (long i = 0; i < 4 * M; i++) {
      acc[i] += dt / 3.0 * H[i] * nh[i];
      us[i] = E[i] * st[i] + dt * H[i] * nh[i];
    }
    rc = oracle_rbc_sff_rhs(us, nh, n);
    if (rc) return rc;
    for (long i = 0; i < 4 * M; i++) st[i] = acc[i] + dt / 6.0 * nh[i];
  }
  free(us);
  free(nh);
  free(acc);
  free(E);
  free(H);
  return 0;
}

/* Shell index K = nint(|k|); |k| is never a half-integer for integer k. */
static long shell_of(long k2) { return (long)floor(sqrt((double)k2) + 0.5); }

int oracle_diag(const cplx *u, int n, double nu, double *E, double *eps, double *EK,
                int kmax) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  double e = 0.0, d = 0.0;
  if (EK)
    for (int K = 0; K <= kmax; K++) EK[K] = 0.0;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        long kx = kxy(a, N), ky = kxy(b, N), k2 = kx * kx + ky * ky + c * c;
        double em = 0.5 * mode_weight(c, N) *
                    (sq(u[idx]) + sq(u[M + idx]) + sq(u[2 * M + idx]));
        e += em;
        d += 2.0 * nu * (double)k2 * em;
        long K = shell_of(k2);
        if (EK && K <= kmax) EK[K] += em;
      }
  if (E) *E = e;
  if (eps) *eps = d;
  return 0;
}

double oracle_transfer(const cplx *u, const cplx *nh, int n) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  double t = 0.0;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        for (int f = 0; f < 3; f++)
          t += mode_weight(c, N) * creal(conj(u[f * M + idx]) * nh[f * M + idx]);
      }
  return t;
}

/* Energy transfer spectrum of the nonlinear term (the scale-by-scale
 * analysis of Sec. 1 and Sec. 7): T(K) = sum over the shell K = nint|k| of
 * w Re(conj(u) . N), w = 1 on k_z = 0 and k_z = n/2, else 2.  The flux
 * through K is Pi(K) = -sum_{K' <= K} T(K'). */
int oracle_transfer_spectrum(const cplx *u, const cplx *nh, int n, double *T, int kmax) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  for (int K = 0; K <= kmax; K++) T[K] = 0.0;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long idx = (a * N + b) * HZ + c;
        long kx = kxy(a, N), ky = kxy(b, N), k2 = kx * kx + ky * ky + c * c;
        double t = 0.0;
        for (int f = 0; f < 3; f++) t += creal(conj(u[f * M + idx]) * nh[f * M + idx]);
        long K = shell_of(k2);
        if (K <= kmax) T[K] += mode_weight(c, N) * t;
      }
  return 0;
}

/* Shell-to-shell energy transfer (Tarang's scale-by-scale analysis, Sec. 1, Sec. 3):
 * shell i holds the modes with bounds[i] <= nint|k| < bounds[i+1], and
 *   T[r * nshells + g] = -<u_r . (u . grad) u_g>
 * is the rate at which shell r (receiver) gains energy from shell g (giver)
 * through the advection by the whole field u.  Pseudo-spectral evaluation:
 * for each giver, the gradient i k_j u_g,i of its modes and u itself go to
 * real space, the product u_j d_j u_g,i comes back, and the receiver sums
 * w Re(conj(u_r) . product) over its modes. */
int oracle_shell_transfer(const cplx *u, int n, int nshells, const int *bounds, double *T) {
  if (!is_pow2(n) || n < 2 || nshells < 1) return -1;
  for (int i = 0; i < nshells; i++)
    if (bounds[i] < 0 || bounds[i + 1] <= bounds[i]) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  int *sh = (int *)malloc(sizeof(int) * (size_t)M); /* shell of each mode, -1 for none */
  double *ur = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  double *gr = (double *)malloc(sizeof(double) * 9 * (size_t)R);
  double *pr = (double *)malloc(sizeof(double) * (size_t)R);
  cplx *gh = (cplx *)malloc(sizeof(cplx) * (size_t)M);
  cplx *ph = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  if (!sh || !ur || !gr || !pr || !gh || !ph) return -2;
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long kx = kxy(a, N), ky = kxy(b, N), K = shell_of(kx * kx + ky * ky + c * c);
        int s = -1;
        for (int i = 0; i < nshells; i++)
          if (K >= bounds[i] && K < bounds[i + 1]) s = i;
        sh[(a * N + b) * HZ + c] = s;
      }
  for (int f = 0; f < 3; f++) oracle_irfft3(u + f * M, ur + f * R, n, n, n);
  for (long i = 0; i < (long)nshells * nshells; i++) T[i] = 0.0;
  for (int g = 0; g < nshells; g++) {
    /* d_j u_g,i in real space, gr[(i * 3 + j) R + x] */
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        for (long a = 0; a < N; a++)
          for (long b = 0; b < N; b++)
            for (long c = 0; c < HZ; c++) {
              long idx = (a * N + b) * HZ + c;
              double k[3] = {(double)kder(kxy(a, N), N), (double)kder(kxy(b, N), N),
                             (double)kder(c, N)};
              gh[idx] = (sh[idx] == g) ? I * k[j] * u[i * M + idx] : 0.0;
            }
        oracle_irfft3(gh, gr + (i * 3 + j) * R, n, n, n);
      }
    /* (u . grad) u_g back to Fourier space */
    for (int i = 0; i < 3; i++) {
      for (long x = 0; x < R; x++) {
        double s = 0.0;
        for (int j = 0; j < 3; j++) s += ur[j * R + x] * gr[(i * 3 + j) * R + x];
        pr[x] = s;
      }
      oracle_rfft3(pr, ph + i * M, n, n, n);
    }
    /* every receiver's share */
    for (long a = 0; a < N; a++)
      for (long b = 0; b < N; b++)
        for (long c = 0; c < HZ; c++) {
          long idx = (a * N + b) * HZ + c;
          int r = sh[idx];
          if (r < 0) continue;
          double t = 0.0;
          for (int f = 0; f < 3; f++) t += creal(conj(u[f * M + idx]) * ph[f * M + idx]);
          T[(long)r * nshells + g] -= mode_weight(c, N) * t;
        }
  }
  free(sh);
  free(ur);
  free(gr);
  free(pr);
  free(gh);
  free(ph);
  return 0;
}

/* ----------------------------------------------------- initial fields ---- */

static int ic_from_real(const double *ur, cplx *uhat, int n) {
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  for (int f = 0; f < 3; f++) {
    int rc = oracle_rfft3(ur + f * R, uhat + f * M, n, n, n);
    if (rc) return rc;
  }
  return 0;
}

int oracle_ic_taylor_green(cplx *uhat, int n) {
  if (!ok_grid(n)) return -1;
  const long N = n, R = N * N * N;
  double *ur = (double *)calloc(3 * (size_t)R, sizeof(double));
  if (!ur) return -2;
  for (long i = 0; i < N; i++)
    for (long j = 0; j < N; j++)
      for (long l = 0; l < N; l++) {
        double x = TWO_PI * (double)i / (double)N, y = TWO_PI * (double)j / (double)N;
        long r = (i * N + j) * N + l;
        ur[r] = sin(x) * cos(y);
        ur[R + r] = -cos(x) * sin(y);
      }
  int rc = ic_from_real(ur, uhat, n);
  free(ur);
  return rc;
}

int oracle_ic_abc(cplx *uhat, int n) {
  if (!ok_grid(n)) return -1;
  const long N = n, R = N * N * N;
  double *ur = (double *)malloc(3 * sizeof(double) * (size_t)R);
  if (!ur) return -2;
  for (long i = 0; i < N; i++)
    for (long j = 0; j < N; j++)
      for (long l = 0; l < N; l++) {
        double x = TWO_PI * (double)i / (double)N, y = TWO_PI * (double)j / (double)N,
               z = TWO_PI * (double)l / (double)N;
        long r = (i * N + j) * N + l;
        ur[r] = sin(z) + cos(y);
        ur[R + r] = sin(x) + cos(z);
        ur[2 * R + r] = sin(y) + cos(x);
      }
  int rc = ic_from_real(ur, uhat, n);
  free(ur);
  return rc;
}

/* Make the planes k_z = 0 and k_z = N/2 exactly Hermitian:
 * f(-kx,-ky) = conj f(kx,ky), by averaging each pair. */
static void hermitianize(cplx *f, int n) {
  const long N = n, HZ = n / 2 + 1;
  long planes[2] = {0, N / 2};
  for (int pl = 0; pl < 2; pl++) {
    long c = planes[pl];
    for (long a = 0; a < N; a++)
      for (long b = 0; b < N; b++) {
        long a2 = (N - a) % N, b2 = (N - b) % N;
        long i1 = (a * N + b) * HZ + c, i2 = (a2 * N + b2) * HZ + c;
        if (i2 < i1) continue;
        if (i1 == i2) {
          f[i1] = creal(f[i1]);
        } else {
          cplx avg = 0.5 * (f[i1] + conj(f[i2]));
          f[i1] = avg;
          f[i2] = conj(avg);
        }
      }
  }
}

int oracle_ic_random(const double *normals, cplx *uhat, int n, double k0, double E0) {
  if (!ok_grid(n) || k0 <= 0.0 || E0 <= 0.0) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ;
  int rc = ic_from_real(normals, uhat, n);
  if (rc) return rc;
  oracle_dealias(uhat, 3, n);
  oracle_project(uhat, n);
  for (int f = 0; f < 3; f++) hermitianize(uhat + f * M, n);
  const long KMAX = shell_of(3 * (N / 2) * (N / 2)) + 1;
  double *eK = (double *)calloc((size_t)KMAX + 1, sizeof(double));
  if (!eK) return -2;
  oracle_diag(uhat, n, 0.0, NULL, NULL, eK, (int)KMAX);
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        long kx = kxy(a, N), ky = kxy(b, N), k2 = kx * kx + ky * ky + c * c;
        long K = shell_of(k2);
        long idx = (a * N + b) * HZ + c;
        double s = 0.0;
        if (K >= 1 && eK[K] > 0.0) {
          double Kd = (double)K;
          double target = Kd * Kd * Kd * Kd * exp(-2.0 * (Kd / k0) * (Kd / k0));
          s = sqrt(target / eK[K]);
        }
        for (int f = 0; f < 3; f++) uhat[f * M + idx] *= s;
      }
  double E = 0.0;
  oracle_diag(uhat, n, 0.0, &E, NULL, NULL, 0);
  double g = sqrt(E0 / E);
  for (long m = 0; m < 3 * M; m++) uhat[m] *= g;
  free(eK);
  return 0;
}

/* ------------------------------------------------------------ closure ---- */

static const int kPairI[6] = {0, 1, 2, 0, 0, 1};
static const int kPairJ[6] = {0, 1, 2, 1, 2, 2};

int oracle_box_filter(const double *u, int n, int factor, double *ubar, double *tau) {
  if (n < 1 || factor < 1 || n % factor) return -1;
  const long N = n, F = factor, m = n / factor, R = N * N * N, Mc = m * m * m;
  const double cnt = (double)(F * F * F);
  for (long ci = 0; ci < m; ci++)
    for (long cj = 0; cj < m; cj++)
      for (long ck = 0; ck < m; ck++) {
        double s[3] = {0, 0, 0}, pr[6] = {0, 0, 0, 0, 0, 0};
        for (long a = 0; a < F; a++)
          for (long b = 0; b < F; b++)
            for (long c = 0; c < F; c++) {
              const long idx = ((ci * F + a) * N + (cj * F + b)) * N + (ck * F + c);
              for (int q = 0; q < 3; q++) s[q] += u[q * R + idx];
              for (int p = 0; p < 6; p++) pr[p] += u[kPairI[p] * R + idx] * u[kPairJ[p] * R + idx];
            }
        const long cell = (ci * m + cj) * m + ck;
        double mean[3];
        for (int q = 0; q < 3; q++) {
          mean[q] = s[q] / cnt;
          ubar[q * Mc + cell] = mean[q];
        }
        for (int p = 0; p < 6; p++)
          tau[p * Mc + cell] = pr[p] / cnt - mean[kPairI[p]] * mean[kPairJ[p]];
      }
  return 0;
}

/* The subgrid stress of the coarse solver as it computes (the closure's
 * training target): the coarse grid keeps only the 2/3 set of the filtered
 * field, ubar_T = T ubar, and forms its products dealiased, so the exact
 * coarse equations for ubar_T carry
 *   tau_les_ij = T[ <u_i u_j> - ubar_T,i ubar_T,j ],
 * with <u_i u_j> = tau_ij + ubar_i ubar_j (the box-filtered products) and T
 * the 2/3 truncation on the m^3 grid.  In: ubar[3][m^3], tau[6][m^3]; out:
 * tau_les[6][m^3] (pairs xx, yy, zz, xy, xz, yz). */
int oracle_les_stress(const double *ubar, const double *tau, int m, double *out) {
  if (!ok_grid(m)) return -1;
  const long Mn = m, HZ = m / 2 + 1, M = Mn * Mn * HZ, R = Mn * Mn * Mn;
  cplx *sp = (cplx *)malloc(sizeof(cplx) * (size_t)M);
  double *ut = (double *)malloc(sizeof(double) * 3 * (size_t)R);
  double *pr = (double *)malloc(sizeof(double) * (size_t)R);
  if (!sp || !ut || !pr) return -2;
  /* ubar_T = T ubar */
  for (int q = 0; q < 3; q++) {
    oracle_rfft3(ubar + q * R, sp, m, m, m);
    oracle_dealias(sp, 1, m);
    oracle_irfft3(sp, ut + q * R, m, m, m);
  }
  for (int p = 0; p < 6; p++) {
    const int i = kPairI[p], j = kPairJ[p];
    for (long x = 0; x < R; x++)
      pr[x] = tau[p * R + x] + ubar[i * R + x] * ubar[j * R + x] - ut[i * R + x] * ut[j * R + x];
    oracle_rfft3(pr, sp, m, m, m);
    oracle_dealias(sp, 1, m);
    oracle_irfft3(sp, out + p * R, m, m, m);
  }
  free(sp);
  free(ut);
  free(pr);
  return 0;
}

int oracle_gradient(const double *u, int m, double *A) {
  if (!is_pow2(m) || m < 2) return -1;
  const long Mn = m, HZ = m / 2 + 1, M = Mn * Mn * HZ, R = Mn * Mn * Mn;
  cplx *uh = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)M);
  cplx *g = (cplx *)malloc(sizeof(cplx) * (size_t)M);
  if (!uh || !g) return -2;
  for (int c = 0; c < 3; c++) oracle_rfft3(u + c * R, uh + c * M, m, m, m);
  oracle_dealias(uh, 3, m);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      for (long a = 0; a < Mn; a++)
        for (long b = 0; b < Mn; b++)
          for (long c = 0; c < HZ; c++) {
            const long idx = (a * Mn + b) * HZ + c;
            const long k[3] = {kder(kxy(a, Mn), Mn), kder(kxy(b, Mn), Mn), kder(c, Mn)};
            g[idx] = I * (double)k[j] * uh[i * M + idx];
          }
      oracle_irfft3(g, A + (i * 3 + j) * R, m, m, m);
    }
  free(uh);
  free(g);
  return 0;
}

static void mat3_mul(const double a[9], const double b[9], double c[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double s = 0;
      for (int k = 0; k < 3; k++) s += a[i * 3 + k] * b[k * 3 + j];
      c[i * 3 + j] = s;
    }
}

static double mat3_trace(const double a[9]) { return a[0] + a[4] + a[8]; }

void oracle_invariants(const double A[9], double inv[5]) {
  double S[9], R[9], S2[9], R2[9], S3[9], R2S[9], R2S2[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      S[i * 3 + j] = 0.5 * (A[i * 3 + j] + A[j * 3 + i]);
      R[i * 3 + j] = 0.5 * (A[i * 3 + j] - A[j * 3 + i]);
    }
  mat3_mul(S, S, S2);
  mat3_mul(R, R, R2);
  mat3_mul(S2, S, S3);
  mat3_mul(R2, S, R2S);
  mat3_mul(R2, S2, R2S2);
  inv[0] = mat3_trace(S2);
  inv[1] = mat3_trace(R2);
  inv[2] = mat3_trace(S3);
  inv[3] = mat3_trace(R2S);
  inv[4] = mat3_trace(R2S2);
}

/* Cyclic Jacobi (Golub and Van Loan, sym. Schur): zero a_pq with the rotation
 * t = sign(theta)/(|theta| + sqrt(1 + theta^2)), theta = (a_qq - a_pp)/(2 a_pq). */
void oracle_sym_eig3(const double S[9], double lam[3], double Q[9]) {
  double a[9], v[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  memcpy(a, S, sizeof(a));
  for (int sweep = 0; sweep < 50; sweep++) {
    const double off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
    if (off == 0.0) break;
    const int pq[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; r++) {
      const int p = pq[r][0], q = pq[r][1];
      const double apq = a[p * 3 + q];
      if (apq == 0.0) continue;
      const double theta = (a[q * 3 + q] - a[p * 3 + p]) / (2.0 * apq);
      const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
      const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      double Jm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Jt[9], tmp[9];
      Jm[p * 3 + p] = c;
      Jm[q * 3 + q] = c;
      Jm[p * 3 + q] = s;
      Jm[q * 3 + p] = -s;
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Jt[i * 3 + j] = Jm[j * 3 + i];
      mat3_mul(Jt, a, tmp);
      mat3_mul(tmp, Jm, a);
      mat3_mul(v, Jm, tmp);
      memcpy(v, tmp, sizeof(v));
    }
  }
  int order[3] = {0, 1, 2};
  for (int i = 0; i < 3; i++)
    for (int j = i + 1; j < 3; j++)
      if (a[order[j] * 4] > a[order[i] * 4]) {
        int t = order[i];
        order[i] = order[j];
        order[j] = t;
      }
  for (int k = 0; k < 3; k++) {
    const int src = order[k];
    lam[k] = a[src * 4];
    int big = 0;
    for (int i = 1; i < 3; i++)
      if (fabs(v[i * 3 + src]) > fabs(v[big * 3 + src])) big = i;
    const double sg = v[big * 3 + src] < 0 ? -1.0 : 1.0;
    for (int i = 0; i < 3; i++) Q[i * 3 + k] = sg * v[i * 3 + src];
  }
}

/* round to bfloat16 (nearest even) of the FP32 value */
static double bf16r(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static const int kMlpDims[5] = {5, 64, 64, 64, 6};

/* offsets of W_l and b_l in the flat parameter vector */
static void mlp_offsets(int l, long *w, long *b) {
  long o = 0;
  for (int i = 0; i < l; i++) o += (long)kMlpDims[i + 1] * kMlpDims[i] + kMlpDims[i + 1];
  *w = o;
  *b = o + (long)kMlpDims[l + 1] * kMlpDims[l];
}

/* forward for one sample; acts[l] = input of layer l (as used), z[l] = pre-activation */
static void mlp_sample(const double *prm, const double *x, int bf16, double acts[4][64], double z[4][64]) {
  for (int i = 0; i < 5; i++) acts[0][i] = bf16 ? bf16r(x[i]) : x[i];
  for (int l = 0; l < 4; l++) {
    long wo, bo;
    mlp_offsets(l, &wo, &bo);
    const int din = kMlpDims[l], dout = kMlpDims[l + 1];
    for (int o = 0; o < dout; o++) {
      double s = prm[bo + o];
      for (int i = 0; i < din; i++) s += prm[wo + (long)o * din + i] * acts[l][i];
      z[l][o] = s;
      if (l < 3) {
        const double h = tanh(s);
        acts[l + 1][o] = bf16 ? bf16r(h) : h;
      }
    }
  }
}

int oracle_mlp_forward(const double *params, const double *x, double *y, int B, int bf16_acts) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; b++) {
    double acts[4][64], z[4][64];
    mlp_sample(params, x + 5L * b, bf16_acts, acts, z);
    for (int o = 0; o < 6; o++) y[6L * b + o] = z[3][o];
  }
  return 0;
}

double oracle_mlp_loss_grad(const double *params, const double *x, const double *t, int B,
                            int bf16_acts, double *grad) {
  for (int i = 0; i < ORACLE_MLP_NPARAMS; i++) grad[i] = 0.0;
  double loss = 0.0;
  const double scale = 1.0 / (6.0 * (double)B);
  for (int b = 0; b < B; b++) {
    double acts[4][64], z[4][64], d[64], dn[64];
    mlp_sample(params, x + 5L * b, bf16_acts, acts, z);
    for (int o = 0; o < 6; o++) {
      const double e = z[3][o] - t[6L * b + o];
      loss += e * e * scale;
      d[o] = 2.0 * e * scale;  /* dL/dz of the output layer */
    }
    for (int l = 3; l >= 0; l--) {
      long wo, bo;
      mlp_offsets(l, &wo, &bo);
      const int din = kMlpDims[l], dout = kMlpDims[l + 1];
      for (int o = 0; o < dout; o++) {
        grad[bo + o] += d[o];
        for (int i = 0; i < din; i++) grad[wo + (long)o * din + i] += d[o] * acts[l][i];
      }
      if (l > 0) {
        /* back through the layer input acts[l] = tanh(z[l-1]); derivative from the
           stored activation 1 - a^2 */
        for (int i = 0; i < din; i++) {
          double s = 0.0;
          for (int o = 0; o < dout; o++) s += params[wo + (long)o * din + i] * d[o];
          dn[i] = s * (1.0 - acts[l][i] * acts[l][i]);
        }
        memcpy(d, dn, sizeof(double) * (size_t)din);
      }
    }
  }
  return loss;
}

void oracle_adam(double *params, double *m, double *v, const double *grad, int nparam, int step,
                 double lr, double beta1, double beta2, double eps) {
  const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
  for (int i = 0; i < nparam; i++) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

int oracle_sgs_force(const double *tau, int n, cplx *fhat) {
  if (!is_pow2(n) || n < 2) return -1;
  const long N = n, HZ = n / 2 + 1, M = N * N * HZ, R = N * N * N;
  cplx *th = (cplx *)malloc(sizeof(cplx) * 6 * (size_t)M);
  if (!th) return -2;
  for (int p = 0; p < 6; p++) oracle_rfft3(tau + p * R, th + p * M, n, n, n);
  /* component index of the symmetric pair (i, j) */
  const int pidx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (long a = 0; a < N; a++)
    for (long b = 0; b < N; b++)
      for (long c = 0; c < HZ; c++) {
        const long idx = (a * N + b) * HZ + c;
        const double k[3] = {(double)kder(kxy(a, N), N), (double)kder(kxy(b, N), N), (double)kder(c, N)};
        for (int i = 0; i < 3; i++) {
          cplx s = 0;
          for (int j = 0; j < 3; j++) s += k[j] * th[pidx[i][j] * M + idx];
          fhat[i * M + idx] = -I * s;
        }
      }
  oracle_dealias(fhat, 3, n);
  oracle_project(fhat, n);
  free(th);
  return 0;
}
