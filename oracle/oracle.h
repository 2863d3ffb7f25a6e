/* Plain, slow FP64 CPU oracle for the FFTK/Tarang hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the product (libfftk) never does, and the
 * two share no code.
 *
 * Conventions (Sec. 2.1, Eq. (1) and the Fourier basis of Eq. (2a)):
 *   inverse  f(x) = sum_k fhat(k) exp(+i k.x)            (no factor)
 *   forward  fhat(k) = (1/(Nx Ny Nz)) sum_x f(x) exp(-i k.x)
 * with x = 2 pi (i/Nx, j/Ny, l/Nz) on a 2 pi-periodic box.
 * Real arrays are double[Nx][Ny][Nz] (z fastest); half spectra are
 * double complex[Nx][Ny][Nz/2+1] (axes not exchanged, as in Appendix A).
 * Index a on an x or y axis stands for k = a if a <= N/2 else a - N; on z, k = c.
 */
#ifndef FFTK_ORACLE_H
#define FFTK_ORACLE_H

#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef double _Complex ocplx;

/* OpenMP threads the oracle uses for independent lines (1 without OpenMP). */
int oracle_threads(void);

/* 1D transforms, out[k] = sum_j in[j] exp(sign 2 pi i j k / n). */
int oracle_fft1d(const ocplx *in, ocplx *out, long n, int sign);   /* recursive radix-2, n = 2^m */
int oracle_dft1d(const ocplx *in, ocplx *out, long n, int sign);   /* O(n^2) definition, any n */

/* Sine and cosine bases (Sec. 2.1, Eq. (2b, 2c)) on the n points
 * s_j = (j + 1/2) pi / n of [0, pi]:
 *   inverse (dir +1)  f(s_j) = sum_k fhat_k 2 sin(k s_j), k = 1..n (stored at k-1),
 *                     or 2 cos(k s_j), k = 0..n-1 (stored at k);
 *   forward (dir -1)  its inverse, fhat_k = (c_k/n) sum_j f(s_j) sin(k s_j) (cos),
 *                     c_k = 1/2 for the cosine k = 0 and the sine k = n, else 1.
 * By the definitions, O(n^2), complex-linear, any n >= 1. */
#define ORACLE_FOURIER 0
#define ORACLE_SINE 1
#define ORACLE_COSINE 2
int oracle_sc1d(const ocplx *in, ocplx *out, long n, int kind, int dir);
/* 3D transforms with a basis per axis (kind[3] for x, y, z; Fourier axes
 * trailing: FFF, SFF, SSF, SSS), passes in the paper's order (forward z, y,
 * x; inverse x, y, z).  Fourier axes as in oracle_rfft3 (1/n per forward
 * axis).  Spectrum: complex [nx][ny][hz], hz = nz/2+1 for a Fourier z axis
 * (half spectrum) else nz (real coefficients, imaginary parts 0). */
int oracle_transform3(const double *in, ocplx *out, int nx, int ny, int nz, const int kind[3]);
int oracle_itransform3(const ocplx *in, double *out, int nx, int ny, int nz, const int kind[3]);
/* One coefficient (a, b, c) of oracle_transform3 of FP32 input by its
 * definition, O(nx ny nz); out = (re, im). */
int oracle_transform3_coeff_f32(const float *in, int nx, int ny, int nz, const int kind[3], int a, int b, int c,
                                double *out);

/* 3D transforms in the paper's pass order (Sec. 3): forward z r2c, y c2c, x c2c
 * then the 1/N^3 factor; inverse x c2c, y c2c, z c2r.  Every dimension 2^m
 * (lines by the radix-2 FFT) or 3 * 2^m (lines by the DFT's definition). */
int oracle_rfft3(const double *in, ocplx *out, int nx, int ny, int nz);
int oracle_irfft3(const ocplx *in, double *out, int nx, int ny, int nz);

/* One forward coefficient by the direct sum over all grid points (float input). */
void oracle_rfft3_coeff_f32(const float *in, int nx, int ny, int nz, int a, int b, int c,
                            double *re_im);
/* One inverse output point by the direct sum over the stored half spectrum
 * (complex64 input), weights 1 on the planes c = 0 and c = Nz/2, 2 elsewhere,
 * real part taken: the line-wise "extend, then take the real part" result. */
double oracle_irfft3_point_c64(const float *in_c64, int nx, int ny, int nz, int i, int j, int l);

/* Pseudo-spectral Navier-Stokes (Sec. 2.2, Eqs. (7)-(8)), 2 pi-periodic cubic box,
 * velocity state uhat[3][n][n][n/2+1]. */
typedef struct {
  double nu;        /* kinematic viscosity */
  double dt;        /* time step */
  double force_eps; /* constant injected power; 0 = unforced */
  int force_k2min;  /* forced modes: force_k2min <= |k|^2 <= force_k2max */
  int force_k2max;
} oracle_ns_params;

/* Nonlinear term in rotational form: P[ F(u x omega) ] dealiased (2/3 rule),
 * plus forcing.  This is the right-hand side without the viscous term. */
int oracle_ns_rhs(const ocplx *uhat, ocplx *nhat, int n, const oracle_ns_params *p);
/* Divergence form -i k_l F(u_l u_j), dealiased and projected (Eq. (7) as printed). */
int oracle_ns_rhs_divergence(const ocplx *uhat, ocplx *nhat, int n);
/* nsteps of RK2 (Heun) with the viscous integrating factor exp(-nu k^2 dt). */
int oracle_ns_step(ocplx *uhat, int n, const oracle_ns_params *p, int nsteps);
/* nsteps of the paper's RK4 with the same integrating factor (Lawson form). */
int oracle_ns_step_rk4(ocplx *uhat, int n, const oracle_ns_params *p, int nsteps);

/* Rayleigh-Benard convection (Sec. 2.2, Eqs. (12)-(13), non-dimensional, FFF
 * basis on the 2 pi-periodic cube, gravity along z), state
 * s[4][n][n][n/2+1] = (u_x, u_y, u_z, theta):
 *   N_u = P[F(u x omega) + theta z],  N_theta = -i k . F(u theta) + u_z
 * (2/3-truncated; diffusion nu = sqrt(Pr/Ra), kappa = 1/sqrt(Ra Pr) is left
 * to the integrating factors of the stepper; scheme 0 RK2, 1 RK4). */
int oracle_rbc_rhs(const ocplx *s, ocplx *out, int n);
int oracle_rbc_step(ocplx *s, int n, double Ra, double Pr, double dt, int nsteps, int scheme);
/* The same between free-slip, isothermal plates (SFF, Eq. (14)): wall-normal
 * axis x on [0, pi] with gravity along it; u_x, theta in the sine basis
 * along x (index a: k_x = a + 1), u_y, u_z in the cosine basis (k_x = a);
 *   N_u = P[u x omega + theta x],  N_theta = -div(u theta) + u_x,
 * truncated to 3 k_x < 2n, 3|k_y| < n, 3|k_z| < n. */
int oracle_rbc_sff_rhs(const ocplx *s, ocplx *out, int n);
int oracle_rbc_sff_step(ocplx *s, int n, double Ra, double Pr, double dt, int nsteps, int scheme);

/* Diagnostics: E = 1/2 sum w |u|^2, eps = nu sum w k^2 |u|^2,
 * EK[K] = 1/2 sum_{nint|k| = K} w |u|^2 for K = 0..kmax (modes beyond kmax dropped). */
int oracle_diag(const ocplx *uhat, int n, double nu, double *E, double *eps,
                double *EK, int kmax);
/* Energy transfer sum w Re(conj(u).N); zero for the rotational form. */
double oracle_transfer(const ocplx *uhat, const ocplx *nhat, int n);
/* T(K), K = 0..kmax: per-shell sum of w Re(conj(u) . N) (shell nint|k|). */
int oracle_transfer_spectrum(const ocplx *uhat, const ocplx *nhat, int n, double *T, int kmax);
/* Shell-to-shell transfer T[r][g] = -<u_r . (u . grad) u_g>, shells
 * bounds[i] <= nint|k| < bounds[i+1] (nshells + 1 increasing bounds). */
int oracle_shell_transfer(const ocplx *uhat, int n, int nshells, const int *bounds, double *T);

/* Initial conditions. */
int oracle_ic_taylor_green(ocplx *uhat, int n);  /* u = (sin x cos y, -cos x sin y, 0) */
int oracle_ic_abc(ocplx *uhat, int n);           /* u = (sin z + cos y, sin x + cos z, sin y + cos x) */
/* Random-phase solenoidal field from three normal fields normals[3][n][n][n]:
 * forward transform, 2/3 truncation, projection, shell K = nint|k| rescaled so that
 * its energy is proportional to K^4 exp(-2 (K/k0)^2), uhat(0) = 0, total energy E0. */
int oracle_ic_random(const double *normals, ocplx *uhat, int n, double k0, double E0);

/* Apply the 2/3 mask, projection, and wavenumber helpers (exposed for tests). */
int oracle_dealias(ocplx *fhat, int nfields, int n);
int oracle_project(ocplx *uhat, int n);

/* ------------------------------------------------------------ closure ----
 * Learned subgrid-stress closure (not in the paper; the task's closure
 * workload).  Reading: the MLP maps the 5 invariants of the filtered velocity
 * gradient to the 6 components of tau in the eigenframe of the filtered
 * strain rate S (sorted eigenvalues, each eigenvector's largest-magnitude
 * component positive), tau = Q tau' Q^T. */

/* Box filter: means over factor^3 blocks of u_i and u_i u_j.  u: real
 * [3][n][n][n]; ubar: [3][m][m][m]; tau: [6][m][m][m] = <u_i u_j> - ubar_i ubar_j
 * in the order xx, yy, zz, xy, xz, yz (m = n / factor). */
int oracle_box_filter(const double *u, int n, int factor, double *ubar, double *tau);

/* The subgrid stress of the coarse solver as it computes: with T the 2/3
 * truncation on the m^3 grid and ubar_T = T ubar,
 *   tau_les_ij = T[ tau_ij + ubar_i ubar_j - ubar_T,i ubar_T,j ]
 * (ubar[3][m^3], tau[6][m^3] from oracle_box_filter; out[6][m^3]). */
int oracle_les_stress(const double *ubar, const double *tau, int m, double *out);

/* Velocity gradient A[i*3+j] = d u_i / d x_j of a real field u[3][m][m][m] on
 * the 2 pi-periodic grid, from the 2/3-truncated spectrum. A: [9][m][m][m]. */
int oracle_gradient(const double *u, int m, double *A);

/* Invariants of S = (A + A^T)/2, R = (A - A^T)/2 at one point:
 * tr S^2, tr R^2, tr S^3, tr R^2 S, tr R^2 S^2. */
void oracle_invariants(const double A[9], double inv[5]);

/* Symmetric 3x3 eigendecomposition by cyclic Jacobi rotations: lam
 * descending, eigenvector k in column k of Q (Q[row*3+k]), largest-magnitude
 * component of each column positive. */
void oracle_sym_eig3(const double S[9], double lam[3], double Q[9]);

/* MLP 5 -> 64 -> 64 -> 64 -> 6, tanh on the three hidden layers.  params
 * (9094): W1[64][5], b1[64], W2[64][64], b2[64], W3[64][64], b3[64],
 * W4[6][64], b4[6].  bf16_acts != 0 rounds each layer's input (x, h1, h2, h3)
 * to bfloat16 (round to nearest even of the FP32 value) before use. */
#define ORACLE_MLP_NPARAMS 9094
int oracle_mlp_forward(const double *params, const double *x, double *y, int B, int bf16_acts);
/* Mean-squared-error loss (1/(6B)) sum (y - t)^2 and its gradient. */
double oracle_mlp_loss_grad(const double *params, const double *x, const double *t, int B,
                            int bf16_acts, double *grad);
/* One Adam step (Kingma and Ba 2015), step counted from 1. */
void oracle_adam(double *params, double *m, double *v, const double *grad, int nparam, int step,
                 double lr, double beta1, double beta2, double eps);

/* SGS force of a real stress tau[6][n][n][n] (order xx, yy, zz, xy, xz, yz):
 * s_i = -i k_j tau_hat_ij, 2/3-truncated and projected.  fhat: [3][n][n][n/2+1]. */
int oracle_sgs_force(const double *tau, int n, ocplx *fhat);

#ifdef __cplusplus
}
#endif
#endif
