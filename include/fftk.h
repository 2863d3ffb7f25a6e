/* fftk.h -- C ABI of the GB300 (sm_103a) FFTK/Tarang hot-path library.
 *
 * Chatterjee, Verma, Kumar, Samtaney, Hadri, Khurram, "Scaling of a Fast
 * Fourier Transform and a Pseudo-spectral Fluid Solver up to 196608 cores"
 * (arXiv:1805.07801).  This library implements, on one GPU, the paper's 3D
 * real-to-complex / complex-to-real FFT (FFTK, Sec. 3) and the pseudo-spectral
 * incompressible Navier-Stokes step built on it (Tarang, Sec. 2.2).
 *
 * Conventions
 *   Transform (Sec. 2.1, Eq. (1) with the Fourier basis of Eq. (2a)):
 *     inverse  f(x) = sum_k fhat(k) exp(+i k.x)                 (no factor)
 *     forward  fhat(k) = (1/(nx ny nz)) sum_x f(x) exp(-i k.x)
 *   on the 2 pi-periodic grid x = 2 pi (i/nx, j/ny, l/nz).
 *   Real array:    float [batch][nx][ny][nz], z fastest (Sec. 3: z is local).
 *   Complex array: float2 (re, im) [batch][nx][ny][nz/2+1]; the axes are not
 *                  exchanged (the transpose-free layout of Appendix A).  Index
 *                  a on x or y means k = a for a < n/2, a - n otherwise; on z,
 *                  k = c.
 *   Sizes: nx, ny are powers of two in [1, 4096]; nz a power of two in
 *          [2, 4096] (ny = 1 gives the paper's 2D mode, Sec. 3).
 *   Pointers: device pointers, 16-byte aligned.  Streams: a cudaStream_t
 *          passed as void* (NULL = legacy default stream).  Calls are
 *          asynchronous on that stream unless stated otherwise.
 *   Ownership: the caller owns every data buffer and stream.  A plan owns its
 *          twiddle tables and, unless fftk_set_workspace was called, its
 *          workspace.  A plan must be used by one stream at a time.
 *   Errors: no call aborts or exits.  Argument checks run before any CUDA
 *          call.  Launch failures return FFTK_ERR_CUDA; faults inside a kernel
 *          surface as FFTK_ERR_CUDA from a later synchronising call.
 */
#ifndef FFTK_H
#define FFTK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftk_plan_s *fftk_plan; /* opaque; created and freed by the library */

typedef enum {
  FFTK_OK = 0,
  FFTK_ERR_INVALID_ARG = 1,      /* NULL / misaligned / overlapping pointer, bad count */
  FFTK_ERR_UNSUPPORTED_SIZE = 2, /* a dimension outside the supported set */
  FFTK_ERR_NO_DEVICE = 3,        /* no CUDA device visible */
  FFTK_ERR_OOM = 4,              /* device allocation failed */
  FFTK_ERR_CUDA = 5,             /* a CUDA runtime call or launch failed */
  FFTK_ERR_NONFINITE = 6,        /* a solver diagnostic was NaN or Inf */
  FFTK_ERR_TIMEOUT = 7           /* a bounded device-side wait expired */
} fftk_status;

typedef enum {
  FFTK_R32 = 0,         /* FP32 data, FP32 arithmetic, FP64-built FP32 twiddles */
  /* FP32 data; in the y and x passes of length 256, 512, 1024 or 2048 the two
   * radix-16 stages run on the tensor cores (tcgen05) as products of split FP16
   * operands, x = x_hi + x_lo and W16 = W_hi + W_lo, with FP32 accumulation:
   * (x_hi + x_lo) W_hi + x_hi W_lo (relative error ~2^-22 per stage); twiddles,
   * power-of-two scaling, the remaining radix-2/4/8 stage and the z pass stay
   * FP32.  Not part of the paper (it uses FFTW in double precision). */
  FFTK_R32_SPLIT16 = 1
} fftk_dtype;

/* Human-readable name of a status code (static storage). */
const char *fftk_status_string(fftk_status s);

/* Name of the CUDA error behind the calling thread's most recent
 * FFTK_ERR_CUDA / FFTK_ERR_OOM / FFTK_ERR_NO_DEVICE (e.g. "cudaErrorInvalidValue"),
 * or "" if there was none (static storage). */
const char *fftk_last_cuda_error(void);

/* Create a plan for nx x ny x nz transforms (paper Sec. 3).  Builds the
 * twiddle tables in FP64 on the host and rounds them once to FP32: exp(-2 pi
 * i m / L) for every power of two L <= 4 max(nx, ny, nz), the same factors
 * laid out per radix stage of the line transforms (256 KB), and for 3 * 2^m
 * dimensions the tables of length 3 * 2^j.  Binds the plan to the current
 * CUDA device.
 * Errors: INVALID_ARG (out NULL, bad dtype), UNSUPPORTED_SIZE, NO_DEVICE, OOM,
 * CUDA.  On error *out is set to NULL. */
fftk_status fftk_plan_create(int nx, int ny, int nz, fftk_dtype dtype, fftk_plan *out);

/* Free a plan and everything it owns.  Synchronises the device.  NULL is
 * INVALID_ARG. */
fftk_status fftk_plan_destroy(fftk_plan p);

/* Bytes of device workspace fftk_r2c and fftk_c2r use for `batch`
 * transforms: two complex arrays of batch * nx * ny * (nz/2+1) * 8 bytes when
 * nx > 1 and ny > 1 (each strided pass then reads one array and writes
 * another), else one.  fftk_r2c uses the first array only.  With one array
 * (a caller's smaller buffer, or a plan-owned one when two cannot be
 * allocated) fftk_c2r runs its y pass in place; with none fftk_r2c runs both
 * passes in place in `out`, and fftk_c2r fails (OOM or INVALID_ARG).
 * fftk_inverse with a Fourier z axis uses the first array.  0 on bad
 * arguments. */
size_t fftk_workspace_bytes(fftk_plan p, int batch);

/* Hand the plan a caller-owned device workspace (NULL, 0 = go back to a
 * plan-owned one).  The caller keeps it alive while the plan uses it. */
fftk_status fftk_set_workspace(fftk_plan p, void *dev_ptr, size_t bytes);

/* Forward 3D real-to-complex transform (paper Sec. 3, steps 1-5): z r2c, then
 * y c2c, then x c2c, with the 1/(nx ny nz) factor of Eq. (1)'s inverse.
 * in:  float [batch][nx][ny][nz]; out: float2 [batch][nx][ny][nz/2+1].
 * Out-of-place: overlapping in/out is INVALID_ARG.  `in` is not modified.
 * With nx > 1 and ny > 1 the y pass writes the plan's workspace and the x
 * pass reads it back, or both run in place in `out` when no workspace can be
 * had (fftk_workspace_bytes). */
fftk_status fftk_r2c(fftk_plan p, const float *in, void *out, int batch, void *cuda_stream);

/* Inverse 3D complex-to-real transform ("the reverse of the above", Sec. 3):
 * x c2c, y c2c, then z c2r, no factor.  in: float2 [batch][nx][ny][nz/2+1];
 * out: float [batch][nx][ny][nz].  `in` is not modified (the y/x passes run in
 * the plan's workspace).  For each z line the imaginary parts of its k_z = 0
 * and k_z = nz/2 coefficients are ignored, which is the exact inverse for
 * Hermitian-consistent spectra (those produced by fftk_r2c).  Out-of-place. */
fftk_status fftk_c2r(fftk_plan p, const void *in, float *out, int batch, void *cuda_stream);

/* Bases per axis (paper Sec. 2.1, Eq. (2a-2c)): FOURIER exp(i k s) on a
 * 2 pi-periodic axis; SINE 2 sin(k s) (k = 1..n, coefficient k stored at
 * k - 1) and COSINE 2 cos(k s) (k = 0..n-1, stored at k) on the n points
 * s_j = (j + 1/2) pi / n of [0, pi] (free-slip walls at 0 and pi).  The
 * inverse is the sum over the basis with no factor; the forward is its exact
 * inverse (1/n per axis; the sine k = n and cosine k = 0 coefficients take
 * 1/(2n)). */
typedef enum { FFTK_FOURIER = 0, FFTK_SINE = 1, FFTK_COSINE = 2 } fftk_basis;

/* Forward 3D transform with a basis per axis, basis[3] = {x, y, z}, Fourier
 * axes trailing: FFF, SFF, SSF or SSS in the paper's naming, where each S
 * axis is FFTK_SINE or FFTK_COSINE (e.g. the all-free-slip u_z is
 * {COSINE, COSINE, SINE}).  Passes in the paper's order: z, then y, then x.
 * in: float [batch][nx][ny][nz].  out: float2 [batch][nx][ny][nz/2+1] when z
 * is Fourier (half spectrum), else float [batch][nx][ny][nz] (all-real
 * coefficients).  Sine/cosine passes are FP32 in both plan dtypes (one
 * complex FFT of the line's length with pre- and post-twiddles, Makhoul's
 * method); Fourier passes follow the plan dtype.  An S axis needs n >= 2.
 * Out-of-place; overlap, a Fourier axis before an S axis or an unknown
 * basis is INVALID_ARG.  fftk_forward(p, {F,F,F}, ...) equals fftk_r2c. */
fftk_status fftk_forward(fftk_plan p, const int *basis, const float *in, void *out, int batch,
                         void *cuda_stream);

/* Inverse of fftk_forward: x, then y, then z; `in` is not modified (with a
 * Fourier z axis the x and y passes run in the plan's c2r workspace, else in
 * `out`).  A Fourier z axis is inverted line-wise as in fftk_c2r. */
fftk_status fftk_inverse(fftk_plan p, const int *basis, const void *in, float *out, int batch,
                         void *cuda_stream);

/* ---------------------------------------------------------------- Tarang --
 * Pseudo-spectral incompressible Navier-Stokes on a 2 pi-periodic cubic grid
 * (plan with nx = ny = nz = n, n >= 8), paper Sec. 2.2, Eqs. (7)-(8).
 * Velocity: float2 uhat[3][n][n][n/2+1] (component outermost), the forward
 * transform of the real velocity.  Modes outside the 2/3-rule set
 * (3|k_x| < n and 3|k_y| < n and 3|k_z| < n) must be zero on entry and stay
 * zero; the solver never reads them.
 * FP32 plans run the right-hand side in five fused kernels (inverse x with
 * the curl, inverse y, z transforms with u x omega, forward y, forward x with
 * projection and update).  FFTK_R32_SPLIT16 plans (n of 256 to 1024) run the
 * x and y passes on the tensor cores (split FP16 radix-16 stages, restricted
 * to the 2/3-rule set) around the same fused FP32 z kernel: curl on the kept
 * modes, inverse x and y of six fields, z with u x omega, forward y and x of
 * three fields, update.
 * Device memory (plan-owned, allocated on the first solver call and kept):
 * a six-field workspace (rows of n/2 + 1 complex values rounded up to a
 * multiple of 16), the three-field stage state, and for FP32 plans a second
 * six-field workspace that the fused passes alternate with the first (about
 * 8.5 GB at 512^3); 3 * 2^m cubes add six real fields.  Out of memory is
 * FFTK_ERR_OOM. */
/* Learned subgrid-stress model (not in the paper; see tarang_mlp_*): the
 * network maps the 5 invariants of the resolved velocity gradient A
 * (tr S^2, tr R^2, tr S^3, tr R^2 S, tr R^2 S^2 with S, R the symmetric and
 * antisymmetric parts of A) to the stress in the eigenframe Q of S
 * (eigenvalues descending, each eigenvector's largest-magnitude component
 * positive); tau = Q tau' Q^T.  The fused inference evaluates the network on
 * the tensor cores like tarang_mlp_forward; an expired wait is reported by
 * fftk_sync of the solver's plan. */
typedef struct {
  const float *params;  /* device, 9094 FP32 values (layout of tarang_mlp_forward) */
  float in_shift[5];    /* network input x = (invariant - in_shift) * in_scale */
  float in_scale[5];
  float out_scale[6];   /* tau' = output * out_scale, order xx, yy, zz, xy, xz, yz */
} tarang_sgs_model;

typedef struct {
  double nu;        /* kinematic viscosity */
  double dt;        /* time step (tarang_ns_step only) */
  double force_eps; /* constant injected power; 0 disables forcing */
  int force_k2min;  /* forced modes: force_k2min <= |k|^2 <= force_k2max */
  int force_k2max;
  /* NULL = resolved simulation.  Otherwise the right-hand side gains the
   * subgrid force P[-i k_j tau_hat_ij] of the model's stress, evaluated per
   * grid point from the current state's gradient (fused inference). */
  const tarang_sgs_model *sgs_model;
  /* tarang_ns_step's time stepper: TARANG_RK2 (0) or TARANG_RK4 (1). */
  int scheme;
} tarang_params;

enum { TARANG_RK2 = 0, TARANG_RK4 = 1 };

/* Nonlinear right-hand side without the viscous term:
 *   nhat = P[ F(u x omega) ] on the 2/3 set, 0 elsewhere, + forcing,
 * with omega = curl u, P the projection k_j uhat_j = 0 of Eq. (8), and the
 * product formed in real space (Orszag's pseudo-spectral method, Sec. 2.2).
 * Forcing (when force_eps > 0): nhat += force_eps uhat / (2 E_f) on the forced
 * modes, E_f = 1/2 sum w |uhat|^2 over them (FP64 reduction), so exactly
 * force_eps is injected.  uhat, nhat: float2 [3][n][n][n/2+1], distinct. */
fftk_status tarang_ns_rhs(fftk_plan p, const void *uhat, void *nhat, const tarang_params *prm,
                          void *cuda_stream);

/* nsteps steps of RK2 (Heun) with the viscous integrating factor
 * E = exp(-nu |k|^2 dt) (scheme TARANG_RK2):
 *   u1 = E (u + dt N(u)),   u <- 1/2 E u + 1/2 (u1 + dt N(u1)),
 * or of the paper's fourth-order Runge-Kutta scheme (Sec. 2.2, 36
 * transforms per step as counted in Sec. 6) with the same factor in
 * Lawson's form (scheme TARANG_RK4), H = exp(-nu |k|^2 dt/2):
 *   N1 = N(u), ua = H (u + dt/2 N1), N2 = N(ua), ub = H u + dt/2 N2,
 *   N3 = N(ub), uc = E u + dt H N3, N4 = N(uc),
 *   u <- E u + dt/6 (E N1 + 2 H N2 + 2 H N3 + N4);
 * RK4 keeps three more fields of device memory (the accumulator).
 * uhat is updated in place.  diag_host: NULL, or room for 2 + kmax + 1
 * doubles, kmax = nint(sqrt(3) n / 2) + 1 (see tarang_diag_kmax); when given,
 * the call synchronises and writes E, eps and E(K) of the final state, and
 * returns FFTK_ERR_NONFINITE if E is not finite. */
fftk_status tarang_ns_step(fftk_plan p, void *uhat, const tarang_params *prm, int nsteps,
                           double *diag_host, void *cuda_stream);

/* Rayleigh-Benard convection (Sec. 2.2, Eqs. (12)-(13) in their
 * non-dimensional form):
 *   d_t u + (u.grad) u = -grad sigma + theta g + sqrt(Pr/Ra) lap u,
 *   d_t theta + (u.grad) theta = u.g + lap theta / sqrt(Ra Pr),
 * g the unit vector against gravity, on one of two bases:
 *   TARANG_RBC_FFF  the 2 pi-periodic cube, g = z;
 *   TARANG_RBC_SFF  free-slip, isothermal plates (Eq. (14)) at x = 0 and pi,
 *                   g = x, y and z 2 pi-periodic: u_x and theta in the sine
 *                   basis along x (storage index a is k_x = a + 1), u_y and
 *                   u_z in the cosine basis (index a is k_x = a), on the
 *                   sine/cosine grid of fftk_forward (n points of [0, pi]).
 * State: float2 [4][n][n][n/2+1] = (u_x, u_y, u_z, theta), truncated (FFF:
 * the 2/3 set of tarang_ns_step; SFF: 3 k_x < 2n, 3|k_y| < n, 3 k_z < n),
 * zero elsewhere.  The right-hand side without diffusion,
 * N_u = P[u x omega + theta g] and N_theta = -div(u theta) + u.g, goes
 * through seven inverse (u, omega, theta) and six forward (u x omega,
 * u theta) transforms per stage, the paper's 52 transforms per RK4 step
 * (Sec. 7), restricted to the truncated set, with the products formed inside
 * the z pass; between plates the x passes are sine/cosine passes.  FP32 in
 * both plan dtypes.  Cubes: n a power of two in [8, 1024] for both bases;
 * the periodic cube also takes n = 3 * 2^m in [12, 768] (the paper's XC40
 * convection sizes, Sec. 7), where the right-hand side runs through the
 * plan's full transforms (radix-3 passes) with the products formed in real
 * space (7 more real fields).  Other sizes: FFTK_ERR_UNSUPPORTED_SIZE.
 * Device memory: 15 more complex fields (allocated on first use, kept by
 * the plan). */
enum { TARANG_RBC_FFF = 0, TARANG_RBC_SFF = 1 };

typedef struct {
  double Ra;  /* Rayleigh number */
  double Pr;  /* Prandtl number */
  double dt;  /* time step */
  int scheme; /* TARANG_RK2 or TARANG_RK4, integrating factors exp(-nu k^2 dt), exp(-kappa k^2 dt) */
  int basis;  /* TARANG_RBC_FFF or TARANG_RBC_SFF */
} tarang_rbc_params;

/* out = (N_u, N_theta), float2 [4][n][n][n/2+1], distinct from state;
 * basis TARANG_RBC_FFF or TARANG_RBC_SFF. */
fftk_status tarang_rbc_rhs(fftk_plan p, int basis, const void *state, void *out, void *cuda_stream);

/* nsteps steps in place, in the forms of tarang_ns_step (u and theta each
 * with its own factor).  Asynchronous.  INVALID_ARG for non-positive or
 * non-finite Ra, Pr, dt or an unknown scheme. */
fftk_status tarang_rbc_step(fftk_plan p, void *state, const tarang_rbc_params *prm, int nsteps,
                            void *cuda_stream);

/* Kinetic and thermal energy transfer of convection on the periodic cube
 * (FFF), the fluxes the paper plots for its convection run (Sec. 7,
 * Pi_u(k) and Pi_theta(k)).  With N the right-hand side of tarang_rbc_rhs:
 *   T_u(K) = sum_{nint|k| = K} w Re(conj(u) . N_u) - w Re(conj(u_z) theta),
 *   T_theta(K) = sum_{nint|k| = K} w Re(conj(theta) N_theta) - w Re(conj(theta) u_z)
 * (the buoyancy and conduction-source exchanges taken out, the advective
 * transfer left; each sums to 0 over K up to rounding) and
 * Pi(K) = -sum_{K' <= K} T(K').  out_host: 2 (1 + 2 (kmax + 1)) doubles:
 * sum T_u, T_u(0..kmax), Pi_u(0..kmax), then the same for theta (kmax of
 * tarang_diag_kmax).  FP64 reductions in a fixed order; synchronises; uses
 * the plan's convection workspace (not concurrently with tarang_rbc_step). */
fftk_status tarang_rbc_transfer(fftk_plan p, const void *state, double *out_host, void *cuda_stream);

/* Largest shell index reported by the diagnostics for this plan. */
int tarang_diag_kmax(fftk_plan p);

/* Diagnostics of a velocity state, reduced in FP64 in a fixed order
 * (bitwise reproducible):  E = 1/2 sum w |u|^2,  eps = nu sum w |k|^2 |u|^2,
 * E(K) = 1/2 sum_{nint|k| = K} w |u|^2, w = 1 on k_z = 0 and k_z = n/2,
 * 2 elsewhere.  Writes 2 + kmax + 1 doubles to diag_host; synchronises. */
fftk_status tarang_diag(fftk_plan p, const void *uhat, double nu, double *diag_host,
                        void *cuda_stream);

/* Energy transfer spectrum and flux, the scale-by-scale analysis of the
 * nonlinear term (Sec. 1 and Sec. 7 of the paper: energy flux Pi(k)).  With
 * N the right-hand side of tarang_ns_rhs for the state uhat,
 *   T(K) = sum_{nint|k| = K} w Re(conj(uhat) . N),  w as in tarang_diag,
 *   Pi(K) = -sum_{K' <= K} T(K')   (energy leaving the sphere of radius K).
 * prm: NULL for the nonlinear term alone (then sum_K T(K) vanishes up to
 * rounding); otherwise the forcing and the subgrid model of prm are included
 * as in tarang_ns_rhs (nu and dt are not used).  out_host: 1 + 2 (kmax + 1)
 * doubles (kmax of tarang_diag_kmax): sum_K T(K), then T(0..kmax), then
 * Pi(0..kmax).  The reduction is FP64 in a fixed order (bitwise
 * reproducible); the right-hand side is the solver's FP32 one.  Uses the
 * plan's solver workspace (do not overlap with tarang_ns_step on the same
 * plan); synchronises cuda_stream.  FFTK_ERR_NONFINITE if the sum is not
 * finite. */
fftk_status tarang_transfer(fftk_plan p, const void *uhat, const tarang_params *prm, double *out_host,
                            void *cuda_stream);

/* Shell-to-shell energy transfer (the scale-by-scale analysis the paper
 * names in Sec. 1 and Sec. 3): shell i holds the kept modes with
 * bounds[i] <= nint|k| < bounds[i+1], and
 *   out_host[r * nshells + g] = T(r <- g) = -<u_r . (u . grad) u_g>
 * (average over the box) is the rate at which shell r receives energy from
 * shell g through advection by the whole field.  T is antisymmetric, the
 * givers of a receiver add up to its share of tarang_transfer's T(K), and
 * the flux through a bound b is the sum of T(r <- g) over r >= b > g.
 * Evaluated pseudo-spectrally with the plan's transforms: u to real space
 * once, then per giver shell the gradient of its modes (nine c2r), the
 * product u_j d_j u_g,i (real space), three r2c and an FP64 reduction over
 * receivers in a fixed order (bitwise reproducible).  Givers beyond the
 * dealiased radius are skipped (zero columns).
 * nshells: 1 .. kmax + 1; bounds: host array of nshells + 1 strictly
 * increasing integers in [0, kmax + 1] (kmax of tarang_diag_kmax); out_host:
 * nshells * nshells doubles, row-major by receiver.  Device memory: nine more
 * real fields (allocated on first use and kept by the plan).  Uses the plan's
 * solver workspace (do not overlap with tarang_ns_step on the same plan);
 * synchronises cuda_stream.  INVALID_ARG for bad bounds, NONFINITE if any
 * entry is not finite. */
fftk_status tarang_shell_transfer(fftk_plan p, const void *uhat, int nshells, const int *bounds,
                                  double *out_host, void *cuda_stream);

/* The diagnostics of tarang_diag for callers that cannot allocate device
 * memory.  The paper has no counterpart: this exists for host code that must
 * not call cudaMalloc (for instance a loop that cannot afford cudaMalloc's
 * implicit device-wide synchronisation, or an application whose own memory
 * manager owns all device allocations).  No plan is needed and nothing is
 * allocated: the FP64 partial sums live in a 2 MiB array that the library
 * reserves statically on every device that loads it, held until the process
 * exits.  n: grid size of a cubic velocity state uhat (float2
 * [3][n][n][n/2+1], 2/3-truncated as for tarang_ns_step), a power of two in
 * [8, 1024]; larger n returns FFTK_ERR_UNSUPPORTED_SIZE.  diag_dev: device
 * buffer of 2 + kmax + 1 doubles, kmax = floor(sqrt(3) n / 2 + 1/2) + 1,
 * receiving E, eps, E(K) exactly as tarang_diag computes them (same kernels,
 * same summation order).  Asynchronous on cuda_stream; the result is valid
 * once the stream reaches it.  The first call on each device looks up the
 * array's device address and sets the reduction kernel's shared-memory limit;
 * make that first call before any stream capture.  All calls on a device
 * share the one array, so calls that overlap on the GPU (concurrent streams,
 * or host threads) race and must be serialised by the caller. */
fftk_status tarang_diag_noalloc(int n, const void *uhat, double nu, double *diag_dev,
                                void *cuda_stream);

/* Random-phase solenoidal initial velocity (used by the decaying- and
 * forced-turbulence workloads): the forward transform of three real fields
 * `normals` (device float [3][n][n][n], e.g. from fftk_fill_normal), 2/3
 * truncation, projection (Eq. (8)), the k_z = 0 plane made exactly Hermitian,
 * each shell K = nint|k| >= 1 rescaled so that its energy is proportional to
 * K^4 exp(-2 (K/k0)^2), uhat(0) = 0, and a final factor making the total
 * energy E0.  Shell energies are reduced in FP64 and the scale factors are
 * computed in FP64 on the host.  Synchronises the stream.
 * uhat: float2 [3][n][n][n/2+1]. */
fftk_status tarang_ic_random(fftk_plan p, const float *normals, void *uhat, double k0, double E0,
                             void *cuda_stream);

/* Make uhat (float2 [3][n][n][n/2+1], in place) a valid solver state: modes
 * outside the 2/3-rule set are zeroed, each kept mode is replaced by its
 * divergence-free part u - k (k.u)/|k|^2 (Eq. (8), FP32), and u(0) = 0.
 * Asynchronous; INVALID_ARG for a null or misaligned pointer,
 * UNSUPPORTED_SIZE for a non-cubic plan or n outside [8, 1024]. */
fftk_status tarang_dealias_project(fftk_plan p, void *uhat, void *cuda_stream);

/* Counter-based SplitMix64 generator (Steele, Lea, Flood 2014): element i of
 * field f for seed s uses the outputs at counters c = s 2^40 + f 2^36 + 2i and
 * c + 1 of the stream started at state 0, x_c = mix64((c + 1) * 0x9E3779B97F4A7C15).
 * fftk_fill_normal: Box-Muller, u1 = ((x1 >> 11) + 1) 2^-53,
 *   u2 = (x2 >> 11) 2^-53, value = sqrt(-2 ln u1) cos(2 pi u2) in FP64, stored
 *   as float.
 * fftk_fill_uniform: value = 2 (x_i >> 40) 2^-24 - 1 with x_i at counter
 *   s 2^40 + f 2^36 + i (exact in FP32, uniform on [-1, 1)).
 * dev: device float[count]; seed < 2^24, field < 16, 2 count <= 2^36. */
fftk_status fftk_fill_normal(float *dev, long long count, int seed, int field, void *cuda_stream);
fftk_status fftk_fill_uniform(float *dev, long long count, int seed, int field, void *cuda_stream);

/* ------------------------------------------------------ learned closure --
 * Closure data from a resolved state (the task's closure workload; no
 * counterpart in the paper).
 *
 * Box filter of the real velocity of uhat (plan n^3, cubic, n >= 32) over
 * factor^3 blocks (factor a power of two <= 32): ubar[3][m^3] (m = n/factor)
 * and tau[6][m^3] = <u_i u_j> - ubar_i ubar_j (xx, yy, zz, xy, xz, yz), block
 * sums in FP64.  Synchronises; allocates its scratch. */
fftk_status tarang_box_filter(fftk_plan p, const void *uhat, int factor, float *ubar, float *tau,
                              void *cuda_stream);

/* Network features on a coarse grid (plan m^3): the gradient A_ij = d_j ubar_i
 * of the 2/3-truncated transform of ubar[3][m^3] (computed spectrally),
 * inv[5][m^3] (the invariants of tarang_sgs_model), frame[9][m^3] (Q, row
 * major per point) and, when tau is given, tau_frame[6][m^3] = Q^T tau Q.
 * Synchronises; allocates its scratch. */
fftk_status tarang_closure_features(fftk_plan p, const float *ubar, const float *tau, float *inv,
                                    float *frame, float *tau_frame, void *cuda_stream);

/* The subgrid stress of the coarse solver as it computes it (the closure's
 * training target; the paper has no closure).  The coarse grid (plan m^3,
 * power of two) keeps only the 2/3 set of a filtered field, ubar_T = T ubar
 * with T the truncation 3|k_i| < m, and forms its products dealiased, so
 * the exact coarse equations for ubar_T carry
 *   tau_les_ij = T[ tau_ij + ubar_i ubar_j - ubar_T,i ubar_T,j ]
 * (tau + ubar ubar = the box-filtered products <u_i u_j>).  ubar[3][m^3] and
 * tau[6][m^3] as from tarang_box_filter; out[6][m^3] in the same pair order.
 * All three 16-byte aligned device arrays.  Synchronises; allocates its
 * scratch. */
fftk_status tarang_les_stress(fftk_plan p, const float *ubar, const float *tau, float *out, void *cuda_stream);

/* MLP 5 -> 64 -> 64 -> 64 -> 6 with tanh on the hidden layers.  params: 9094
 * FP32 values W1[64][5], b1[64], W2[64][64], b2[64], W3[64][64], b3[64],
 * W4[6][64], b4[6].  Each layer's input (x, h1, h2, h3) is rounded to
 * bfloat16; products and sums are FP32.  x: [B][5], y and targets t: [B][6].
 * A context owns the per-block gradient partials for up to max_batch samples;
 * gradients are reduced in a fixed order (bitwise reproducible). */
typedef struct tarang_mlp_s *tarang_mlp;
fftk_status tarang_mlp_create(int max_batch, tarang_mlp *out);
fftk_status tarang_mlp_destroy(tarang_mlp m);
/* Inference runs on the tensor cores (tcgen05, kind::f16 with BF16 operands):
 * each layer's BF16 input times its weights split into two BF16 parts
 * W = W_hi + W_lo (16 significant bits), FP32 accumulation; bias and tanh in
 * FP32.  A bounded wait that expires inside it is reported by tarang_mlp_sync. */
fftk_status tarang_mlp_forward(tarang_mlp m, const float *params, const float *x, float *y, int B,
                               void *cuda_stream);
/* Training of the closure network: `steps` Adam steps numbered first_step,
 * first_step + 1, ... (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the device
 * data set x [nsamples][5], t [nsamples][6].  The batch of step s is the
 * contiguous window of `batch` samples at offset
 *   splitmix64(seed * 2^32 + s) mod (nsamples - batch + 1)
 * (SplitMix64 output number c of the stream from state 0; shuffle the set once
 * beforehand).  With loss_log (device, steps / log_every doubles), the loss
 * of every log_every-th step is recorded.  Equivalent to the same sequence of
 * tarang_mlp_train_step calls; asynchronous. */
fftk_status tarang_sgs_train(tarang_mlp m, float *params, float *adam_m, float *adam_v, int first_step,
                             int steps, const float *x, const float *t, long long nsamples, int batch,
                             float lr, unsigned long long seed, double *loss_log, int log_every,
                             void *cuda_stream);
/* Wait for the stream; FFTK_ERR_TIMEOUT if a tensor-core wait of this
 * context's inference expired since the last call (the flag is cleared). */
fftk_status tarang_mlp_sync(tarang_mlp m, void *cuda_stream);
/* Mean-squared-error loss (1/(6B)) sum (y - t)^2 (device double, may be NULL)
 * and its gradient grad[9094] (device), on the CUDA cores (128 samples per
 * block, per-block partials summed in a fixed order). */
fftk_status tarang_mlp_loss_grad(tarang_mlp m, const float *params, const float *x, const float *t,
                                 int B, float *grad, double *loss, void *cuda_stream);
/* Layer-input precision of the CUDA-core training kernels: BF16 (the
 * network's definition, used by every other MLP call) or FP32, a test mode
 * with the BF16 roundings left out, so that the kernels' own arithmetic can
 * be held to FP32 accuracy against an FP64 reference. */
typedef enum { TARANG_ACT_BF16 = 0, TARANG_ACT_FP32 = 1 } tarang_act_mode;
/* tarang_mlp_loss_grad with the layer inputs in act_mode (FFTK_ERR_INVALID_ARG
 * for any other value); TARANG_ACT_BF16 is tarang_mlp_loss_grad itself. */
fftk_status tarang_mlp_loss_grad_mode(tarang_mlp m, const float *params, const float *x, const float *t,
                                      int B, float *grad, double *loss, int act_mode, void *cuda_stream);
/* The forward pass of tarang_mlp_loss_grad alone (CUDA cores, FP32 weights,
 * FP32 products and sums, layer inputs in act_mode): y[B][6] (device). */
fftk_status tarang_mlp_forward_mode(tarang_mlp m, const float *params, const float *x, float *y, int B,
                                    int act_mode, void *cuda_stream);
/* One Adam step (Kingma and Ba 2015; step counted from 1) on 9094 values. */
fftk_status tarang_mlp_adam(float *params, float *m, float *v, const float *grad, int step,
                            float lr, float beta1, float beta2, float eps, void *cuda_stream);
/* loss_grad followed by Adam (beta1 0.9, beta2 0.999, eps 1e-8). */
fftk_status tarang_mlp_train_step(tarang_mlp m, float *params, float *adam_m, float *adam_v, int step,
                                  const float *x, const float *t, int B, float lr, double *loss,
                                  void *cuda_stream);

/* Wait for the stream, then report a device-side bounded wait that expired in
 * any kernel of this plan since the last check (FFTK_ERR_TIMEOUT; the word is
 * cleared), or a CUDA fault (FFTK_ERR_CUDA). */
fftk_status fftk_sync(fftk_plan p, void *cuda_stream);

/* ------------------------------------------------------- instrumentation --
 * Kernel launches made by this plan since its creation. */
long long fftk_launch_count(fftk_plan p);

/* Turn per-launch CUDA-event timing on (and clear old records) or off. */
fftk_status fftk_profile_enable(fftk_plan p, int on);

/* Sum of device time (ms) and number of launches recorded for kernel kind
 * `kind` (0 .. fftk_kernel_kinds()-1) since profiling was enabled.
 * Synchronises on the recorded events. */
fftk_status fftk_profile_read(fftk_plan p, int kind, double *total_ms, long long *launches);
int fftk_kernel_kinds(void);
const char *fftk_kernel_name(int kind);

#ifdef __cplusplus
}
#endif
#endif /* FFTK_H */
