/*
 * lagwave.h -- C ABI of the GB300 (sm_103a) Laguerre-transform wave solver.
 *
 * Method: Fatyanov & Terekhov, "High-performance modeling acoustic and elastic waves using the
 * Parallel Dichotomy Algorithm" (arXiv:1005.0542).  The Laguerre transform in time (Sec. 2.1,
 * Eqs. 7-9) turns the wave equation into one elliptic problem per harmonic m with the SAME
 * operator and a right-hand side that depends on the earlier harmonics.  Each problem is solved
 * by preconditioned CG (acoustic, Sec. 2.3) or GMRES(k) (elastic, Sec. 2.3), preconditioned by a
 * constant-coefficient Laplace operator (Sec. 2.4, Eqs. 21-22) that is inverted by separation of
 * variables: a sine transform along x, then one tridiagonal system along z per x-mode, solved by
 * a partitioned ("Dichotomy-style") elimination whose factors are computed once (Sec. 1).
 *
 * Problem form used here (2D Cartesian, Dirichlet on all four sides):
 *   grid      nx x nz interior nodes, x_i = (i+1) dx, z_k = (k+1) dz; u = 0 on the frame.
 *   layout    every field is row-major [rhs][z][x] (x fastest), float64, interior nodes only.
 *   acoustic  A R_m = b_m,  A = -div(kappa grad) + rho h^2/4,  kappa = rho c^2,
 *             b_m = delta_s f_m - rho h^2 c_m sum_{k<m} (m-k) c^_k R_k     (Eq. 9, SPD form),
 *             c_m = sqrt(m!/(m+alpha)!), c^_k = 1/c_k, delta_s = 1/(dx dz) at the source node.
 *   elastic   C [Q;U]_m = [0; delta_s f_m] - rho h^2 c_m sum_{k<m}(m-k) c^_k [Q;U]_k  (Eq. 12,
 *             Cartesian plane strain, vertical point force), fields ordered [rhs][comp][z][x].
 *
 * Conventions
 *   - Every function returns a status (0 = LAG_OK, negative = error) and never throws or aborts.
 *     lag_strerror() names a status; lag_last_error() gives the context's last message.
 *   - The caller owns every pointer it passes.  Host arrays ("_host") are read during the call
 *     (or copied, where stated).  Device arrays ("_dev") must hold the stated number of float64
 *     values on the context's device and stay valid until the context's stream reaches the work.
 *   - The library owns contexts, media, plans, shots and their device memory.  All device work is
 *     issued on the context's CUDA stream.  Functions documented "stream-ordered" return after
 *     enqueueing; the others return when their results are on the host.
 *   - One context serves one host thread at a time (the serving loop runs its own thread and
 *     touches only its own streams).
 *   - There is no CPU fallback: a missing or unusable GPU returns LAG_ECUDA.
 */
#ifndef LAGWAVE_H
#define LAGWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define LAG_OK          0
#define LAG_EINVAL     (-1)  /* bad argument: null pointer, size out of range, mismatched objects */
#define LAG_ENOMEM     (-2)  /* device allocation failed or the context's HBM budget is exceeded */
#define LAG_ENOTCONV   (-3)  /* Krylov solve hit max_iter; results and stats are still filled in  */
#define LAG_ENUMERIC   (-4)  /* NaN or Inf in a residual norm                                      */
#define LAG_ECUDA      (-5)  /* CUDA runtime/driver error (message in lag_last_error)              */
#define LAG_EAGAIN     (-6)  /* lag_serve_poll: request not finished yet                          */
#define LAG_ETIMEDOUT  (-7)  /* a bounded device wait gave up (device status word)                 */
#define LAG_ECANCELED  (-8)  /* request was cancelled                                              */

/* precision of the preconditioner (the Krylov vectors, residuals, dot products, the Laguerre
 * recurrence and the inverse summation are always float64) */
#define LAG_FP64   0   /* plain path: preconditioner in float64 (DST as an FP64 GEMM)              */
#define LAG_MIXED  1   /* preconditioner in float32, DST as a split-bf16 tcgen05 GEMM (FP32 acc.), */
                       /* flexible (Polak-Ribiere) CG / flexible GMRES                              */

/* wavelet kinds */
#define LAG_WAVELET_RICKER 0   /* (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)              */
#define LAG_WAVELET_PAPER  1   /* exp[-(2 pi f0 (t-t0))^2 / gamma^2] sin(2 pi f0 (t-t0))  (Eq. 23)  */

typedef struct lag_ctx     lag_ctx;
typedef struct lag_medium  lag_medium;
typedef struct lag_precond lag_precond;
typedef struct lag_shot    lag_shot;

/* Interior nodes nx x nz with spacing dx, dz (m); u = 0 on the ghost nodes around them, except
 * that free_surface = 1 puts a free surface on top (Sec. 2.1, Eq. 3: du/dz = 0 at z = 0), read
 * as a top face of node row 0 that carries no flux (on Cartesian grids acoustic problems only;
 * elastic media return LAG_EINVAL).  The surface lies half a cell above row 0.  Fields are
 * [nz][nx], x fastest.
 *
 * cylindrical = 1: the paper's own 2.5D axisymmetric problem (Sec. 2.1 Eqs. 1-5, the scheme of
 * Sec. 2.3 Eqs. 17-19; elastic media: Sec. 2.2, below).  x is then the radius r: nodes
 * r_i = (i + 1/2) dx from the axis (the axis face carries no flux, Eq. 5), u = 0 on the ghost
 * node r = (nx + 1/2) dx; z_k =
 * (k + 1/2) dz with zero-flux faces at z = 0 (the free surface, Eq. 3) and at z = nz dz (the
 * auxiliary boundary).  free_surface must be 1.  Every term carries the factor r (a1 = rbar
 * kappa, a2 = r kappa, w = r rho h^2/4; the source f_m / (2 pi dx dz) at its node, the history
 * term r rho h^2).  Fields of cylindrical grids are [nx][nz]: radius index slow, depth index
 * fastest (the DCT-II along z runs over contiguous rows, the general tridiagonal systems along r
 * over columns); lag_point (ix, iz) is still (radius index, depth index).
 *
 * Elastic media on a cylindrical grid (Sec. 2.2, Eqs. 10-12): u = (u_r, u_z) = (Q, U), fields
 * [rhs][comp][nx][nz] (comp 0 = u_r); the operator is the gradient of a discrete strain energy
 * (symmetric; each strain term sampled at r-faces, z-faces, nodes or cell corners), so the
 * traction-free surface sigma_zz = sigma_rz = 0 (the paper's condition with Q and U put back in
 * place) is its natural condition at z = 0 and at the bottom; a vertical point force on the axis
 * (delta(r) delta(z - d) / (2 pi r)) enters the u_z equation as f_m / (2 pi dx dz); K = diag(B1, B2)
 * with the cylindrical coefficients of Eq. 22 (B1's d includes (l+2m)~ / r). */
typedef struct { int nx, nz; double dx, dz; int free_surface; int cylindrical; } lag_grid;
typedef struct { double h; int alpha; int n_harm; } lag_laguerre; /* Sec. 2.1: h (1/s), alpha >= 2 */
typedef struct {
  double tol;       /* stop when ||r||_2 / ||b||_2 <= tol (recursive residual)                    */
  int max_iter;     /* Krylov iterations per harmonic (GMRES: inner steps)                         */
  int restart_k;    /* GMRES(k) restart length (elastic), 1..64                                    */
  int prec;         /* LAG_FP64 or LAG_MIXED                                                       */
  int partitions;   /* z-partitions of the tridiagonal solve; 0 = automatic                        */
  int tune;         /* 1: shots run lag_precond_autotune on their plans at creation                */
  int layered;      /* 1: shots on Cartesian grids precondition with per-row midranges
                       (lag_precond_create_layered) instead of the whole-medium midranges of
                       Eq. 21 (acoustic) or Eq. 22 (elastic: B1, B2 with (l+2m)~(z), mu~(z),
                       rho~(z)); acoustic shots on cylindrical grids with per-radius midranges
                       kappa~(r), rho~(r) (the DCT along z still separates); cylindrical
                       elastic: 0 only                                                           */
} lag_solver;
typedef struct { int ix, iz; } lag_point;                          /* 0-based interior node        */
typedef struct { double f0, t0, gamma; int kind; } lag_wavelet;

typedef struct {
  int    *iters;         /* [nsrc][n_harm] Krylov iterations per harmonic and source, or NULL    */
  double *relres;        /* [nsrc][n_harm] final recursive ||r||/||b||, or NULL                   */
  long long total_iters; /* sum over harmonics of the iterations of the batch                      */
  double   seconds;      /* wall time of the call                                                  */
} lag_stats;

/* ---------------------------------------------------------------- context */
const char *lag_strerror(int status);
const char *lag_last_error(const lag_ctx *ctx);     /* last error text of ctx ("" if none)       */
int  lag_version(void);                              /* 100 * major + minor                       */

/* Create a context on CUDA device `device`.  hbm_budget_bytes (0 = no limit) caps the device
 * memory the context may hold; allocations beyond it fail with LAG_ENOMEM.  cuda_stream is a
 * cudaStream_t to issue work on (NULL: the context creates its own non-blocking stream). */
int  lag_create(lag_ctx **ctx, int device, size_t hbm_budget_bytes, void *cuda_stream);
void lag_destroy(lag_ctx *ctx);                      /* frees everything the context still owns   */
int  lag_synchronize(lag_ctx *ctx);                  /* waits for the context's stream            */
size_t lag_bytes_in_use(const lag_ctx *ctx);
/* Number of the library's kernels launched so far in this process (launch accounting). */
long long lag_kernel_launches(const lag_ctx *ctx);
/* Kernel-class timing.  enable(1) clears the records and starts bracketing every launch of the
 * profiled kernel classes with CUDA events on the launching stream; enable(0) stops.  read()
 * waits for the recorded events and returns per class the number of launches and the summed
 * milliseconds (arrays of nclasses entries; class names via lag_profile_class_name). */
int  lag_profile_enable(lag_ctx *ctx, int on);
int  lag_profile_read(lag_ctx *ctx, int nclasses, long long *counts, double *ms);
int  lag_profile_num_classes(void);
const char *lag_profile_class_name(int cls);

/* ---------------------------------------------------------------- preconditioner (Sec. 2.4)
 * The plan is the one-time "preparatory" step of the Dichotomy solve (Sec. 1): DST-I matrices
 * (folded into even/odd halves) and, for every x-mode j, the tridiagonal system
 *     T_j = tridiag(-az/dz^2, 2 az/dz^2 + ax lambda_j + d, -az/dz^2),
 *     lambda_j = (4/dx^2) sin^2(pi (j+1) / (2 (nx+1))),
 * factored once into partition-local eliminations, spike vectors and the reduced (interface)
 * system.  Acoustic B (Eq. 21): ax = az = kappa~, d = rho~ h^2/4 with f~ = (min f + max f)/2.
 * Elastic K = diag(B1, B2) (Eq. 22): B1 (ax, az) = ((lambda+2mu)~, mu~), B2 = (mu~, (lambda+2mu)~).
 * prec = LAG_FP64 or LAG_MIXED.  partitions = 0 picks the partition count automatically.
 * Cylindrical grids (lag_grid.cylindrical): B of Eq. 21 with the paper's coefficients a1 = rbar ax,
 * a2 = r az, d(r) = r d; the transform is the orthonormal DCT-II along z (zero-flux faces,
 * mu_q = (4/dz^2) sin^2(pi q / (2 nz))) and each z-mode q leaves one general tridiagonal system
 * along r with rows (-ax i/dr, ax (2i+1)/dr + r_i az mu_q + r_i d, -ax (i+1)/dr),
 * r_i = (i + 1/2) dr.  Both paths run on the tensor cores as for Cartesian plans. */
int  lag_precond_create(lag_ctx *ctx, const lag_grid *grid, double kappa_t, double rho_t,
                        double h_lag, int prec, lag_precond **out);
int  lag_precond_create_sep(lag_ctx *ctx, const lag_grid *grid, double ax_t, double az_t,
                            double d_t, int prec, int partitions, lag_precond **out);
/* Layered preconditioner (an extension of Eq. 21; the paper has no counterpart): coefficients that
 * vary with z only, ax~(z), az~(z), d~(z) (host arrays of nz values, positive / d >= 0; a shot
 * with lag_solver.layered takes the midranges of kappa and rho over each node row).  The x part
 * still commutes with the DST along x, so Sec. 2.4's separation of variables holds; each T_j
 * becomes a general tridiagonal matrix with rows
 *     (-zf_k,  zf_k + zf_{k+1} + ax~(k) lambda_j + d~(k),  -zf_{k+1}),   zf_k = az_f(k) / dz^2,
 * az_f the z-face coefficient (mean of the two rows; a boundary face takes its row's value; the
 * top face carries no flux under a free surface).  For a medium whose kappa and rho depend on z
 * only, this operator equals A.  The factors are stored per partition (nz x nx values of each of
 * five factor arrays instead of 3 L x nx).  Everything else (apply, steps, layout, autotune) is
 * as for the other plans.
 * Cylindrical grids (the radial variant): coefficients that vary with r only, arrays of nx values
 * (one per radius): the r faces take a1 = rbar ax~_face (mean of the two radii, the outer face its
 * radius's value), a2 = r az~(r), d(r) = r d~(r); the DCT-II along z still separates, and for a
 * medium whose kappa and rho depend on r only the operator equals A. */
int  lag_precond_create_layered(lag_ctx *ctx, const lag_grid *grid, const double *ax_z,
                                const double *az_z, const double *d_z, int prec, int partitions,
                                lag_precond **out);
int  lag_precond_is_layered(const lag_precond *p);   /* 1 for plans of lag_precond_create_layered */
/* Cylindrical grids only: B of Eq. 21 / Eq. 22 with a1 = rbar ax_t, a2 = r az_t and
 * d(r) = r d_t + hoop_t / r (B1 of the elastic K: ax_t = (l+2m)~, az_t = mu~, hoop_t = (l+2m)~;
 * B2: ax_t = mu~, az_t = (l+2m)~, hoop_t = 0).  LAG_EINVAL on a Cartesian grid. */
int  lag_precond_create_cyl(lag_ctx *ctx, const lag_grid *grid, double ax_t, double az_t, double d_t,
                            double hoop_t, int prec, int partitions, lag_precond **out);
void lag_precond_destroy(lag_precond *p);
/* z = B^{-1} r for nrhs fields [nrhs][nz][nx] (device, float64; cylindrical: [nrhs][nx][nz]).
 * Stream-ordered.  r and z may not overlap.  Steps: forward DST-I along x, one tridiagonal solve
 * along z per mode, DST-I (cylindrical: DCT-II along z, systems along r, inverse DCT-II). */
int  lag_precond_apply(lag_precond *p, const double *r_dev, double *z_dev, int nrhs);
/* The steps alone (parity and roofline of each kernel).  Stream-ordered.
 * dst:      y[b][k][:] = S x[b][k][:] (orthonormal DST-I, S^2 = I); in the plan's precision
 *           (cylindrical plans: y = V^T x along z, the forward DCT-II).
 * tridiag:  for every rhs b and mode j solve T_j y[b][:][j] = d[b][:][j] along z (float64 plan).
 * tridiag_f32: the same on float32 data (LAG_MIXED plan). */
int  lag_precond_dst(lag_precond *p, const double *x_dev, double *y_dev, int nrhs);
/* The inverse transform of a float64 plan: the forward one again for the DST-I (S^2 = I); for
 * cylindrical plans x = V y with the orthonormal DCT-II V[k][q] = c_q cos(pi q (k + 1/2) / n)
 * (lag_precond_dst applies V^T there).  LAG_EINVAL for mixed plans. */
int  lag_precond_dst_inverse(lag_precond *p, const double *x_dev, double *y_dev, int nrhs);
int  lag_precond_tridiag(lag_precond *p, const double *d_dev, double *y_dev, int nrhs);
int  lag_precond_tridiag_f32(lag_precond *p, const float *d_dev, float *y_dev, int nrhs);
/* Mixed plan only: y = S x from a float32 input (the inverse-transform kernel of the mixed path,
 * float32 in, float64 out).  lag_precond_dst on a mixed plan runs the forward kernel (float64 in,
 * float32 spectrum) and widens its result to float64. */
int  lag_precond_dst_f32(lag_precond *p, const float *x_dev, double *y_dev, int nrhs);
/* 1 if the plan's DST (cylindrical: DCT-II) runs on the tcgen05 tensor cores, else 0.  Mixed plans: split-bf16 operands,
 * FP32 accumulation.  Float64 plans (n >= 16, ceil(n/2) <= 4224): exact slices -- each folded row
 * and S are cut into small integer slices on a power-of-two grid (7 balanced 8-bit digits of a
 * 55-bit expansion for ceil(n/2) <= 1024, else 8 seven-bit or 9 six-bit slices), the slice products
 * are summed exactly in FP32 tensor memory (integers below 2^24) and combined in int64, so the
 * result carries float64 rounding only (relative error < 1e-14 per row in the tests).  The
 * environment variable LAGWAVE_DST_KERNEL=simt at plan creation selects the SIMT kernels. */
int  lag_precond_uses_tensor_cores(const lag_precond *p);
/* bf16 slice products the float64 tensor-core DST of length n forms per float64 multiply-add:
 * 28 (7 balanced 8-bit digits) for ceil(n/2) <= 1024 (36 with LAGWAVE_OZ_BITS=7 in the
 * environment), 36 (8 seven-bit slices) or 45 (9 six-bit slices) above; 0 where the exact-slice
 * path does not apply (n < 16 or ceil(n/2) > 4224). */
int  lag_dst_f64_slice_products(int n);
/* The GEMM kernel that the forward transform (lag_precond_dst, and the forward DST inside
 * lag_precond_apply and the solvers) of nrhs right-hand sides launches on this plan and device:
 *   LAG_GEMM_SIMT           no tensor-core GEMM (SIMT kernels)
 *   LAG_GEMM_SPLIT_BF16     mixed plan: split-bf16 operands, FP32 accumulation
 *   LAG_GEMM_SLICE_TILES    float64 exact slices, one CTA per 128 x 128 output tile
 *   LAG_GEMM_SLICE_STREAMK  float64 exact slices, the steps of all tiles cut into equal ranges, one
 *                           per SM (LAGWAVE_OZ_SK=1, opt-in: one right-hand side whose tile count is
 *                           not a multiple of the SM count)
 *   LAG_GEMM_SLICE_PAIRS    float64 exact slices on two-SM pairs (LAGWAVE_OZ_PAIR=1, opt-in)
 *   LAG_GEMM_SLICE_CLUSTER  float64 exact slices on clusters of 2 x 2, 1 x 2 or 2 x 1 tiles whose
 *                           shared operand tiles are read once and multicast (LAGWAVE_OZ_CLUSTER)
 * A negative LAG_E* code for a null plan or nrhs < 1. */
#define LAG_GEMM_SIMT 0
#define LAG_GEMM_SPLIT_BF16 1
#define LAG_GEMM_SLICE_TILES 2
#define LAG_GEMM_SLICE_STREAMK 3
#define LAG_GEMM_SLICE_PAIRS 4
#define LAG_GEMM_SLICE_CLUSTER 5
int  lag_precond_dst_gemm(lag_precond *p, int nrhs);
/* Tensor-core DST of a mixed plan: number of bf16 products per K step (3: split hi*hi + hi*lo +
 * lo*hi, relative error ~1e-5; 2: hi*hi + lo*hi with S rounded to bf16, ~2e-3; 1: hi*hi, ~4e-3).
 * Default 3 (or the environment variable LAGWAVE_DST_PRODUCTS at plan creation).  The flexible
 * Krylov solvers converge to the same float64 tolerance with any of them; fewer products move
 * fewer operand bytes and issue fewer MMAs.  LAG_EINVAL for other values or plans without the
 * tensor-core DST (3 is accepted there as a no-op). */
int  lag_precond_set_dst_products(lag_precond *p, int products);
/* z = B^{-1} r like lag_precond_apply, but allocating nothing.  The paper has no counterpart: this
 * entry point is for callers that cannot let a library allocate device memory at call time (a
 * framework whose own allocator owns the device memory, or a real-time loop that must not block in
 * cudaMalloc/cudaFree).  The intermediate spectrum lives in a file-scope static device array of
 * lag_precond_static_capacity() float64 values (2^21 = 16 MiB), which every GPU that loads the
 * library holds until the process exits; the plan is created beforehand by lag_precond_create*.
 * Float64 (LAG_FP64) plans only; the DST runs on the FP64 SIMT pipes (the tensor-core float64 DST
 * keeps operand slices in plan scratch allocated on demand), so results equal lag_precond_apply's
 * to float64 rounding.  nrhs * nz * nx beyond the capacity returns LAG_EINVAL with a
 * message in lag_last_error.  The first call on a device looks up the array's device address once
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents (nothing in it has to start at zero): calls that
 * overlap on the GPU, on any stream or context of the process, race on it.  Stream-ordered on the
 * context's stream. */
int  lag_precond_apply_static(lag_precond *p, const double *r_dev, double *z_dev, int nrhs);
size_t lag_precond_static_capacity(void);
/* Layout of the partitioned tridiagonal solve (Sec. 1; partitions are the paper's subdomains, here
 * threads of one CTA): partitions 1..32 (0 = automatic, the largest count with >= 2 rows each) and
 * the register kernel's mode tile, the x-modes one CTA solves together (float32 plans 8, 16, 32
 * (the last only with partition length <= 32), float64 plans 4, 8; 0 = default 16 / 4).  Rebuilds
 * the factors (blocking).  LAG_EINVAL for values outside those sets or a tile the layout cannot
 * use (partition length > 64, which takes the shared-memory kernel). */
int  lag_precond_set_layout(lag_precond *p, int partitions, int modes_per_cta);
/* Autotuner (no counterpart in the paper; the tuning choices of this implementation): times every
 * (partition count 8, 16, 32) x (mode tile, see lag_precond_set_layout) layout of the tridiagonal
 * solve and, on mixed plans with the tensor-core DST, the bf16 product counts 3, 2 and 1 on nrhs
 * seeded right-hand sides (a few applies each, CUDA events on the context's stream), keeps the
 * fastest (a product count only if its result is within 2e-2 relative L2 of the 3-product split)
 * and leaves the plan configured with it.  Blocking; allocates 3 nrhs nz nx float64 scratch values
 * for the duration of the call.  Outputs may be NULL. */
int  lag_precond_autotune(lag_precond *p, int nrhs, int *partitions_out, int *modes_per_cta_out,
                          int *products_out, double *ms_per_apply_out);
/* plan facts: partitions P, partition length L, modes per CTA of the tridiagonal kernel */
int  lag_precond_info(const lag_precond *p, int *partitions, int *part_len, int *modes_per_cta);
/* Waits for the context's stream, then reports the plan's device error word: LAG_OK, or
 * LAG_ETIMEDOUT when a bounded pipeline wait inside the tensor-core DST gave up since the plan was
 * created (sticky; that apply's output is invalid and the plan should be rebuilt).  Krylov solves
 * and shots read the same word after every chunk of iterations and fail with LAG_ETIMEDOUT. */
int  lag_precond_status(lag_precond *p);

/* ---------------------------------------------------------------- medium and operator
 * Acoustic (Sec. 2.3, Eqs. 16-18, Cartesian SPD form): face coefficient = mean of the two nodal
 * kappa (boundary faces take the interior node's value), mass w = rho h^2/4.
 * Elastic (Eq. 12, plane strain): second-derivative terms with face-averaged (lambda+2mu) and mu,
 * mixed terms as centred differences with nodal lambda and mu; lambda = rho (vp^2 - 2 vs^2),
 * mu = rho vs^2.  Host arrays [nz][nx] are copied. */
int  lag_medium_create_acoustic(lag_ctx *ctx, const lag_grid *grid, const double *c_host,
                                const double *rho_host, double h_lag, lag_medium **out);
int  lag_medium_create_elastic(lag_ctx *ctx, const lag_grid *grid, const double *vp_host,
                               const double *vs_host, const double *rho_host, double h_lag,
                               lag_medium **out);
void lag_medium_destroy(lag_medium *m);
/* Midranges computed on the device: acoustic out[0..1] = kappa~, rho~; elastic out[0..2] =
 * (lambda+2mu)~, mu~, rho~.  Blocking. */
int  lag_medium_midranges(lag_medium *m, double *out);
/* q = A p (acoustic: [nrhs][nz][nx]) or q = C p (elastic: [nrhs][2][nz][nx]).  Stream-ordered. */
int  lag_apply_operator(lag_medium *m, const double *p_dev, double *q_dev, int nrhs);

/* ---------------------------------------------------------------- one harmonic system
 * Solve A x = b (acoustic: PCG with B; plain CG beta of Fletcher-Reeves for LAG_FP64, flexible
 * Polak-Ribiere for LAG_MIXED) or C x = b (elastic: right-preconditioned flexible GMRES(k) with
 * K = diag(B1, B2)) for nrhs independent right-hand sides, zero initial guess.  Blocking.
 * iters_host[nrhs] / relres_host[nrhs] (may be NULL) receive per-rhs results.
 * The preconditioner plans must match the medium's grid and the solver's precision. */
int  lag_solve_system(lag_medium *m, lag_precond *p1, lag_precond *p2, const double *b_dev,
                      double *x_dev, int nrhs, const lag_solver *s, int *iters_host,
                      double *relres_host);

/* ---------------------------------------------------------------- Laguerre pieces (Sec. 2.1)
 * f_m = int f(t) (ht)^{-alpha/2} l_m(ht) dt, m < n_harm, by composite Gauss-Legendre on the
 * wavelet's support; computed on the device, copied to fm_host[n_harm]. */
int  lag_source_coeffs(lag_ctx *ctx, const lag_laguerre *lag, const lag_wavelet *w, double *fm_host);
/* tab[m][j] = (h t_j)^{alpha/2} l_m(h t_j) for the inverse summation u(t) = sum_m R_m tab[m][.]
 * (Eq. 8); l_m evaluated by a scaled three-term recurrence.  Copied to tab_host[n_harm][nt]. */
int  lag_laguerre_table(lag_ctx *ctx, const lag_laguerre *lag, int nt, const double *t_host,
                        double *tab_host);

/* ---------------------------------------------------------------- shots (whole Laguerre loops)
 * A shot holds the device-resident state of nsrc sources on one medium: the Krylov vectors, the
 * two running history sums T, S per source (S_m = sum_{k<m}(m-k) c^_k R_k, updated as
 * T += c^_m R_m, S += T), the receiver values of every harmonic, and its own CUDA stream
 * (created by the library).  vs_host == NULL selects the acoustic problem. */
int  lag_shot_create(lag_ctx *ctx, const lag_grid *grid, const double *c_host, const double *vs_host,
                     const double *rho_host, const lag_laguerre *lag, const lag_solver *s,
                     const lag_wavelet *w, int nsrc, const lag_point *src, int nrcv,
                     const lag_point *rcv, int nt, const double *t_out_host, lag_shot **out);
void lag_shot_destroy(lag_shot *sh);
/* Advance up to nharm harmonics (blocking).  Returns LAG_OK, LAG_ENOTCONV (a harmonic hit
 * max_iter; the shot continues from the best iterate) or an error. */
int  lag_shot_step(lag_shot *sh, int nharm);
/* Non-blocking progress: issues the next chunk of work if the previous one finished.
 * *done is set to 1 when all n_harm harmonics are finished. */
int  lag_shot_pump(lag_shot *sh, int *done);
int  lag_shot_harmonic(const lag_shot *sh);          /* harmonics completed so far              */
void *lag_shot_stream(const lag_shot *sh);           /* the shot's cudaStream_t                 */
/* traces[nsrc][ncomp][nrcv][nt] (ncomp = 1 acoustic, 2 elastic) summed over the harmonics done */
int  lag_shot_traces(lag_shot *sh, double *traces_host);
/* receiver values of every finished harmonic: R_rcv[n_harm][nsrc][ncomp][nrcv] */
int  lag_shot_receiver_harmonics(lag_shot *sh, double *rrcv_host);
/* device pointer to the latest solved harmonic R_m ([nsrc][ncomp][nz][nx]); valid until the next step */
const double *lag_shot_field(const lag_shot *sh);
/* copy the latest solved harmonic into out_dev ([nsrc][ncomp][nz][nx], device); blocking */
int  lag_shot_copy_field(lag_shot *sh, double *out_dev);
int  lag_shot_stats(const lag_shot *sh, lag_stats *st);
/* Checkpoint between harmonics (no counterpart in the paper): the state after harmonic m is m, the
 * two history sums of every source, the receiver values of harmonics < m and the statistics.
 * checkpoint copies it into host_buf (lag_shot_checkpoint_size bytes, blocking); restore loads it
 * into a shot created from the same inputs, which then continues with identical arithmetic
 * (a resumed run equals an uninterrupted one bit for bit).  LAG_EINVAL on a size/shape mismatch. */
size_t lag_shot_checkpoint_size(const lag_shot *sh);
int  lag_shot_checkpoint(lag_shot *sh, void *host_buf, size_t bytes);
int  lag_shot_restore(lag_shot *sh, const void *host_buf, size_t bytes);

/* Whole shot in one call: create, step all harmonics, copy traces, destroy.  Blocking.
 * traces_host[nsrc][nrcv][nt] (acoustic) or [nsrc][2][nrcv][nt] (elastic). */
int  lag_solve_acoustic(lag_ctx *ctx, const lag_grid *grid, const double *c_host,
                        const double *rho_host, const lag_laguerre *lag, const lag_solver *s,
                        const lag_wavelet *w, int nsrc, const lag_point *src, int nrcv,
                        const lag_point *rcv, int nt, const double *t_out_host,
                        double *traces_host, lag_stats *stats);
int  lag_solve_elastic(lag_ctx *ctx, const lag_grid *grid, const double *vp_host,
                       const double *vs_host, const double *rho_host, const lag_laguerre *lag,
                       const lag_solver *s, const lag_wavelet *w, int nsrc, const lag_point *src,
                       int nrcv, const lag_point *rcv, int nt, const double *t_out_host,
                       double *traces_host, lag_stats *stats);

/* ---------------------------------------------------------------- serving
 * Continuous batching of shots: a request is admitted when its device memory fits the context's
 * HBM budget next to the running ones, then advanced chunk by chunk on its own stream alongside
 * every other admitted request (work of different requests overlaps on the device; results do not
 * depend on what else runs).  The request's host arrays are copied at submit. */
typedef struct {
  int kind;                    /* 0 acoustic, 1 elastic                                   */
  lag_grid grid;
  const double *c_host;        /* c (acoustic) or vp (elastic) [nz][nx]                    */
  const double *vs_host;       /* elastic only                                            */
  const double *rho_host;
  lag_laguerre lag;
  lag_solver solver;
  lag_wavelet wavelet;
  int nsrc; const lag_point *src;
  int nrcv; const lag_point *rcv;
  int nt;   const double *t_out_host;
} lag_request;

typedef struct {
  int status;                  /* LAG_OK, LAG_ENOTCONV, LAG_ECANCELED, ...                 */
  double *traces_host;         /* caller-provided [nsrc][ncomp][nrcv][nt], filled by poll  */
  double t_submit, t_admit, t_done;   /* seconds since the context was created             */
  long long total_iters;
  size_t device_bytes;         /* device memory the request held                           */
  int harmonics_done;          /* harmonics solved (all of them unless cancelled or failed) */
} lag_result;

/* Failure-detection self-test (no counterpart in the paper): launches one kernel that waits on an
 * mbarrier nothing arrives on, for at most `polls` polls (about 1 us each), and returns
 * LAG_ETIMEDOUT when the bounded wait gives up; the context stays usable.  Every wait in the
 * library's kernels is bounded the same way and reports through an error word. */
int lag_selftest_wait_timeout(lag_ctx *ctx, long long polls);

int lag_serve_start(lag_ctx *ctx, int max_active);   /* starts the scheduler thread       */
int lag_serve_stop(lag_ctx *ctx);                    /* drains nothing: cancels the rest  */
int lag_serve_submit(lag_ctx *ctx, const lag_request *req, uint64_t *ticket);
int lag_serve_poll(lag_ctx *ctx, uint64_t ticket, lag_result *out);  /* LAG_EAGAIN until done */
int lag_serve_cancel(lag_ctx *ctx, uint64_t ticket);

#ifdef __cplusplus
}
#endif
#endif /* LAGWAVE_H */
