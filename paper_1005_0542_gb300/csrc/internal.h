// Host-side structures of the library and the launchers of its kernels.
#pragma once

#include <atomic>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lagwave.h"
#include "common.cuh"

// ----------------------------------------------------------------------------- context
struct lag_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;                 // 0 = unlimited
  std::atomic<size_t> in_use{0};
  std::string last_error;
  double t_created = 0.0;
  struct Server *server = nullptr;   // serving loop (lazily created)
  std::mutex mem_mu;
};

void server_destroy(lag_ctx *ctx);  // stops the serving thread of ctx, if any

namespace lag {

double now_seconds();

// ------------------------------------------------------------------ kernel-class timing
enum KClass { KC_DST64 = 0, KC_DST32_FWD, KC_DST32_INV, KC_DSTTC_FWD, KC_DSTTC_INV, KC_TRI64, KC_TRI32,
              KC_STENCIL_A, KC_STENCIL_E, KC_VEC, KC_LAGUERRE, KC_GMRES, KC_SETUP, NK_CLASSES };
const char *kclass_name(int c);
bool profiling_on();  // kernel-class timing enabled (no graph capture then: events are per launch)
// Records a CUDA event pair around the launches in its scope when profiling is enabled.
struct ProfScope {
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  bool active = false;
  ProfScope(int c, cudaStream_t st);
  ~ProfScope();
};

// Device buffer owned by a context; counted against its HBM budget.
struct DevBuf {
  lag_ctx *ctx = nullptr;
  void *ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void alloc(lag_ctx *c, size_t nbytes, bool zero = false);
  void release();
  template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// ----------------------------------------------------------------- tridiagonal plan (a2, a8)
// Factors of the partitioned solve for every x-mode (see k_tridiag.cu for the algorithm).
struct TriFactors {
  int nx = 0, nz = 0;   // modes, rows
  int P = 1, L = 1;     // partitions, partition length (P * L >= nz; rows >= nz are identity)
  int ncls = 1;         // factor sets (3 classes for Toeplitz-in-z systems, one per partition in general)
  bool gen = false;     // general (layered) systems: one factor set per partition
  int levels = 0;       // PCR levels of the reduced system (P - 1 unknowns)
  int nf = 3;           // values per separator in the reduced block: 3 + 3 * levels
  int mt = 1;           // modes per CTA
  int threads = 32;     // threads per CTA (mt * P rounded up to whole warps)
  bool reg = false;     // register-resident kernel (L a power of two <= 64)
  size_t smem = 0;      // dynamic shared memory of the solve kernel
  // device arrays, element type double or float: [cls][i][j] with j fastest
  void *fm = nullptr, *fc = nullptr, *fa = nullptr, *sv = nullptr, *sw = nullptr;
  void *red = nullptr;  // [j][nf][32]
};

void tri_choose_layout(TriFactors &tf, int elem_bytes, int want_P, int want_mt = 0, bool general = false);
bool tri_mode_tile_ok(int elem_bytes, int L, int mt);
// Coefficients of the z-systems T_j.  Constant (Eq. 21 midranges): T_j = tridiag(-az/dz^2,
// 2 az/dz^2 + ax lambda_j + d, -az/dz^2); free_surface: row 0 has no flux through its top face
// (diagonal az/dz^2 + ax lambda_j + d).  Layered (zrows != null, device, nz*3 + 1 values):
// [zf: nz + 1 z-face coefficients over dz^2 | ax(z): nz | d(z): nz], row k of T_j being
// (-zf[k], zf[k] + zf[k+1] + ax(k) lambda_j + d(k), -zf[k+1]); the free surface is zf[0] = 0.
struct TriCoef {
  double ax = 0, az = 0, d = 0;
  const double *zrows = nullptr;
  bool free_surface = false;
  bool dct = false;  // modes of a DCT-II plan (cylindrical z): lambda_j = 4/dx^2 sin^2(pi j / (2 nx))
};
// Build float64 factors of every T_j on the device (tf.gen must equal k.zrows != null).
// perm_ku > 0: column c holds mode 2c (c < perm_ku) or 2(c - perm_ku) + 1 (parity-permuted spectra)
void tri_build_factors(TriFactors &tf, DevBuf &store, const TriCoef &k, double dx, double dz, cudaStream_t s,
                       int perm_ku = 0);
// Round a float64 factor set to float32 into `store32` (same layout).
void tri_make_f32(const TriFactors &t64, TriFactors &t32, DevBuf &store32, cudaStream_t s);
// y = T^{-1} d per (plane, mode); d and y [planes][nz][nx]; in place allowed.  The launch covers
// `nplanes` planes pstride * i + poff; sc (nullable) skips planes whose right-hand side
// (plane / ncomp) is no longer iterating.
void tri_solve_f64(const TriFactors &tf, const double *d, double *y, int nplanes,
                   const KrylovScalars *sc, cudaStream_t s, int pstride = 1, int poff = 0,
                   int ncomp = 1);
void tri_solve_f32(const TriFactors &tf, const float *d, float *y, int nplanes,
                   const KrylovScalars *sc, cudaStream_t s, int pstride = 1, int poff = 0,
                   int ncomp = 1);
// y = T^{-1} d for nrhs one-component planes (d != y) and, per plane b, (d, y) summed in a fixed
// order into rz_new, then PCG's Fletcher-Reeves beta = rz_new / sc[b].rz (0 on a solve's first
// iteration) and sc[b].rz = rz_new.  Between z = S T^{-1} S r and d = S r with one symmetric S
// (the DST-I on both sides), (d, y) = (S r, T^{-1} S r) = (r, z).  Only where
// tri_rz_fusable (the register kernel, and no more CTAs per plane than red holds blocks).
bool tri_rz_fusable(const TriFactors &tf, const Reduce &red);
void tri_solve_f64_rz(const TriFactors &tf, const double *d, double *y, int nrhs, KrylovScalars *sc,
                      const Reduce &red, cudaStream_t s);

// ----------------------------------------------------------------- DST (a7, a9)
struct DstPlan {
  int kind = 0;         // 0: DST-I (Dirichlet, self-inverse); 1: DCT-II (zero-flux faces, cylindrical z)
  int n = 0;            // transform length nx
  int ku = 0, kv = 0;   // ceil(n/2), floor(n/2): inner dimensions of the two folded GEMMs
  double *su = nullptr; // [ku][ku]  S[j][2k]    (float64)
  double *sv = nullptr; // [kv][kv]  S[j][2k+1]
  float *su_f = nullptr, *sv_f = nullptr;  // float32 copies (SIMT float32 kernel)
  // DCT-II inverse (kind 1): ie [ku][ku] = V[k][2q'] as [q'][k], io [kv][ku] = V[k][2q'+1] as [q'][k]
  double *ie = nullptr, *io = nullptr;
  float *ie_f = nullptr, *io_f = nullptr;
  // tensor-core path: four packed split-bf16 B operands (forward even/odd, inverse E/O), each
  // [n tile][k stage][hi|lo][256 x 64 swizzled]; per-apply A-operand / E-O scratch; error word
  uint8_t *tc_b = nullptr;
  size_t tc_bmat_bytes = 0;
  int kpad_u = 0;             // K stages (64 wide)
  int npad_u = 0;             // N tiles (256 wide)
  uint8_t *tc_scratch = nullptr;
  int *tc_err = nullptr;
  int tc_products = 3;        // split products per K step: 3 (hi*hi+hi*lo+lo*hi), 2 or 1
  // float64 path on the tensor cores (exact slices): packed B slices [2][9][n tile][k stage]
  bool oz = false;
  uint8_t *oz_b = nullptr;
  uint8_t *oz_bi = nullptr;   // DCT-II inverse operands (kind 1): [2][9][n tile][k stage]
  size_t oz_slice_bytes = 0;
  int oz_eB = 0;              // |S| < 2^oz_eB
  int oz_nb = 6, oz_ns = 9;   // exact slices: bits per slice, slices per operand
};
// tc_mode: 0 none, 1 split-bf16 operands (mixed path), 2 exact slices (float64 path); kind 0 = DST-I,
// 1 = DCT-II (both fold alike; the DCT-II adds inverse operands, see k_dst.cu)
void dst_build(DstPlan &dp, DevBuf &store, int n, int tc_mode, cudaStream_t s, int kind = 0);
// the inverse transform: the forward one again for DST-I (S^2 = I), the transpose for DCT-II
void dst_inverse_f64(const DstPlan &dp, const double *x, double *y, int rows, int rows_per_rhs,
                     const KrylovScalars *sc, cudaStream_t s);
void dst_inverse_f64_simt(const DstPlan &dp, const double *x, double *y, int rows, int rows_per_rhs,
                          const KrylovScalars *sc, cudaStream_t s);
// rscale (PCG only, sc non-null): the float32 pipeline sees each right-hand side scaled by 2^-e,
// e = the binary exponent of its residual norm sc[b].rr, undone exactly on the float64 output
void dst_inverse_f32_f2d(const DstPlan &dp, const float *x, double *y, int rows, int rows_per_rhs,
                         const KrylovScalars *sc, cudaStream_t s, bool rscale = false);
// Y[row][:] = S X[row][:] for `rows` rows of length n.  Input/output types as named.
void dst_apply_f64(const DstPlan &dp, const double *x, double *y, int rows, int rows_per_rhs,
                   const KrylovScalars *sc, cudaStream_t s);
// the same on the FP64 SIMT pipes (no scratch; the no-allocation entry point uses it)
void dst_apply_f64_simt(const DstPlan &dp, const double *x, double *y, int rows, int rows_per_rhs,
                        const KrylovScalars *sc, cudaStream_t s);
// exact-slice tensor-core float64 DST (dp.oz); scratch dp.tc_scratch of dst_oz_scratch_bytes
bool dst_oz_supported(int n);
int dst_oz_products(int n);  // bf16 slice products per float64 product of a length-n transform
size_t dst_oz_scratch_bytes(const DstPlan &dp, int rows);
// exact-slice GEMM kernels (the values of LAG_GEMM_SLICE_* in lagwave.h)
constexpr int OZ_GEMM_TILES = 2, OZ_GEMM_STREAMK = 3, OZ_GEMM_PAIRS = 4, OZ_GEMM_CLUSTER = 5;
int dst_oz_gemm_variant(const DstPlan &dp, int rows, int rpr, int inv);
// inverse (DCT-II plans only): gather the even / odd modes, GEMM with the inverse operands into
// E / O sums (plan scratch), butterfly into y
void dst_apply_oz(const DstPlan &dp, const double *x, double *y, int rows, int rows_per_rhs,
                  const KrylovScalars *sc, cudaStream_t s, bool inverse = false);
// mixed path on SIMT float32 arithmetic: float64 in -> float32 out and float32 in -> float64 out
void dst_apply_f32_d2f(const DstPlan &dp, const double *x, float *y, int rows, int rows_per_rhs,
                       const KrylovScalars *sc, cudaStream_t s, bool rscale = false);
void dst_apply_f32_f2d(const DstPlan &dp, const float *x, double *y, int rows, int rows_per_rhs,
                       const KrylovScalars *sc, cudaStream_t s, bool rscale = false);
// mixed path: float64 in -> float32 out, and float32 in -> float64 out (tensor cores)
// rscale: PCG residual scaling (see dst_inverse_f32_f2d); the fused _beta variant always scales
void dst_apply_tc_d2f(const DstPlan &dp, const double *x, float *y, int rows, int rows_per_rhs,
                      const KrylovScalars *sc, cudaStream_t s, bool rscale = false);
void dst_apply_tc_f2d(const DstPlan &dp, const float *x, double *y, int rows, int rows_per_rhs,
                      const KrylovScalars *sc, cudaStream_t s, bool rscale = false);
bool dst_tc_supported(int n);
// inverse tensor-core DST fused with the CG beta of the next step (per rhs: rpr rows)
void dst_apply_tc_f2d_beta(const DstPlan &dp, const float *y, double *z, int nrhs, int rpr, const double *r,
                           const double *q, int flexible, KrylovScalars *sc, const Reduce &red, cudaStream_t s);
size_t dst_tc_scratch_bytes(const DstPlan &dp, int rows);
// parity permutation of a float32 spectrum: natural mode order <-> [even modes | odd modes]
void spectrum_permute(const float *in, float *out, int rows, int n, int ku, bool to_perm, cudaStream_t s);
void spectrum_unpermute_widen(const float *in, double *out, int rows, int n, int ku, cudaStream_t s);

}  // namespace lag

// ----------------------------------------------------------------------------- preconditioner
struct lag_precond {
  lag_ctx *ctx = nullptr;
  lag_grid grid{};
  int prec = LAG_FP64;
  double ax = 0, az = 0, d = 0;
  lag::DevBuf zrows;        // general z-systems: z-face / per-row coefficients (see lag::TriCoef)
  bool layered = false;     // built from per-row (or per-radius) midranges, not the whole medium's
  lag::TriCoef coef() const;
  lag::DstPlan dst;
  lag::TriFactors tri64, tri32;
  lag::DevBuf dst_store, tri_store, tri32_store;
  lag::DevBuf scratch;      // intermediate spectra (float64 or float32), grows with nrhs
  lag::DevBuf tc_scratch;   // tensor-core DST: packed A operands and E/O halves
  int scratch_rhs = 0;
  bool use_tc = false;      // mixed path: DST on tcgen05 tensor cores (else SIMT float32)
  void ensure_scratch(int nplanes);
  // z = B^{-1} r for nrhs planes; sc (nullable) lets converged right-hand sides skip the work;
  // rscale: r is a PCG residual whose norm is sc[b].rr (scales the float32 SIMT pipeline)
  void apply(const double *r, double *z, int nrhs, const lag::KrylovScalars *sc, cudaStream_t s,
             bool rscale = false);
};

namespace lag {
// K^{-1} for ncomp interleaved components ([rhs][comp][nz][nx]): component 0 with p1, 1 with p2.
void precond_apply_multi(lag_precond *p1, lag_precond *p2, const double *r, double *z, int nrhs,
                         int ncomp, const KrylovScalars *sc, cudaStream_t s);
}

// ----------------------------------------------------------------------------- medium
struct lag_medium {
  lag_ctx *ctx = nullptr;
  lag_grid grid{};
  bool elastic = false;
  double h = 0;
  double mid[3] = {0, 0, 0};   // kappa~, rho~ | (l+2m)~, mu~, rho~
  lag::DevBuf coef;            // operator coefficients (see k_ops.cu)
  lag::DevBuf rho_h2;          // rho h^2 at nodes (right-hand side history term)
  lag::DevBuf rowmm;           // per-row [nz][min, max] of [kappa | rho] (acoustic) or [lambda+2mu | mu |
                               // rho] (Cartesian elastic), for the layered preconditioner
  size_t ncoef = 0;
  // q = C p (elastic) or A p; sub (elastic only, nullable): q = C p - sub, same layout as q
  void apply(const double *p, double *q, int nrhs, const lag::KrylovScalars *sc,
             const lag::Reduce *red, int mode, cudaStream_t s, const double *sub = nullptr);
};

namespace lag {
// ----------------------------------------------------------------- operator and vector kernels
void medium_build_acoustic(lag_medium &m, const double *c_host, const double *rho_host,
                           cudaStream_t s);
// cylindrical (r, z) acoustic medium on the kernel grid (rows = radii; see kernel_grid)
void medium_build_cylindrical(lag_medium &m, const double *c_host, const double *rho_host, cudaStream_t s);
// cylindrical (r, z) elastic medium: energy-derived axisymmetric operator (k_elastic_cyl.cu)
void medium_build_elastic_cylindrical(lag_medium &m, const double *vp_host, const double *vs_host,
                                      const double *rho_host, cudaStream_t s);
void elastic_cyl_apply(const lag_medium &m, const double *p, double *q, int nrhs, const KrylovScalars *sc,
                       int mode, cudaStream_t s, const double *sub);
void medium_build_elastic(lag_medium &m, const double *vp_host, const double *vs_host,
                          const double *rho_host, cudaStream_t s);
// The grid the kernels run on.  Cartesian: the user's grid.  Cylindrical (fields [nr][nz], depth
// fastest): rows are the radii and the row length the depth nodes, i.e. nx = nz_user,
// nz = nr, dx = dz_user, dz = dr (the transform runs along z, the tridiagonal systems along r).
// Throws LAG_EINVAL on an inconsistent grid.
lag_grid kernel_grid(const lag_grid &g);
// build a medium / a separable preconditioner plan on stream s (blocking); both take the user's grid
// and keep the kernel grid
lag_medium *medium_new(lag_ctx *ctx, const lag_grid &g, const double *c, const double *vs,
                       const double *rho, double h, cudaStream_t s);
// rebuild the tridiagonal factors with another partition count / register-kernel mode tile
// (0 = automatic); used by lag_precond_set_layout and the autotuner
void precond_rebuild_tri(lag_precond *p, int want_P, int want_mt, cudaStream_t s);
// layered (nullable, host): [ax(z): nz | az(z): nz | d(z): nz] per-row coefficients; then ax, az, d
// are unused
// hoop (cylindrical grids only): d(r) = r d + hoop / r (the (l+2m)~/r term of B1, Eq. 22)
lag_precond *precond_new(lag_ctx *ctx, const lag_grid &g, double ax, double az, double d, int prec,
                         int partitions, cudaStream_t s, const double *layered = nullptr, double hoop = 0.0);
// mode 0: q = Ap only; mode 1: also (p,q) -> alpha = rz/pq  (PCG)
void acoustic_apply(const lag_medium &m, const double *p, double *q, int nrhs,
                    const KrylovScalars *sc, const Reduce *red, int mode, cudaStream_t s);
void elastic_apply(const lag_medium &m, const double *p, double *q, int nrhs,
                   const KrylovScalars *sc, const Reduce *red, int mode, cudaStream_t s,
                   const double *sub = nullptr);

int reduce_blocks(size_t n);  // blocks per rhs of the vector kernels for n values per rhs

// p_new = z + beta p_old, q = A p_new, (p_new, q) -> alpha (PCG's direction update and operator in
// one pass; p_new and p_old are different buffers)
void acoustic_apply_dir(const lag_medium &m, const double *z, const double *pold, double *pnew, double *q,
                        int nrhs, const KrylovScalars *sc, const Reduce &red, cudaStream_t s);

// PCG pieces (per rhs, n values each).  One iteration: z = B^{-1} r and beta (0 on the first), the
// direction update with q = A p and alpha, then x, r and the convergence test.
void pcg_start(const double *b, double *x, double *r, double *p, size_t n, int nrhs, double tol,
               KrylovScalars *sc, const Reduce &red, cudaStream_t s);
void pcg_update_xr(double *x, double *r, const double *p, const double *q, size_t n, int nrhs,
                   int max_iter, KrylovScalars *sc, const Reduce &red, cudaStream_t s);
void pcg_beta(const double *r, const double *z, const double *q, size_t n, int nrhs, int flexible,
              KrylovScalars *sc, const Reduce &red, cudaStream_t s);

// FGMRES pieces: vectors of n values per rhs; V, Z: [k+1][nrhs][n] bases; H: [nrhs][(k+1)*k]
struct GmresDev {
  double *H, *cs, *sn, *g, *y;   // per rhs: H [(k+1) k], cs/sn [k], g [k+1], y [k]
  double *hcol;                  // per rhs: [k+1] current column (Gram-Schmidt coefficients)
  int k;
};
void gm_start(const double *b, const double *cx, double *v0, size_t n, int nrhs, int first,
              double tol, int max_iter, KrylovScalars *sc, GmresDev &g, const Reduce &red,
              cudaStream_t s);
// shifted: w holds C z_j - V_j (the shifted Arnoldi step); h_jj gets the 1 back
void gm_orthogonalize(double *w, const double *V, int j, size_t n, int nrhs, size_t vstride,
                      KrylovScalars *sc, GmresDev &g, const Reduce &red, int pass, bool shifted,
                      cudaStream_t s);
void gm_normalize(double *w, double *vnext, int j, size_t n, int nrhs, KrylovScalars *sc,
                  GmresDev &g, const Reduce &red, int max_iter, cudaStream_t s);
void gm_update_x(double *x, const double *Z, int jdone, size_t n, int nrhs, size_t zstride,
                 const KrylovScalars *sc, GmresDev &g, cudaStream_t s);

// Laguerre pieces
void source_coeffs_device(const lag_laguerre &lag, const lag_wavelet &w, double *fm_dev,
                          DevBuf &scratch, lag_ctx *ctx, cudaStream_t s);
void laguerre_table_device(const lag_laguerre &lag, int nt, const double *t_dev, double *tab_dev,
                           cudaStream_t s);
// r = -c_m rho h^2 S (+ f_m/(dx dz) at each source), x = 0, p = 0 (p nullable), ||r||^2 -> sc.bb;
// per rhs/comp.
void laguerre_rhs(const double *rho_h2, const double *S, double cm, const double *fm, int m,
                  const int *src_idx, int src_comp, double inv_cell, int ncomp, size_t nplane,
                  int nrhs, double *r, double *x, double *p, double tol, KrylovScalars *sc,
                  const Reduce &red, cudaStream_t s);
void laguerre_accumulate(const double *x, double *T, double *S, double chat, size_t n, int nrhs,
                         cudaStream_t s);
void gather_receivers(const double *x, const int *rcv_idx, int nrcv, int ncomp, size_t nplane,
                      int nrhs, double *out, cudaStream_t s);
void inverse_sum(const double *rrcv, const double *tab, int nharm, int nrows, int nt,
                 double *traces, cudaStream_t s);
void midrange_device(const double *f, size_t n, double *minmax_dev, cudaStream_t s);
// per-row min/max of f [nz][nx] -> minmax_dev [nz][2]
void row_minmax_device(const double *f, int nx, int nz, double *minmax_dev, cudaStream_t s);

}  // namespace lag
