// Stencil operator, PCG vector updates and Laguerre-series kernels (all float64).
//
// Acoustic operator (Sec. 2.3, Eqs. 16-18, Cartesian SPD form, Dirichlet frame):
//   (A p)_{k,i} = dg p_c - axW p_w - axE p_e - azN p_n - azS p_s,
//   axW/axE = kappa at the x-faces / dx^2 (face = mean of the two nodes, boundary face = node),
//   azN/azS likewise in z, dg = axW + axE + azN + azS + rho h^2 / 4.
// Coefficients are built once per medium and shared by every right-hand side.
// PCG (Sec. 2.3) keeps every scalar on the device: each reduction is finished by the last block
// of its kernel (deterministic order), which also forms alpha / beta / the convergence state.
#include "internal.h"

namespace lag {

unsigned long long g_launches = 0;
thread_local bool g_capturing = false;

// ------------------------------------------------------------------------------ medium
__global__ void acoustic_coef_kernel(const double *__restrict__ c, const double *__restrict__ rho, int nx, int nz,
                                     double idx2, double idz2, double h2, double *ax, double *az, double *dg,
                                     double *rh2, double *kap, int free_surface) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i > nx || k > nz) return;
  auto K = [&](int kk, int ii) { const size_t o = (size_t)kk * nx + ii; return rho[o] * c[o] * c[o]; };
  if (k < nz) {  // x-face i of row k (between nodes i-1 and i)
    const double v = (i == 0) ? K(k, 0) : (i == nx ? K(k, nx - 1) : 0.5 * (K(k, i - 1) + K(k, i)));
    ax[(size_t)k * (nx + 1) + i] = v * idx2;
  }
  if (i < nx) {  // z-face k of column i (the top face carries no flux under a free surface)
    const double v = (k == 0) ? (free_surface ? 0.0 : K(0, i)) : (k == nz ? K(nz - 1, i) : 0.5 * (K(k - 1, i) + K(k, i)));
    az[(size_t)k * nx + i] = v * idz2;
  }
  if (i < nx && k < nz) {
    const size_t o = (size_t)k * nx + i;
    rh2[o] = rho[o] * h2;
    kap[o] = K(k, i);
  }
}

__global__ void acoustic_diag_kernel(const double *ax, const double *az, const double *rh2, int nx, int nz, double *dg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= nx || k >= nz) return;
  const size_t o = (size_t)k * nx + i;
  dg[o] = ax[(size_t)k * (nx + 1) + i] + ax[(size_t)k * (nx + 1) + i + 1] + az[(size_t)k * nx + i] +
          az[(size_t)(k + 1) * nx + i] + 0.25 * rh2[o];
}

// min/max of f[blockIdx.x * n ...][n] -> out[2 blockIdx.x], out[2 blockIdx.x + 1] (setup only; one
// block per row, or one block for the whole array)
__global__ void minmax_kernel(const double *f, size_t n, double *out) {
  f += (size_t)blockIdx.x * n;
  out += 2 * (size_t)blockIdx.x;
  double lo = INFINITY, hi = -INFINITY;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) { lo = fmin(lo, f[i]); hi = fmax(hi, f[i]); }
  __shared__ double sl[32], sh[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sl[w] = lo; sh[w] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { lo = fmin(lo, sl[k]); hi = fmax(hi, sh[k]); }
    lo = fmin(lo, sl[0]);
    hi = fmax(hi, sh[0]);
    out[0] = lo;
    out[1] = hi;
  }
}

void midrange_device(const double *f, size_t n, double *minmax_dev, cudaStream_t s) {
  minmax_kernel<<<1, 1024, 0, s>>>(f, n, minmax_dev);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void row_minmax_device(const double *f, int nx, int nz, double *minmax_dev, cudaStream_t s) {
  minmax_kernel<<<nz, 256, 0, s>>>(f, (size_t)nx, minmax_dev);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// layout of lag_medium::coef (acoustic): ax [nz][nx+1] | az [nz+1][nx] | dg [nz][nx] | kappa [nz][nx]
void medium_build_acoustic(lag_medium &m, const double *c_host, const double *rho_host, cudaStream_t s) {
  const int nx = m.grid.nx, nz = m.grid.nz;
  const size_t n = (size_t)nx * nz;
  const size_t nax = (size_t)nz * (nx + 1), naz = (size_t)(nz + 1) * nx;
  m.ncoef = nax + naz + 2 * n;
  m.coef.alloc(m.ctx, m.ncoef * sizeof(double));
  m.rho_h2.alloc(m.ctx, n * sizeof(double));
  DevBuf tmp;
  tmp.alloc(m.ctx, (2 * n + 4) * sizeof(double));
  double *dc = tmp.as<double>(), *drho = dc + n, *mm = drho + n;
  LAG_CUDA_CHECK(cudaMemcpyAsync(dc, c_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(drho, rho_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  double *ax = m.coef.as<double>(), *az = ax + nax, *dg = az + naz, *kap = dg + n;
  dim3 g((nx + 1 + 127) / 128, nz + 1);
  acoustic_coef_kernel<<<g, 128, 0, s>>>(dc, drho, nx, nz, 1.0 / (m.grid.dx * m.grid.dx),
                                         1.0 / (m.grid.dz * m.grid.dz), m.h * m.h, ax, az, dg,
                                         m.rho_h2.as<double>(), kap, m.grid.free_surface ? 1 : 0);
  count_launch();
  LAG_LAUNCH_CHECK();
  dim3 g2((nx + 127) / 128, nz);
  acoustic_diag_kernel<<<g2, 128, 0, s>>>(ax, az, m.rho_h2.as<double>(), nx, nz, dg);
  count_launch();
  LAG_LAUNCH_CHECK();
  // midranges kappa~ and rho~ (footnote to Eq. 21)
  midrange_device(kap, n, mm, s);
  midrange_device(drho, n, mm + 2, s);
  double h_mm[4];
  LAG_CUDA_CHECK(cudaMemcpyAsync(h_mm, mm, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
  m.mid[0] = 0.5 * (h_mm[0] + h_mm[1]);
  m.mid[1] = 0.5 * (h_mm[2] + h_mm[3]);
  // per-row extremes of kappa and rho (layered preconditioner): [kappa | rho][nz][min, max]
  m.rowmm.alloc(m.ctx, 4 * (size_t)nz * sizeof(double));
  row_minmax_device(kap, nx, nz, m.rowmm.as<double>(), s);
  row_minmax_device(drho, nx, nz, m.rowmm.as<double>() + 2 * (size_t)nz, s);
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
}

// Cylindrical (r, z) medium (Sec. 2.3, Eqs. 17-19, the equation multiplied by r), kernel layout
// rows = radius i (nr rows), row length = depth k (nzc nodes): ax holds the z faces (a2 = r_i
// kappa(face) / dz^2, zero on the surface and on the bottom face), az the r faces (a1 = rbar kappa /
// dr^2 with rbar = i dr: zero on the axis; the outer face to the ghost node takes its node's
// kappa), rh2 = r rho h^2.  c, rho: [nr][nzc].
__global__ void cylindrical_coef_kernel(const double *__restrict__ c, const double *__restrict__ rho, int nzc, int nr,
                                        double dz, double dr, double h2, double *ax, double *az, double *rh2,
                                        double *kap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // depth index (fastest)
  const int i = blockIdx.y;                             // radius index
  if (k > nzc || i > nr) return;
  auto K = [&](int ii, int kk) { const size_t o = (size_t)ii * nzc + kk; return rho[o] * c[o] * c[o]; };
  if (i < nr) {  // z face k of radius i (between depth nodes k-1 and k)
    const double ri = (i + 0.5) * dr;
    const double v = (k == 0 || k == nzc) ? 0.0 : ri * 0.5 * (K(i, k - 1) + K(i, k));
    ax[(size_t)i * (nzc + 1) + k] = v / (dz * dz);
  }
  if (k < nzc) {  // r face i of depth k (between radii i-1 and i), rbar = i dr
    const double rb = i * dr;
    const double v = (i == 0) ? 0.0 : rb * (i == nr ? K(nr - 1, k) : 0.5 * (K(i - 1, k) + K(i, k)));
    az[(size_t)i * nzc + k] = v / (dr * dr);
  }
  if (i < nr && k < nzc) {
    const size_t o = (size_t)i * nzc + k;
    rh2[o] = (i + 0.5) * dr * rho[o] * h2;
    kap[o] = K(i, k);
  }
}

void medium_build_cylindrical(lag_medium &m, const double *c_host, const double *rho_host, cudaStream_t s) {
  const int nzc = m.grid.nx, nr = m.grid.nz;  // kernel layout: rows = radii
  const size_t n = (size_t)nzc * nr;
  const size_t nax = (size_t)nr * (nzc + 1), naz = (size_t)(nr + 1) * nzc;
  m.ncoef = nax + naz + 2 * n;
  m.coef.alloc(m.ctx, m.ncoef * sizeof(double));
  m.rho_h2.alloc(m.ctx, n * sizeof(double));
  DevBuf tmp;
  tmp.alloc(m.ctx, (2 * n + 4) * sizeof(double));
  double *dc = tmp.as<double>(), *drho = dc + n, *mm = drho + n;
  LAG_CUDA_CHECK(cudaMemcpyAsync(dc, c_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(drho, rho_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  double *ax = m.coef.as<double>(), *az = ax + nax, *dg = az + naz, *kap = dg + n;
  dim3 g((nzc + 1 + 127) / 128, nr + 1);
  cylindrical_coef_kernel<<<g, 128, 0, s>>>(dc, drho, nzc, nr, m.grid.dx, m.grid.dz, m.h * m.h, ax, az,
                                            m.rho_h2.as<double>(), kap);
  count_launch();
  LAG_LAUNCH_CHECK();
  dim3 g2((nzc + 127) / 128, nr);
  acoustic_diag_kernel<<<g2, 128, 0, s>>>(ax, az, m.rho_h2.as<double>(), nzc, nr, dg);
  count_launch();
  LAG_LAUNCH_CHECK();
  // whole-medium midranges kappa~ and rho~ (footnote to Eq. 21; the r weights enter the plan)
  midrange_device(kap, n, mm, s);
  midrange_device(drho, n, mm + 2, s);
  // per-radius extremes (the radial preconditioner): [kappa | rho][nr][min, max]
  m.rowmm.alloc(m.ctx, 4 * (size_t)nr * sizeof(double));
  row_minmax_device(kap, nzc, nr, m.rowmm.as<double>(), s);
  row_minmax_device(drho, nzc, nr, m.rowmm.as<double>() + 2 * (size_t)nr, s);
  double h_mm[4];
  LAG_CUDA_CHECK(cudaMemcpyAsync(h_mm, mm, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
  m.mid[0] = 0.5 * (h_mm[0] + h_mm[1]);
  m.mid[1] = 0.5 * (h_mm[2] + h_mm[3]);
}

// ------------------------------------------------------------------------------ acoustic apply
// 32 x 8 point tiles walked grid-stride by a bounded number of blocks per rhs (the partial sums of
// (p, q) stay few, so the last block's deterministic sum is short).  mode 1: also alpha = rz / pq.
__global__ void __launch_bounds__(256) acoustic_apply_kernel(const double *__restrict__ p, double *__restrict__ q,
                                                             int nx, int nz, const double *__restrict__ ax,
                                                             const double *__restrict__ az,
                                                             const double *__restrict__ dg, KrylovScalars *sc,
                                                             Reduce red, int mode) {
  const int b = blockIdx.y;
  if (sc != nullptr && sc[b].state != ST_RUN) return;
  const int tx = (nx + 31) / 32, tz = (nz + 7) / 8;
  const size_t plane = (size_t)nx * nz;
  const double *pb = p + (size_t)b * plane;
  double *qb = q + (size_t)b * plane;
  double dot = 0.0;
  for (int t = blockIdx.x; t < tx * tz; t += gridDim.x) {
    const int i = (t % tx) * 32 + (threadIdx.x & 31);
    const int k = (t / tx) * 8 + (threadIdx.x >> 5);
    if (i < nx && k < nz) {
      const size_t o = (size_t)k * nx + i;
      const double pc = pb[o];
      const double pw = (i > 0) ? pb[o - 1] : 0.0;
      const double pe = (i + 1 < nx) ? pb[o + 1] : 0.0;
      const double pn = (k > 0) ? pb[o - nx] : 0.0;
      const double ps = (k + 1 < nz) ? pb[o + nx] : 0.0;
      const size_t fx = (size_t)k * (nx + 1) + i;
      double v = dg[o] * pc;
      v = fma(-ax[fx], pw, v);
      v = fma(-ax[fx + 1], pe, v);
      v = fma(-az[o], pn, v);
      v = fma(-az[o + nx], ps, v);
      qb[o] = v;
      dot = fma(pc, v, dot);
    }
  }
  if (mode == 1) {
    double v1[1] = {dot}, tot[1];
    __shared__ double sh[32];
    block_sum<1>(v1, sh);
    if (publish_partials<1>(red, b, blockIdx.x, gridDim.x, v1, tot)) {
      const double pq = tot[0];
      sc[b].pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) sc[b].state = ST_NAN;
      else sc[b].alpha = sc[b].rz / pq;
    }
  }
}

// The CG direction update fused with the operator (Sec. 2.3): p_new = z + beta p_old (beta of the
// right-hand side's record, 0 on its first iteration), q = A p_new and (p_new, q) -> alpha = rz / pq.
// p_new goes to a buffer of its own because neighbouring tiles still read p_old for their halos.
// 32 x 8 point tiles as above; a tile's p_new with its one-point halo is formed in shared memory
// (the same fma(beta, p_old, z) per point as a separate update would take, and the same stencil
// arithmetic in the same order), so the results equal those of the two separate passes bit for bit.
__global__ void __launch_bounds__(256) acoustic_apply_dir_kernel(const double *__restrict__ z,
                                                                 const double *__restrict__ pold,
                                                                 double *__restrict__ pnew, double *__restrict__ q,
                                                                 int nx, int nz, const double *__restrict__ ax,
                                                                 const double *__restrict__ az,
                                                                 const double *__restrict__ dg, KrylovScalars *sc,
                                                                 Reduce red) {
  const int b = blockIdx.y;
  if (sc[b].state != ST_RUN) return;
  const double beta = sc[b].beta;
  const int tx = (nx + 31) / 32, tz = (nz + 7) / 8;
  const size_t plane = (size_t)nx * nz;
  const double *zb = z + (size_t)b * plane, *pob = pold + (size_t)b * plane;
  double *pnb = pnew + (size_t)b * plane, *qb = q + (size_t)b * plane;
  __shared__ double sp[10][34];
  const int lx = threadIdx.x & 31, lz = threadIdx.x >> 5;
  double dot = 0.0;
  for (int t = blockIdx.x; t < tx * tz; t += gridDim.x) {
    const int i0 = (t % tx) * 32, k0 = (t / tx) * 8;
    __syncthreads();  // the previous tile is finished with sp
    for (int e = threadIdx.x; e < 10 * 34; e += 256) {
      const int hz = e / 34, hx = e - hz * 34;
      const int i = i0 + hx - 1, k = k0 + hz - 1;
      double v = 0.0;  // Dirichlet: p = 0 outside the grid
      if (i >= 0 && i < nx && k >= 0 && k < nz) {
        const size_t o = (size_t)k * nx + i;
        v = fma(beta, pob[o], zb[o]);
      }
      sp[hz][hx] = v;
    }
    __syncthreads();
    const int i = i0 + lx, k = k0 + lz;
    if (i < nx && k < nz) {
      const size_t o = (size_t)k * nx + i;
      const size_t fx = (size_t)k * (nx + 1) + i;
      const double pc = sp[lz + 1][lx + 1];
      double v = dg[o] * pc;
      v = fma(-ax[fx], sp[lz + 1][lx], v);
      v = fma(-ax[fx + 1], sp[lz + 1][lx + 2], v);
      v = fma(-az[o], sp[lz][lx + 1], v);
      v = fma(-az[o + nx], sp[lz + 2][lx + 1], v);
      pnb[o] = pc;
      qb[o] = v;
      dot = fma(pc, v, dot);
    }
  }
  double v1[1] = {dot}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (publish_partials<1>(red, b, blockIdx.x, gridDim.x, v1, tot)) {
    const double pq = tot[0];
    sc[b].pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) sc[b].state = ST_NAN;
    else sc[b].alpha = sc[b].rz / pq;
  }
}

int stencil_blocks_per_rhs(int nx, int nz) {
  const int tiles = ((nx + 31) / 32) * ((nz + 7) / 8);
  return tiles < 1216 ? tiles : 1216;
}

void acoustic_apply(const lag_medium &m, const double *p, double *q, int nrhs, const KrylovScalars *sc,
                    const Reduce *red, int mode, cudaStream_t s) {
  const int nx = m.grid.nx, nz = m.grid.nz;
  const size_t nax = (size_t)nz * (nx + 1), naz = (size_t)(nz + 1) * nx;
  const double *ax = m.coef.as<double>(), *az = ax + nax, *dg = az + naz;
  dim3 g(stencil_blocks_per_rhs(nx, nz), nrhs);
  Reduce r = red ? *red : Reduce{nullptr, nullptr, 0, 0};
  ProfScope prof(KC_STENCIL_A, s);
  acoustic_apply_kernel<<<g, 256, 0, s>>>(p, q, nx, nz, ax, az, dg, const_cast<KrylovScalars *>(sc), r, mode);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void acoustic_apply_dir(const lag_medium &m, const double *z, const double *pold, double *pnew, double *q, int nrhs,
                        const KrylovScalars *sc, const Reduce &red, cudaStream_t s) {
  const int nx = m.grid.nx, nz = m.grid.nz;
  const size_t nax = (size_t)nz * (nx + 1), naz = (size_t)(nz + 1) * nx;
  const double *ax = m.coef.as<double>(), *az = ax + nax, *dg = az + naz;
  dim3 g(stencil_blocks_per_rhs(nx, nz), nrhs);
  ProfScope prof(KC_STENCIL_A, s);
  acoustic_apply_dir_kernel<<<g, 256, 0, s>>>(z, pold, pnew, q, nx, nz, ax, az, dg, const_cast<KrylovScalars *>(sc),
                                              red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------ vector kernels
int reduce_blocks(size_t n) {
  const size_t b = (n + 1023) / 1024;
  return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

// r = b, x = 0, p = 0 (the first direction update takes beta = 0 and reads p), ||b||^2
__global__ void __launch_bounds__(256) pcg_start_kernel(const double *__restrict__ b, double *__restrict__ x,
                                                        double *__restrict__ r, double *__restrict__ p, size_t n,
                                                        double tol2, KrylovScalars *sc, Reduce red) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = b[off + i];
    r[off + i] = v;
    x[off + i] = 0.0;
    p[off + i] = 0.0;
    acc = fma(v, v, acc);
  }
  double v1[1] = {acc}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (publish_partials<1>(red, rhs, blockIdx.x, gridDim.x, v1, tot)) {
    KrylovScalars &S = sc[rhs];
    S.bb = tot[0];
    S.tol2 = tol2;
    S.iters = 0;
    S.rr = tot[0];
    S.alpha = S.beta = S.rz = S.pq = S.zq = 0.0;
    S.state = (tot[0] == 0.0) ? ST_CONV : (isfinite(tot[0]) ? ST_RUN : ST_NAN);
  }
}

void pcg_start(const double *b, double *x, double *r, double *p, size_t n, int nrhs, double tol, KrylovScalars *sc,
               const Reduce &red, cudaStream_t s) {
  dim3 g(reduce_blocks(n), nrhs);
  ProfScope prof(KC_VEC, s);
  pcg_start_kernel<<<g, 256, 0, s>>>(b, x, r, p, n, tol * tol, sc, red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// x += alpha p, r -= alpha q, rr = (r, r) -> convergence state
__global__ void __launch_bounds__(256) pcg_update_xr_kernel(double *__restrict__ x, double *__restrict__ r,
                                                            const double *__restrict__ p,
                                                            const double *__restrict__ q, size_t n, int max_iter,
                                                            KrylovScalars *sc, Reduce red) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const double a = sc[rhs].alpha;
  const size_t off = (size_t)rhs * n;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    x[off + i] = fma(a, p[off + i], x[off + i]);
    const double rv = fma(-a, q[off + i], r[off + i]);
    r[off + i] = rv;
    acc = fma(rv, rv, acc);
  }
  double v1[1] = {acc}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (publish_partials<1>(red, rhs, blockIdx.x, gridDim.x, v1, tot)) {
    KrylovScalars &S = sc[rhs];
    S.rr = tot[0];
    S.iters += 1;
    if (!isfinite(tot[0])) S.state = ST_NAN;
    else if (tot[0] <= S.tol2 * S.bb) S.state = ST_CONV;
    else if (S.iters >= max_iter) S.state = ST_STOP;
  }
}

void pcg_update_xr(double *x, double *r, const double *p, const double *q, size_t n, int nrhs, int max_iter,
                   KrylovScalars *sc, const Reduce &red, cudaStream_t s) {
  dim3 g(reduce_blocks(n), nrhs);
  ProfScope prof(KC_VEC, s);
  pcg_update_xr_kernel<<<g, 256, 0, s>>>(x, r, p, q, n, max_iter, sc, red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// rz_new = (r, z), zq = (z, q); beta = rz_new / rz (Fletcher-Reeves) or -alpha zq / rz (Polak-Ribiere),
// 0 on the first iteration of a solve
__global__ void __launch_bounds__(256) pcg_beta_kernel(const double *__restrict__ r, const double *__restrict__ z,
                                                       const double *__restrict__ q, size_t n, int flexible,
                                                       KrylovScalars *sc, Reduce red) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const size_t off = (size_t)rhs * n;
  double a0 = 0.0, a1 = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double zv = z[off + i];
    a0 = fma(r[off + i], zv, a0);
    if (flexible) a1 = fma(zv, q[off + i], a1);
  }
  double v2[2] = {a0, a1}, tot[2];
  __shared__ double sh[64];
  block_sum<2>(v2, sh);
  if (publish_partials<2>(red, rhs, blockIdx.x, gridDim.x, v2, tot)) {
    KrylovScalars &S = sc[rhs];
    const double rz_new = tot[0];
    S.zq = tot[1];
    // the first direction of a solve is z itself (beta = 0)
    S.beta = (S.iters == 0) ? 0.0 : (flexible ? (-S.alpha * tot[1] / S.rz) : (rz_new / S.rz));
    S.rz = rz_new;
    if (!isfinite(S.beta) || !isfinite(rz_new) || !isfinite(tot[1])) S.state = ST_NAN;
  }
}

// the same for (r, z) alone (Fletcher-Reeves) with n even: 16-byte pairs (every right-hand side's
// row then starts on a 16-byte boundary), two pairs in flight per thread, and few enough registers
// that the whole grid is resident at once (the sweep is one round of loads, latency-bound)
__global__ void __launch_bounds__(256, 8) pcg_rz_beta_kernel(const double *__restrict__ r, const double *__restrict__ z,
                                                             size_t n, KrylovScalars *sc, Reduce red) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const double2 *r2 = reinterpret_cast<const double2 *>(r + (size_t)rhs * n);
  const double2 *z2 = reinterpret_cast<const double2 *>(z + (size_t)rhs * n);
  const size_t n2 = n / 2, stride = (size_t)gridDim.x * blockDim.x;
  double a0 = 0.0, a1 = 0.0;
#pragma unroll 1
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += 2 * stride) {
    const double2 ra = __ldg(r2 + i), za = __ldg(z2 + i);
    double2 rb = make_double2(0.0, 0.0), zb = rb;
    if (i + stride < n2) {
      rb = __ldg(r2 + i + stride);
      zb = __ldg(z2 + i + stride);
    }
    a0 = fma(ra.x, za.x, a0);
    a1 = fma(ra.y, za.y, a1);
    a0 = fma(rb.x, zb.x, a0);
    a1 = fma(rb.y, zb.y, a1);
  }
  double v1[1] = {a0 + a1}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (publish_partials<1>(red, rhs, blockIdx.x, gridDim.x, v1, tot)) {
    KrylovScalars &S = sc[rhs];
    const double rz_new = tot[0];
    S.zq = 0.0;
    S.beta = (S.iters == 0) ? 0.0 : rz_new / S.rz;
    S.rz = rz_new;
    if (!isfinite(S.beta) || !isfinite(rz_new)) S.state = ST_NAN;
  }
}

void pcg_beta(const double *r, const double *z, const double *q, size_t n, int nrhs, int flexible,
              KrylovScalars *sc, const Reduce &red, cudaStream_t s) {
  dim3 g(reduce_blocks(n), nrhs);
  ProfScope prof(KC_VEC, s);
  if (!flexible && (n & 1) == 0) pcg_rz_beta_kernel<<<g, 256, 0, s>>>(r, z, n, sc, red);
  else pcg_beta_kernel<<<g, 256, 0, s>>>(r, z, q, n, flexible, sc, red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------ Laguerre series
// Right-hand side of harmonic m (Eq. 9 in SPD form), per rhs b and component c:
//   r = -c_m rho h^2 S + (f_m / (dx dz)) at the source node of component src_comp;  x = 0.
__global__ void __launch_bounds__(256) laguerre_rhs_kernel(const double *__restrict__ rh2, const double *__restrict__ S,
                                                           double cm, const double *__restrict__ fm, int m,
                                                           const int *__restrict__ src_idx,
                                                           int src_comp, double inv_cell, int ncomp, size_t nplane,
                                                           double *__restrict__ r, double *__restrict__ x,
                                                           double *__restrict__ p, double tol2, KrylovScalars *sc,
                                                           Reduce red) {
  const int rhs = blockIdx.y;
  const size_t n = nplane * ncomp;
  const size_t off = (size_t)rhs * n;
  const size_t sidx = (size_t)src_comp * nplane + (size_t)src_idx[rhs];
  const double fmv = fm[m];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t node = i % nplane;
    double v = -cm * rh2[node] * S[off + i];
    if (i == sidx) v += fmv * inv_cell;
    r[off + i] = v;
    x[off + i] = 0.0;
    if (p != nullptr) p[off + i] = 0.0;
    acc = fma(v, v, acc);
  }
  double v1[1] = {acc}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (publish_partials<1>(red, rhs, blockIdx.x, gridDim.x, v1, tot)) {
    KrylovScalars &K = sc[rhs];
    K.bb = tot[0];
    K.rr = tot[0];
    K.tol2 = tol2;
    K.iters = 0;
    K.alpha = K.beta = K.rz = K.pq = K.zq = 0.0;
    K.state = (tot[0] == 0.0) ? ST_CONV : (isfinite(tot[0]) ? ST_RUN : ST_NAN);
  }
}

void laguerre_rhs(const double *rho_h2, const double *S, double cm, const double *fm, int m, const int *src_idx,
                  int src_comp, double inv_cell, int ncomp, size_t nplane, int nrhs, double *r, double *x,
                  double *p, double tol, KrylovScalars *sc, const Reduce &red, cudaStream_t s) {
  dim3 g(reduce_blocks(nplane * ncomp), nrhs);
  ProfScope prof(KC_LAGUERRE, s);
  laguerre_rhs_kernel<<<g, 256, 0, s>>>(rho_h2, S, cm, fm, m, src_idx, src_comp, inv_cell, ncomp, nplane, r, x, p,
                                        tol * tol, sc, red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// T += c^_m R_m ; S += T   (S_{m+1} = sum_{k<=m} (m+1-k) c^_k R_k)
__global__ void __launch_bounds__(256) laguerre_acc_kernel(const double *__restrict__ x, double *__restrict__ T,
                                                           double *__restrict__ S, double chat, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double t = fma(chat, x[i], T[i]);
    T[i] = t;
    S[i] += t;
  }
}

void laguerre_accumulate(const double *x, double *T, double *S, double chat, size_t n, int nrhs, cudaStream_t s) {
  const size_t tot = n * (size_t)nrhs;
  ProfScope prof(KC_LAGUERRE, s);
  laguerre_acc_kernel<<<reduce_blocks(tot), 256, 0, s>>>(x, T, S, chat, tot);
  count_launch();
  LAG_LAUNCH_CHECK();
}

__global__ void gather_kernel(const double *__restrict__ x, const int *__restrict__ idx, int nrcv, int ncomp,
                              size_t nplane, int nrhs, double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = nrhs * ncomp * nrcv;
  if (t >= total) return;
  const int r = t % nrcv, c = (t / nrcv) % ncomp, b = t / (nrcv * ncomp);
  out[t] = x[((size_t)b * ncomp + c) * nplane + (size_t)idx[r]];
}

void gather_receivers(const double *x, const int *rcv_idx, int nrcv, int ncomp, size_t nplane, int nrhs,
                      double *out, cudaStream_t s) {
  const int total = nrhs * ncomp * nrcv;
  if (total <= 0) return;
  ProfScope prof(KC_LAGUERRE, s);
  gather_kernel<<<(total + 255) / 256, 256, 0, s>>>(x, rcv_idx, nrcv, ncomp, nplane, nrhs, out);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// traces[row][t] = sum_m rrcv[m][row] tab[m][t]   (Eq. 8)
__global__ void inverse_sum_kernel(const double *__restrict__ rrcv, const double *__restrict__ tab, int nharm,
                                   int nrows, int nt, double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (t >= nt) return;
  double acc = 0.0;
  for (int m = 0; m < nharm; ++m) acc = fma(rrcv[(size_t)m * nrows + row], tab[(size_t)m * nt + t], acc);
  out[(size_t)row * nt + t] = acc;
}

void inverse_sum(const double *rrcv, const double *tab, int nharm, int nrows, int nt, double *traces,
                 cudaStream_t s) {
  if (nrows <= 0 || nt <= 0) return;
  dim3 g((nt + 127) / 128, nrows);
  inverse_sum_kernel<<<g, 128, 0, s>>>(rrcv, tab, nharm, nrows, nt, traces);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------ Laguerre functions
// Normalised functions ell_m(x) = sqrt(m!/(m+alpha)!) x^{alpha/2} e^{-x/2} L_m^alpha(x) by the
// three-term recurrence of L_m^alpha (renormalised), carried as mantissa * exp(log-scale) and
// rescaled by 2^-500 whenever the mantissa grows past 2^500 (e^{-x/2} underflows for x > ~1400).
struct EllRec {
  double prev, cur, logs;
  double alpha, x;
  int m;
  __device__ void start(double x_, double alpha_, double log_extra) {
    x = x_;
    alpha = alpha_;
    m = 0;
    prev = 0.0;
    cur = 1.0;
    logs = -0.5 * x - 0.5 * lgamma(alpha + 1.0) + log_extra;
  }
  __device__ double value() const {
    if (cur == 0.0) return 0.0;
    const double mag = exp(log(fabs(cur)) + logs);
    return cur < 0.0 ? -mag : mag;
  }
  __device__ void next() {
    const double md = (double)m;
    const double nx = ((2.0 * md + alpha + 1.0 - x) * cur - sqrt(md * (md + alpha)) * prev) /
                      sqrt((md + 1.0) * (md + alpha + 1.0));
    prev = cur;
    cur = nx;
    ++m;
    if (fabs(cur) > 0x1p500) {
      cur *= 0x1p-500;
      prev *= 0x1p-500;
      logs += 500.0 * 0.69314718055994530942;
    }
  }
};

// f_m partial sums: one thread per Gauss-Legendre node, warp sums written per (warp, m).
struct WaveletDev {
  double f0, t0, gamma;
  int kind;
  __device__ double operator()(double t) const {
    if (kind == LAG_WAVELET_PAPER) {
      const double s = 2.0 * 3.14159265358979323846 * f0 * (t - t0);
      return exp(-(s * s) / (gamma * gamma)) * sin(s);
    }
    const double a = 3.14159265358979323846 * f0 * (t - t0);
    const double a2 = a * a;
    return (1.0 - 2.0 * a2) * exp(-a2);
  }
};

__constant__ double c_gl_x[16];
__constant__ double c_gl_w[16];

__global__ void source_coeff_kernel(WaveletDev wv, double h, double alpha, int n, double t_end, int panels,
                                    double *wpart /* [nwarps_total][n] */) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nodes = panels * 16;
  double t = 0.0, wq = 0.0;
  if (q < nodes) {
    const int pnl = q >> 4, g = q & 15;
    const double a = t_end * (double)pnl / panels, b = t_end * (double)(pnl + 1) / panels;
    t = 0.5 * (b - a) * c_gl_x[g] + 0.5 * (a + b);
    wq = 0.5 * (b - a) * c_gl_w[g];
  }
  const double weight = (q < nodes) ? wq * wv(t) * sqrt(h) : 0.0;
  EllRec e;
  // (ht)^{-alpha/2} ell_m(ht): the start leaves the x^{alpha/2} factor of ell_0 out already
  e.start(h * t, alpha, 0.0);
  const int gw = q >> 5, lane = threadIdx.x & 31;
  for (int m = 0; m < n; ++m) {
    double v = (q < nodes) ? weight * e.value() : 0.0;
    v = warp_sum(v);
    if (lane == 0) wpart[(size_t)gw * n + m] = v;
    e.next();
  }
}

__global__ void sum_columns_kernel(const double *wpart, int nrows, int n, double *out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double acc = 0.0;
  for (int r = 0; r < nrows; ++r) acc += wpart[(size_t)r * n + m];
  out[m] = acc;
}

// 16-point Gauss-Legendre nodes by Newton's iteration on P_16 (host, once)
static void gauss_legendre16(double *x, double *w) {
  const int N = 16;
  for (int i = 0; i < N; ++i) {
    double z = cos(3.14159265358979323846 * (i + 0.75) / (N + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= N; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = N * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (fabs(z - z1) < 1e-16) break;
    }
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

void source_coeffs_device(const lag_laguerre &lag, const lag_wavelet &w, double *fm_dev, DevBuf &scratch,
                          lag_ctx *ctx, cudaStream_t s) {
  static PerDeviceOnce gl_done;  // constant memory belongs to each device
  gl_done.run([] {
    double x[16], wt[16];
    gauss_legendre16(x, wt);
    LAG_CUDA_CHECK(cudaMemcpyToSymbol(c_gl_x, x, sizeof(x)));
    LAG_CUDA_CHECK(cudaMemcpyToSymbol(c_gl_w, wt, sizeof(wt)));
  });
  const int n = lag.n_harm;
  const double t_end = (w.kind == LAG_WAVELET_PAPER) ? w.t0 + 2.0 * w.gamma / w.f0 : w.t0 + 4.0 / w.f0;
  int panels = 4 * n + (int)(8.0 * lag.h * t_end / 16.0) + 64;
  if (panels < 64) panels = 64;
  const int nodes = panels * 16;
  const int blocks = (nodes + 255) / 256;
  const int nwarps = blocks * 8;
  scratch.alloc(ctx, (size_t)nwarps * n * sizeof(double));
  WaveletDev wv{w.f0, w.t0, w.gamma, w.kind};
  source_coeff_kernel<<<blocks, 256, 0, s>>>(wv, lag.h, (double)lag.alpha, n, t_end, panels, scratch.as<double>());
  count_launch();
  LAG_LAUNCH_CHECK();
  sum_columns_kernel<<<(n + 127) / 128, 128, 0, s>>>(scratch.as<double>(), nwarps, n, fm_dev);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// tab[m][j] = (h t_j)^{alpha/2} sqrt(h) ell_m(h t_j)
__global__ void laguerre_table_kernel(const double *t, int nt, double h, double alpha, int n, double *tab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const double x = h * t[j];
  if (!(x > 0.0)) {
    for (int m = 0; m < n; ++m) tab[(size_t)m * nt + j] = 0.0;
    return;
  }
  EllRec e;
  e.start(x, alpha, alpha * log(x) + 0.5 * log(h));  // x^{alpha/2} of ell_0 and (ht)^{alpha/2} sqrt(h)
  for (int m = 0; m < n; ++m) {
    tab[(size_t)m * nt + j] = e.value();
    e.next();
  }
}

void laguerre_table_device(const lag_laguerre &lag, int nt, const double *t_dev, double *tab_dev, cudaStream_t s) {
  if (nt <= 0) return;
  laguerre_table_kernel<<<(nt + 127) / 128, 128, 0, s>>>(t_dev, nt, lag.h, (double)lag.alpha, lag.n_harm, tab_dev);
  count_launch();
  LAG_LAUNCH_CHECK();
}

}  // namespace lag
