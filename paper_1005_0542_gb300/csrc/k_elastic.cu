// Elastic operator C (Sec. 2.2 Eq. 12, Sec. 2.3 Eq. 19) and the flexible GMRES(k) kernels.
//
// Cartesian plane-strain form of Eq. (12), Dirichlet frame, SPD sign (C = -(elastic terms) + rho h^2/4):
//   (C[u;w])_u = du u - pxE u_e - pxW u_w - mzS u_s - mzN u_n - [Dx(l Dz w) + Dz(m Dx w)]
//   (C[u;w])_w = dw w - mxE w_e - mxW w_w - pzS w_s - pzN w_n - [Dx(m Dz u) + Dz(l Dx u)]
// px/pz: (lambda + 2 mu) on x/z faces over dx^2/dz^2, mx/mz: mu on faces (face = mean of the two
// nodes, boundary face = node), du/dw the matching diagonals plus rho h^2/4; the mixed terms are
// centred differences with nodal coefficients l4 = lambda/(4 dx dz), m4 = mu/(4 dx dz):
//   Dx(l Dz w) = l4[k][i+1](w[k+1][i+1] - w[k-1][i+1]) - l4[k][i-1](w[k+1][i-1] - w[k-1][i-1])
//   Dz(m Dx w) = m4[k+1][i](w[k+1][i+1] - w[k+1][i-1]) - m4[k-1][i](w[k-1][i+1] - w[k-1][i-1])
// (and the same with u, l <-> m swapped in the second row), which makes C symmetric.
#include "internal.h"

namespace lag {

// coef layout: px [nz][nx+1] | mx [nz][nx+1] | pz [nz+1][nx] | mz [nz+1][nx] | l4 | m4 | du | dw  ([nz][nx] each)
struct ElasticCoef {
  const double *px, *mx, *pz, *mz, *l4, *m4, *du, *dw;
};

static ElasticCoef elastic_coef(const lag_medium &m) {
  const int nx = m.grid.nx, nz = m.grid.nz;
  const size_t nxf = (size_t)nz * (nx + 1), nzf = (size_t)(nz + 1) * nx, n = (size_t)nx * nz;
  const double *b = m.coef.as<double>();
  ElasticCoef c;
  c.px = b;
  c.mx = c.px + nxf;
  c.pz = c.mx + nxf;
  c.mz = c.pz + nzf;
  c.l4 = c.mz + nzf;
  c.m4 = c.l4 + n;
  c.du = c.m4 + n;
  c.dw = c.du + n;
  return c;
}

__global__ void elastic_nodal_kernel(const double *vp, const double *vs, const double *rho, size_t n, double *lam,
                                     double *mu, double *p2m, double *rh2, double h2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double r = rho[i], a = vp[i], b = vs[i];
    const double l = r * (a * a - 2.0 * b * b), m = r * b * b;
    lam[i] = l;
    mu[i] = m;
    p2m[i] = l + 2.0 * m;
    rh2[i] = r * h2;
  }
}

__global__ void elastic_coef_kernel(const double *lam, const double *mu, int nx, int nz, double idx2, double idz2,
                                    double i4, double *px, double *mx, double *pz, double *mz, double *l4,
                                    double *m4) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i > nx || k > nz) return;
  auto P = [&](int kk, int ii) { const size_t o = (size_t)kk * nx + ii; return lam[o] + 2.0 * mu[o]; };
  auto M = [&](int kk, int ii) { return mu[(size_t)kk * nx + ii]; };
  if (k < nz) {
    const size_t f = (size_t)k * (nx + 1) + i;
    const double vp = (i == 0) ? P(k, 0) : (i == nx ? P(k, nx - 1) : 0.5 * (P(k, i - 1) + P(k, i)));
    const double vm = (i == 0) ? M(k, 0) : (i == nx ? M(k, nx - 1) : 0.5 * (M(k, i - 1) + M(k, i)));
    px[f] = vp * idx2;
    mx[f] = vm * idx2;
  }
  if (i < nx) {
    const size_t f = (size_t)k * nx + i;
    const double vp = (k == 0) ? P(0, i) : (k == nz ? P(nz - 1, i) : 0.5 * (P(k - 1, i) + P(k, i)));
    const double vm = (k == 0) ? M(0, i) : (k == nz ? M(nz - 1, i) : 0.5 * (M(k - 1, i) + M(k, i)));
    pz[f] = vp * idz2;
    mz[f] = vm * idz2;
  }
  if (i < nx && k < nz) {
    const size_t o = (size_t)k * nx + i;
    l4[o] = lam[o] * i4;
    m4[o] = mu[o] * i4;
  }
}

__global__ void elastic_diag_kernel(const double *px, const double *mx, const double *pz, const double *mz,
                                    const double *rh2, int nx, int nz, double *du, double *dw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= nx || k >= nz) return;
  const size_t o = (size_t)k * nx + i, fx = (size_t)k * (nx + 1) + i, fz = (size_t)k * nx + i;
  const double w = 0.25 * rh2[o];
  du[o] = px[fx] + px[fx + 1] + mz[fz] + mz[fz + nx] + w;
  dw[o] = mx[fx] + mx[fx + 1] + pz[fz] + pz[fz + nx] + w;
}

void medium_build_elastic(lag_medium &m, const double *vp_host, const double *vs_host, const double *rho_host,
                          cudaStream_t s) {
  const int nx = m.grid.nx, nz = m.grid.nz;
  const size_t n = (size_t)nx * nz;
  const size_t nxf = (size_t)nz * (nx + 1), nzf = (size_t)(nz + 1) * nx;
  m.ncoef = 2 * nxf + 2 * nzf + 4 * n;
  m.coef.alloc(m.ctx, m.ncoef * sizeof(double));
  m.rho_h2.alloc(m.ctx, n * sizeof(double));
  DevBuf tmp;
  tmp.alloc(m.ctx, (6 * n + 8) * sizeof(double));
  double *dvp = tmp.as<double>(), *dvs = dvp + n, *drho = dvs + n, *lam = drho + n, *mu = lam + n, *p2m = mu + n;
  double *mm = p2m + n;
  LAG_CUDA_CHECK(cudaMemcpyAsync(dvp, vp_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(dvs, vs_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(drho, rho_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  elastic_nodal_kernel<<<reduce_blocks(n), 256, 0, s>>>(dvp, dvs, drho, n, lam, mu, p2m, m.rho_h2.as<double>(),
                                                        m.h * m.h);
  count_launch();
  LAG_LAUNCH_CHECK();
  ElasticCoef c = elastic_coef(m);
  dim3 g((nx + 1 + 127) / 128, nz + 1);
  elastic_coef_kernel<<<g, 128, 0, s>>>(lam, mu, nx, nz, 1.0 / (m.grid.dx * m.grid.dx), 1.0 / (m.grid.dz * m.grid.dz),
                                        1.0 / (4.0 * m.grid.dx * m.grid.dz), const_cast<double *>(c.px),
                                        const_cast<double *>(c.mx), const_cast<double *>(c.pz),
                                        const_cast<double *>(c.mz), const_cast<double *>(c.l4),
                                        const_cast<double *>(c.m4));
  count_launch();
  LAG_LAUNCH_CHECK();
  dim3 g2((nx + 127) / 128, nz);
  elastic_diag_kernel<<<g2, 128, 0, s>>>(c.px, c.mx, c.pz, c.mz, m.rho_h2.as<double>(), nx, nz,
                                         const_cast<double *>(c.du), const_cast<double *>(c.dw));
  count_launch();
  LAG_LAUNCH_CHECK();
  midrange_device(p2m, n, mm, s);
  midrange_device(mu, n, mm + 2, s);
  midrange_device(drho, n, mm + 4, s);
  // per-row extremes (layered K): [lambda+2mu | mu | rho][nz][min, max]
  m.rowmm.alloc(m.ctx, 6 * (size_t)nz * sizeof(double));
  row_minmax_device(p2m, nx, nz, m.rowmm.as<double>(), s);
  row_minmax_device(mu, nx, nz, m.rowmm.as<double>() + 2 * (size_t)nz, s);
  row_minmax_device(drho, nx, nz, m.rowmm.as<double>() + 4 * (size_t)nz, s);
  double h_mm[6];
  LAG_CUDA_CHECK(cudaMemcpyAsync(h_mm, mm, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
  m.mid[0] = 0.5 * (h_mm[0] + h_mm[1]);
  m.mid[1] = 0.5 * (h_mm[2] + h_mm[3]);
  m.mid[2] = 0.5 * (h_mm[4] + h_mm[5]);
}

// mode 0: every rhs (or those running when sc is given); mode 2: rhs running or ST_MET
__global__ void __launch_bounds__(256) elastic_apply_kernel(const double *__restrict__ U, double *__restrict__ Q,
                                                            int nx, int nz, ElasticCoef c,
                                                            const KrylovScalars *__restrict__ sc, int mode,
                                                            const double *__restrict__ sub) {
  const int b = blockIdx.z;
  if (sc != nullptr) {
    const int st = sc[b].state;
    if (!(st == ST_RUN || (mode == 2 && st == ST_MET))) return;
  }
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int k = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (i >= nx || k >= nz) return;
  const size_t plane = (size_t)nx * nz;
  const double *u = U + (size_t)b * 2 * plane, *w = u + plane;
  double *qu = Q + (size_t)b * 2 * plane, *qw = qu + plane;
  const size_t o = (size_t)k * nx + i;
  const bool hw = i > 0, he = i + 1 < nx, hn = k > 0, hs = k + 1 < nz;
  auto F = [&](const double *f, int dk, int di) -> double {
    const int kk = k + dk, ii = i + di;
    return (kk >= 0 && kk < nz && ii >= 0 && ii < nx) ? f[(size_t)kk * nx + ii] : 0.0;
  };
  const size_t fx = (size_t)k * (nx + 1) + i;
  // u-equation
  const double uc = u[o], ue = he ? u[o + 1] : 0.0, uw = hw ? u[o - 1] : 0.0;
  const double un = hn ? u[o - nx] : 0.0, us = hs ? u[o + nx] : 0.0;
  const double wc = w[o], we = he ? w[o + 1] : 0.0, ww = hw ? w[o - 1] : 0.0;
  const double wn = hn ? w[o - nx] : 0.0, ws = hs ? w[o + nx] : 0.0;
  const double upp = F(u, 1, 1), upm = F(u, 1, -1), ump = F(u, -1, 1), umm = F(u, -1, -1);
  const double wpp = F(w, 1, 1), wpm = F(w, 1, -1), wmp = F(w, -1, 1), wmm = F(w, -1, -1);
  const double l4e = he ? c.l4[o + 1] : 0.0, l4w = hw ? c.l4[o - 1] : 0.0;
  const double l4s = hs ? c.l4[o + nx] : 0.0, l4n = hn ? c.l4[o - nx] : 0.0;
  const double m4e = he ? c.m4[o + 1] : 0.0, m4w = hw ? c.m4[o - 1] : 0.0;
  const double m4s = hs ? c.m4[o + nx] : 0.0, m4n = hn ? c.m4[o - nx] : 0.0;
  double vu = c.du[o] * uc;
  vu = fma(-c.px[fx + 1], ue, vu);
  vu = fma(-c.px[fx], uw, vu);
  vu = fma(-c.mz[o + nx], us, vu);
  vu = fma(-c.mz[o], un, vu);
  const double mixu = l4e * (wpp - wmp) - l4w * (wpm - wmm) + m4s * (wpp - wpm) - m4n * (wmp - wmm);
  const double *su = sub ? sub + (size_t)b * 2 * plane : nullptr;
  qu[o] = su ? (vu - mixu) - su[o] : vu - mixu;
  double vw = c.dw[o] * wc;
  vw = fma(-c.mx[fx + 1], we, vw);
  vw = fma(-c.mx[fx], ww, vw);
  vw = fma(-c.pz[o + nx], ws, vw);
  vw = fma(-c.pz[o], wn, vw);
  const double mixw = m4e * (upp - ump) - m4w * (upm - umm) + l4s * (upp - upm) - l4n * (ump - umm);
  qw[o] = su ? (vw - mixw) - su[plane + o] : vw - mixw;
}

void elastic_apply(const lag_medium &m, const double *p, double *q, int nrhs, const KrylovScalars *sc,
                   const Reduce *, int mode, cudaStream_t s, const double *sub) {
  if (m.grid.cylindrical) {
    elastic_cyl_apply(m, p, q, nrhs, sc, mode, s, sub);
    return;
  }
  dim3 g((m.grid.nx + 31) / 32, (m.grid.nz + 7) / 8, nrhs);
  ProfScope prof(KC_STENCIL_E, s);
  elastic_apply_kernel<<<g, 256, 0, s>>>(p, q, m.grid.nx, m.grid.nz, elastic_coef(m), sc, mode, sub);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------ FGMRES kernels
// start of a cycle: r = b - Cx (first: r = b), beta = ||r||, g = beta e_1, state from the true residual
__global__ void __launch_bounds__(256) gm_start_kernel(const double *__restrict__ b, double *__restrict__ w,
                                                       size_t n, int first, double tol2, int max_iter,
                                                       KrylovScalars *sc, GmresDev g, Reduce red) {
  const int rhs = blockIdx.y;
  KrylovScalars &S = sc[rhs];
  if (!first && !(S.state == ST_RUN || S.state == ST_MET)) return;
  const size_t off = (size_t)rhs * n;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = first ? b[off + i] : b[off + i] - w[off + i];
    w[off + i] = v;
    acc = fma(v, v, acc);
  }
  double v1[1] = {acc}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (publish_partials<1>(red, rhs, blockIdx.x, gridDim.x, v1, tot)) {
    const int k = g.k;
    if (first) {
      S.bb = tot[0];
      S.tol2 = tol2;
      S.iters = 0;
      S.alpha = S.beta = S.rz = S.pq = S.zq = 0.0;
    }
    S.rr = tot[0];
    S.jdone = 0;
    if (!isfinite(tot[0])) S.state = ST_NAN;
    else if (tot[0] <= S.tol2 * S.bb) S.state = ST_CONV;
    else if (!first && S.iters >= max_iter) S.state = ST_STOP;
    else S.state = ST_RUN;
    double *gg = g.g + (size_t)rhs * (k + 1);
    gg[0] = sqrt(tot[0]);
    for (int i = 1; i <= k; ++i) gg[i] = 0.0;
  }
}

// v = w / ||w|| for running systems (norm taken from g[0] at a cycle start or from H at a step)
__global__ void gm_scale_kernel(const double *__restrict__ w, double *__restrict__ v, size_t n,
                                const KrylovScalars *sc, const double *__restrict__ nrm, int nstride) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const double s = nrm[(size_t)rhs * nstride];
  if (!(s > 0.0)) return;
  const double inv = 1.0 / s;
  const size_t off = (size_t)rhs * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[off + i] = w[off + i] * inv;
}

void gm_start(const double *b, const double *cx, double *v0, size_t n, int nrhs, int first, double tol,
              int max_iter, KrylovScalars *sc, GmresDev &g, const Reduce &red, cudaStream_t s) {
  ProfScope prof(KC_GMRES, s);
  dim3 grid(reduce_blocks(n), nrhs);
  gm_start_kernel<<<grid, 256, 0, s>>>(b, const_cast<double *>(cx), n, first, tol * tol, max_iter, sc, g, red);
  count_launch();
  LAG_LAUNCH_CHECK();
  gm_scale_kernel<<<grid, 256, 0, s>>>(cx, v0, n, sc, g.g, g.k + 1);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// Warp sum of eight per-thread values, scattered: lane l ends with the warp total of value l >> 2
// (recursive halving: each butterfly step keeps half of the values and adds the partner's copy of
// them, 4 + 2 + 1 + 1 + 1 = 9 FP64 adds instead of 40 for eight full butterflies; the FP64 pipe,
// not HBM, bounds the Gram-Schmidt kernels on this part).  Fixed order: deterministic.
__device__ __forceinline__ double warp_sum8_scatter(const double (&a)[8]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  double h4[4], h2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double keep = b4 ? a[4 + i] : a[i], send = b4 ? a[i] : a[4 + i];
    h4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double keep = b3 ? h4[2 + i] : h4[i], send = b3 ? h4[i] : h4[2 + i];
    h2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  double h1 = (b2 ? h2[1] : h2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? h2[0] : h2[1], 4);
  h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
  h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
  return h1;
}

// acc[q] += (w, V_q) over this thread's elements for q < C (and aw += (w, w) when W)
template <int C, int W>
__device__ __forceinline__ void gm_dots_sweep(const double *__restrict__ w, const double *__restrict__ V,
                                              size_t vstride, size_t n, double (&acc)[8], double &aw) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = fma(we, V[(size_t)q * vstride + e], acc[q]);
    if (W) aw = fma(we, we, aw);
  }
}

// blocks per rhs of the Gram-Schmidt dot kernel: four per SM, so that each thread sums many
// elements before the (FP64) block reduction
static int dots_blocks(size_t n) { return std::min(reduce_blocks(n), 4 * 152); }

// h_i = (w, V_i), i <= j: partials per block, the last block finishes all j+1 sums.
// Pass 0 also sums (w, w) and decides whether the second pass runs (selective reorthogonalisation,
// the criterion of Daniel, Gragg, Kaufman and Stewart, 1976, with eta = 1/sqrt(2)): the projected
// norm ||w - V h||^2 = (w, w) - sum h_i^2 (V orthonormal); when more than half of (w, w) remains,
// little cancellation took place, the estimate is accurate and one pass leaves w orthogonal to
// working precision; otherwise (or for a non-finite estimate) the second pass runs as in CGS2.
// shifted: w = C Z_j - V_j, so the Hessenberg entry h_jj is the dot plus one.
__global__ void __launch_bounds__(256) gm_dots_kernel(const double *__restrict__ w, const double *__restrict__ V,
                                                      int j, size_t n, size_t vstride, KrylovScalars *sc,
                                                      GmresDev g, Reduce red, int pass, int shifted) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  if (pass == 1 && sc[rhs].reorth == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // 8 warps
  const size_t off = (size_t)rhs * n;
  __shared__ double sh[9 * 8];
  __shared__ double tot[72];
  __shared__ bool is_last;
  double *part = red.part + (size_t)rhs * red.rstride;
  // eight basis vectors per sweep: w is read once per eight dots instead of once per dot (w does
  // not stay in L2 across a batch of right-hand sides); each dot keeps its own summation order.
  // The first sweep of pass 0 also sums (w, w), stored as value j + 1.
  for (int i0 = 0; i0 <= j; i0 += 8) {
    const int cnt = min(8, j + 1 - i0);
    const bool ww = pass == 0 && i0 == 0;
    double acc[8], aw = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    // one instantiation per basis count and (w, w) flag: predicated-off FMAs would still take
    // FP64 issue slots, the limit of this kernel
    const double *Vi = V + (size_t)i0 * vstride + off;
    const double *wp = w + off;
    switch (cnt * 2 + (ww ? 1 : 0)) {
#define LAG_GM_SWEEP(C, W) \
      case C * 2 + W: gm_dots_sweep<C, W>(wp, Vi, vstride, n, acc, aw); break;
      LAG_GM_SWEEP(1, 0) LAG_GM_SWEEP(1, 1) LAG_GM_SWEEP(2, 0) LAG_GM_SWEEP(2, 1)
      LAG_GM_SWEEP(3, 0) LAG_GM_SWEEP(3, 1) LAG_GM_SWEEP(4, 0) LAG_GM_SWEEP(4, 1)
      LAG_GM_SWEEP(5, 0) LAG_GM_SWEEP(5, 1) LAG_GM_SWEEP(6, 0) LAG_GM_SWEEP(6, 1)
      LAG_GM_SWEEP(7, 0) LAG_GM_SWEEP(7, 1) LAG_GM_SWEEP(8, 0) LAG_GM_SWEEP(8, 1)
#undef LAG_GM_SWEEP
      default: break;
    }
    const double sv = warp_sum8_scatter(acc);
    if ((lane & 3) == 0) sh[(lane >> 2) * 8 + warp] = sv;
    if (ww) {
      aw = warp_sum(aw);
      if (lane == 0) sh[64 + warp] = aw;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
      const int q = threadIdx.x;
      if (q < cnt || (q == 8 && ww)) {
        double t = 0.0;
        for (int u = 0; u < 8; ++u) t += sh[q * 8 + u];
        part[(size_t)(q < 8 ? i0 + q : j + 1) * red.nblk + blockIdx.x] = t;
      }
    }
    __syncthreads();  // sh is reused by the next sweep
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(red.count + rhs, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // the last block: warp v sums value v (then v + 8, ...) over the blocks, lanes strided
  const int nsum = pass == 0 ? j + 2 : j + 1;
  for (int v = warp; v < nsum; v += 8) {
    double a = 0.0;
    for (int bb = lane; bb < (int)gridDim.x; bb += 32) a += __ldcg(part + (size_t)v * red.nblk + bb);
    a = warp_sum(a);
    if (lane == 0) tot[v] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int k = g.k;
    double *hc = g.hcol + (size_t)rhs * (k + 1);
    double *tmp = g.y + (size_t)rhs * k;  // this pass's coefficients
    double hsum = 0.0;
    for (int i = 0; i <= j; ++i) {
      const double h = tot[i];
      tmp[i] = h;
      hc[i] = pass == 0 ? (shifted && i == j ? h + 1.0 : h) : hc[i] + h;
      hsum = fma(h, h, hsum);
    }
    if (pass == 0) {
      const double wnorm2 = tot[j + 1], rest = wnorm2 - hsum;
      sc[rhs].reorth = (rest > 0.5 * wnorm2 && isfinite(rest)) ? 0 : 1;
    }
    red.count[rhs] = 0u;
  }
}

// w -= sum_i tmp_i V_i
__global__ void __launch_bounds__(256) gm_axpy_kernel(double *__restrict__ w, const double *__restrict__ V, int j,
                                                      size_t n, size_t vstride, const KrylovScalars *sc, GmresDev g,
                                                      int pass) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  if (pass == 1 && sc[rhs].reorth == 0) return;
  const size_t off = (size_t)rhs * n;
  const double *tmp = g.y + (size_t)rhs * g.k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = w[off + e];
    for (int i = 0; i <= j; ++i) v = fma(-tmp[i], V[(size_t)i * vstride + off + e], v);
    w[off + e] = v;
  }
}

void gm_orthogonalize(double *w, const double *V, int j, size_t n, int nrhs, size_t vstride, KrylovScalars *sc,
                      GmresDev &g, const Reduce &red, int pass, bool shifted, cudaStream_t s) {
  ProfScope prof(KC_GMRES, s);
  if (j + 2 > 72) throw Error(LAG_EINVAL, "GMRES restart length above 70");
  dim3 gd(dots_blocks(n), nrhs), grid(reduce_blocks(n), nrhs);
  gm_dots_kernel<<<gd, 256, 0, s>>>(w, V, j, n, vstride, sc, g, red, pass, shifted ? 1 : 0);
  count_launch();
  LAG_LAUNCH_CHECK();
  gm_axpy_kernel<<<grid, 256, 0, s>>>(w, V, j, n, vstride, sc, g, pass);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// h_{j+1,j} = ||w||; Givens rotations on column j; g update; residual estimate -> state
__global__ void __launch_bounds__(256) gm_norm_kernel(const double *__restrict__ w, int j, size_t n,
                                                      KrylovScalars *sc, GmresDev g, Reduce red, int max_iter) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const size_t off = (size_t)rhs * n;
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    acc = fma(w[off + e], w[off + e], acc);
  double v1[1] = {acc}, tot[1];
  __shared__ double sh[32];
  block_sum<1>(v1, sh);
  if (!publish_partials<1>(red, rhs, blockIdx.x, gridDim.x, v1, tot)) return;
  const int k = g.k;
  KrylovScalars &S = sc[rhs];
  double *H = g.H + (size_t)rhs * (k + 1) * k;  // column-major: H[col * (k+1) + row]
  double *cs = g.cs + (size_t)rhs * k, *sn = g.sn + (size_t)rhs * k, *gg = g.g + (size_t)rhs * (k + 1);
  const double *hc = g.hcol + (size_t)rhs * (k + 1);
  double *col = H + (size_t)j * (k + 1);
  const double hnext = sqrt(tot[0]);
  for (int i = 0; i <= j; ++i) col[i] = hc[i];
  col[j + 1] = hnext;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  cs[j] = col[j] / den;
  sn[j] = col[j + 1] / den;
  col[j] = den;
  col[j + 1] = hnext;  // kept for the scaling of V_{j+1}; not part of the triangular factor
  gg[j + 1] = -sn[j] * gg[j];
  gg[j] = cs[j] * gg[j];
  S.iters += 1;
  S.jdone = j + 1;
  S.rr = gg[j + 1] * gg[j + 1];
  if (!isfinite(S.rr) || !isfinite(den)) S.state = ST_NAN;
  else if (S.rr <= S.tol2 * S.bb || hnext == 0.0 || S.iters >= max_iter || j + 1 >= k) S.state = ST_MET;
}

// V_{j+1} = w / h_{j+1,j}  (only systems still expanding)
__global__ void gm_next_kernel(const double *__restrict__ w, double *__restrict__ v, int j, size_t n,
                               const KrylovScalars *sc, GmresDev g) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const int k = g.k;
  const double h = g.H[(size_t)rhs * (k + 1) * k + (size_t)j * (k + 1) + j + 1];
  const double inv = 1.0 / h;
  const size_t off = (size_t)rhs * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    v[off + e] = w[off + e] * inv;
}

void gm_normalize(double *w, double *vnext, int j, size_t n, int nrhs, KrylovScalars *sc, GmresDev &g,
                  const Reduce &red, int max_iter, cudaStream_t s) {
  ProfScope prof(KC_GMRES, s);
  dim3 grid(reduce_blocks(n), nrhs);
  gm_norm_kernel<<<grid, 256, 0, s>>>(w, j, n, sc, g, red, max_iter);
  count_launch();
  LAG_LAUNCH_CHECK();
  gm_next_kernel<<<grid, 256, 0, s>>>(w, vnext, j, n, sc, g);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// end of cycle: y = R^{-1} g (R = rotated H, upper triangular), x += sum_i y_i Z_i
__global__ void gm_tri_kernel(KrylovScalars *sc, GmresDev g, int nrhs) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  const KrylovScalars &S = sc[rhs];
  const int k = g.k;
  double *y = g.y + (size_t)rhs * k;
  if (!(S.state == ST_RUN || S.state == ST_MET)) {
    for (int i = 0; i < k; ++i) y[i] = 0.0;
    return;
  }
  const int jd = S.jdone;
  const double *H = g.H + (size_t)rhs * (k + 1) * k, *gg = g.g + (size_t)rhs * (k + 1);
  for (int i = jd; i < k; ++i) y[i] = 0.0;
  for (int i = jd - 1; i >= 0; --i) {
    double acc = gg[i];
    for (int c = i + 1; c < jd; ++c) acc -= H[(size_t)c * (k + 1) + i] * y[c];
    y[i] = acc / H[(size_t)i * (k + 1) + i];
  }
}

__global__ void __launch_bounds__(256) gm_xupd_kernel(double *__restrict__ x, const double *__restrict__ Z, size_t n,
                                                      size_t zstride, const KrylovScalars *sc, GmresDev g) {
  const int rhs = blockIdx.y;
  const int st = sc[rhs].state;
  if (!(st == ST_RUN || st == ST_MET)) return;
  const int jd = sc[rhs].jdone;
  if (jd == 0) return;
  const double *y = g.y + (size_t)rhs * g.k;
  const size_t off = (size_t)rhs * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = x[off + e];
    for (int i = 0; i < jd; ++i) v = fma(y[i], Z[(size_t)i * zstride + off + e], v);
    x[off + e] = v;
  }
}

void gm_update_x(double *x, const double *Z, int, size_t n, int nrhs, size_t zstride, const KrylovScalars *sc,
                 GmresDev &g, cudaStream_t s) {
  ProfScope prof(KC_GMRES, s);
  gm_tri_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(const_cast<KrylovScalars *>(sc), g, nrhs);
  count_launch();
  LAG_LAUNCH_CHECK();
  dim3 grid(reduce_blocks(n), nrhs);
  gm_xupd_kernel<<<grid, 256, 0, s>>>(x, Z, n, zstride, sc, g);
  count_launch();
  LAG_LAUNCH_CHECK();
}

}  // namespace lag
