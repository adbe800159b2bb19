// Axisymmetric elastic operator (Sec. 2.2 Eqs. 10-12 in cylindrical coordinates (r, z)), the
// Hessian of a discrete strain energy, so that C is symmetric and the traction-free surface is the
// energy's natural condition.  Kernel layout: rows = radii i (nr), row length = depth nodes k (nzc);
// fields [rhs][comp][nr][nzc], comp 0 = Q (u_r), comp 1 = U (u_z).  With r_i = (i + 1/2) hr and
// rbar_i = (i + 1) hr (the face between radii i and i + 1), the energy per unit area is
//   r-faces (i+1/2, k), weight rbar: (l+2m) e_rr^2 + m U_r^2 + 2 l e_rr <e_tt>,
//   z-faces (i, k+1/2), weight r:    (l+2m) e_zz^2 + m Q_z^2 + 2 l e_zz <e_tt>,
//   nodes, weight r:                 (l+2m) e_tt^2 (e_tt = Q / r),
//   corners (i+1/2, k+1/2), weight rbar: 2 l <e_rr> <e_zz> + 2 m <Q_z> <U_r>,
// (one half in front of the sum), <.> the mean of the two neighbouring values, e_rr = dQ/dr and U_r
// across r-faces, e_zz = dU/dz and Q_z across z-faces; Q = U = 0 on the ghost radius nr; no faces on
// the axis (rbar = 0), at z = 0 or at the bottom; face coefficients are node means (the ghost radius
// repeats the last node), corner coefficients means of the two r-face means.
//
// The energy is quadratic, so C is a fixed stencil: at the medium's creation one thread per node
// differentiates the energy terms around its node twice and stores the node's row of C,
//   Q-Q: diagonal dq, r-neighbour wqr (node i with i + 1), z-neighbour wqz (k with k + 1),
//   U-U: du, wur, wuz,
//   Q-U: x[9], the weights of U at (i + di, k + dk), di, dk in {-1, 0, 1} (index 3 (di+1) + dk+1),
// the mass r rho h^2/4 in both diagonals.  The U-Q block is the transpose (C is symmetric): the
// weight of Q(i + di, k + dk) in row U(i, k) is x[3 (1-di) + 1-dk] of node (i + di, k + dk).  The
// apply is then 28 FP64 multiply-adds per node, the least the stencil's 28 couplings allow (FP64
// throughput, not HBM, bounds this kernel on this part: about two FP64 FMAs per clock per SM).
#include "internal.h"

namespace lag {

// coef layout (each [nr][nzc]): dq, du, wqr, wur, wqz, wuz, x0..x8
enum { CE_DQ = 0, CE_DU, CE_WQR, CE_WUR, CE_WQZ, CE_WUZ, CE_X0, CE_NARRAYS = CE_X0 + 9 };

// one node's row of C from the energy terms around it (Hessian entries, see the file header)
__global__ void cyl_elastic_stencil_kernel(const double *__restrict__ vp, const double *__restrict__ vs,
                                           const double *__restrict__ rho, int nzc, int nr, double hr, double hz,
                                           double h2, double *out, double *rh2, double *p2m, double *mu_n) {
  const size_t n = (size_t)nr * nzc;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = (int)(t / nzc), k = (int)(t % nzc);
  // lambda, mu, l+2m on the 3 x 3 neighbourhood (the ghost radius repeats the last node; entries
  // outside the grid are never used)
  double Lm[3][3], Mu[3][3], Pn[3][3];
  for (int di = -1; di <= 1; ++di)
    for (int dk = -1; dk <= 1; ++dk) {
      const int ii = min(i + di, nr - 1), kk = k + dk;
      double l = 0.0, m = 0.0;
      if (ii >= 0 && kk >= 0 && kk < nzc) {
        const size_t o = (size_t)ii * nzc + kk;
        const double r = rho[o], a = vp[o], b = vs[o];
        m = r * b * b;
        l = r * (a * a - 2.0 * b * b);
      }
      Lm[di + 1][dk + 1] = l;
      Mu[di + 1][dk + 1] = m;
      Pn[di + 1][dk + 1] = l + 2.0 * m;
    }
  // face and corner means; di, dk are offsets of the face's / corner's lower node from (i, k)
  auto rf = [&](const double (&f)[3][3], int di, int dk) { return 0.5 * (f[di + 1][dk + 1] + f[di + 2][dk + 1]); };
  auto zf = [&](const double (&f)[3][3], int dk) { return 0.5 * (f[1][dk + 1] + f[1][dk + 2]); };
  auto cf = [&](const double (&f)[3][3], int di, int dk) { return 0.5 * (rf(f, di, dk) + rf(f, di, dk + 1)); };
  const double a = 1.0 / hr, c = 1.0 / hz;
  const double r_i = (i + 0.5) * hr, b0 = 0.5 / r_i;
  double dq = 0.0, du = 0.0, wqr = 0.0, wur = 0.0, wqz = 0.0, wuz = 0.0, x[9];
  for (int j = 0; j < 9; ++j) x[j] = 0.0;
  {  // r-face i: the node is its inner side
    const double p = rf(Pn, 0, 0), l = rf(Lm, 0, 0), m = rf(Mu, 0, 0), rb = (i + 1.0) * hr;
    dq += rb * (p * a * a - 2.0 * l * a * b0);
    du += rb * m * a * a;
    if (i + 1 < nr) {
      const double b1 = 0.5 / ((i + 1.5) * hr);
      wqr = rb * (-p * a * a + l * a * (b0 - b1));
      wur = -rb * m * a * a;
    }
  }
  if (i >= 1) {  // r-face i-1: the node is its outer side
    const double p = rf(Pn, -1, 0), l = rf(Lm, -1, 0), m = rf(Mu, -1, 0), rb = i * hr;
    dq += rb * (p * a * a + 2.0 * l * a * b0);
    du += rb * m * a * a;
  }
  if (k + 1 < nzc) {  // z-face k: the node is its upper side
    const double p = zf(Pn, 0), l = zf(Lm, 0), m = zf(Mu, 0);
    dq += r_i * m * c * c;
    du += r_i * p * c * c;
    wqz = -r_i * m * c * c;
    wuz = -r_i * p * c * c;
    x[4] -= 0.5 * l * c;   // U(i, k)
    x[5] += 0.5 * l * c;   // U(i, k+1)
  }
  if (k >= 1) {  // z-face k-1: the node is its lower side
    const double p = zf(Pn, -1), l = zf(Lm, -1), m = zf(Mu, -1);
    dq += r_i * m * c * c;
    du += r_i * p * c * c;
    x[3] -= 0.5 * l * c;   // U(i, k-1)
    x[4] += 0.5 * l * c;   // U(i, k)
  }
  dq += Pn[1][1] / r_i;  // node term (l+2m) e_tt^2
  const size_t o = (size_t)i * nzc + k;
  const double mass = 0.25 * r_i * rho[o] * h2;
  dq += mass;
  du += mass;
  // corners (ci + 1/2, ck + 1/2) around the node: l <e_rr><e_zz> + m <Q_z><U_r> with weight rbar
  for (int ci = i - 1; ci <= i; ++ci) {
    if (ci < 0) continue;
    for (int ck = k - 1; ck <= k; ++ck) {
      if (ck < 0 || ck + 1 >= nzc) continue;
      const double lc = cf(Lm, ci - i, ck - k), mc = cf(Mu, ci - i, ck - k);
      const double sc = (ci + 1.0) * hr * a * c * 0.25;
      const double srA = (ci == i - 1) ? 1.0 : -1.0, szA = (ck == k - 1) ? 1.0 : -1.0;
      for (int bi = ci; bi <= ci + 1; ++bi) {
        if (bi >= nr) continue;  // ghost radius
        for (int bk = ck; bk <= ck + 1; ++bk) {
          const double srB = (bi == ci + 1) ? 1.0 : -1.0, szB = (bk == ck + 1) ? 1.0 : -1.0;
          x[3 * (bi - i + 1) + (bk - k + 1)] += sc * (lc * srA * szB + mc * szA * srB);
        }
      }
    }
  }
  out[CE_DQ * n + o] = dq;
  out[CE_DU * n + o] = du;
  out[CE_WQR * n + o] = wqr;
  out[CE_WUR * n + o] = wur;
  out[CE_WQZ * n + o] = wqz;
  out[CE_WUZ * n + o] = wuz;
  for (int j = 0; j < 9; ++j) out[(CE_X0 + j) * n + o] = x[j];
  rh2[o] = r_i * rho[o] * h2;
  p2m[o] = Pn[1][1];
  mu_n[o] = Mu[1][1];
}

// mode 0: every rhs (or those running when sc is given); mode 2: rhs running or ST_MET
__global__ void __launch_bounds__(256) cyl_elastic_apply_kernel(const double *__restrict__ X, double *__restrict__ Y,
                                                                int nzc, int nr, const double *__restrict__ cf,
                                                                const KrylovScalars *__restrict__ sc, int mode,
                                                                const double *__restrict__ sub) {
  const int b = blockIdx.z;
  if (sc != nullptr) {
    const int st = sc[b].state;
    if (!(st == ST_RUN || (mode == 2 && st == ST_MET))) return;
  }
  const int k = blockIdx.x * 32 + (threadIdx.x & 31);
  const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (k >= nzc || i >= nr) return;
  const size_t n = (size_t)nr * nzc;
  const size_t o = (size_t)i * nzc + k;
  const double *Qf = X + (size_t)b * 2 * n, *Uf = Qf + n;
  const bool im = i >= 1, ip = i + 1 < nr, km = k >= 1, kp = k + 1 < nzc;
  const int s = nzc;
  double gq = __ldg(cf + CE_DQ * n + o) * __ldg(Qf + o);
  double gu = __ldg(cf + CE_DU * n + o) * __ldg(Uf + o);
  if (ip) {
    gq = fma(__ldg(cf + CE_WQR * n + o), __ldg(Qf + o + s), gq);
    gu = fma(__ldg(cf + CE_WUR * n + o), __ldg(Uf + o + s), gu);
  }
  if (im) {
    gq = fma(__ldg(cf + CE_WQR * n + o - s), __ldg(Qf + o - s), gq);
    gu = fma(__ldg(cf + CE_WUR * n + o - s), __ldg(Uf + o - s), gu);
  }
  if (kp) {
    gq = fma(__ldg(cf + CE_WQZ * n + o), __ldg(Qf + o + 1), gq);
    gu = fma(__ldg(cf + CE_WUZ * n + o), __ldg(Uf + o + 1), gu);
  }
  if (km) {
    gq = fma(__ldg(cf + CE_WQZ * n + o - 1), __ldg(Qf + o - 1), gq);
    gu = fma(__ldg(cf + CE_WUZ * n + o - 1), __ldg(Uf + o - 1), gu);
  }
  // Q-U block (row Q(i, k): x of this node) and its transpose (row U(i, k): x of the neighbour)
#pragma unroll
  for (int di = -1; di <= 1; ++di) {
    const bool vi = di < 0 ? im : (di > 0 ? ip : true);
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      const bool vk = dk < 0 ? km : (dk > 0 ? kp : true);
      if (vi && vk) {
        const long long off = (long long)di * s + dk;
        gq = fma(__ldg(cf + (CE_X0 + 3 * (di + 1) + dk + 1) * n + o), __ldg(Uf + o + off), gq);
        gu = fma(__ldg(cf + (CE_X0 + 3 * (1 - di) + 1 - dk) * n + o + off), __ldg(Qf + o + off), gu);
      }
    }
  }
  double *yq = Y + (size_t)b * 2 * n;
  if (sub != nullptr) {
    const double *sq = sub + (size_t)b * 2 * n;
    gq -= sq[o];
    gu -= sq[n + o];
  }
  yq[o] = gq;
  yq[n + o] = gu;
}

void medium_build_elastic_cylindrical(lag_medium &m, const double *vp_host, const double *vs_host,
                                      const double *rho_host, cudaStream_t s) {
  const int nzc = m.grid.nx, nr = m.grid.nz;  // kernel layout: rows = radii
  const size_t n = (size_t)nzc * nr;
  m.ncoef = CE_NARRAYS * n;
  m.coef.alloc(m.ctx, m.ncoef * sizeof(double));
  m.rho_h2.alloc(m.ctx, n * sizeof(double));
  DevBuf tmp;
  tmp.alloc(m.ctx, (5 * n + 8) * sizeof(double));
  double *dvp = tmp.as<double>(), *dvs = dvp + n, *drho = dvs + n, *p2m = drho + n, *mun = p2m + n, *mm = mun + n;
  LAG_CUDA_CHECK(cudaMemcpyAsync(dvp, vp_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(dvs, vs_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(drho, rho_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  if ((nr + 7) / 8 > 65535) throw Error(LAG_EINVAL, "cylindrical elastic grid: at most 524280 radii");
  cyl_elastic_stencil_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dvp, dvs, drho, nzc, nr, m.grid.dz, m.grid.dx,
                                               m.h * m.h, m.coef.as<double>(), m.rho_h2.as<double>(), p2m, mun);
  count_launch();
  LAG_LAUNCH_CHECK();
  // whole-medium midranges (l+2m)~, m~, rho~ (footnote to Eq. 21; Eq. 22 puts the r weights in the plan)
  midrange_device(p2m, n, mm, s);
  midrange_device(mun, n, mm + 2, s);
  midrange_device(drho, n, mm + 4, s);
  double h_mm[6];
  LAG_CUDA_CHECK(cudaMemcpyAsync(h_mm, mm, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
  m.mid[0] = 0.5 * (h_mm[0] + h_mm[1]);
  m.mid[1] = 0.5 * (h_mm[2] + h_mm[3]);
  m.mid[2] = 0.5 * (h_mm[4] + h_mm[5]);
}

void elastic_cyl_apply(const lag_medium &m, const double *p, double *q, int nrhs, const KrylovScalars *sc, int mode,
                       cudaStream_t s, const double *sub) {
  const int nzc = m.grid.nx, nr = m.grid.nz;
  dim3 g((nzc + 31) / 32, (nr + 7) / 8, nrhs);
  ProfScope prof(KC_STENCIL_E, s);
  cyl_elastic_apply_kernel<<<g, 256, 0, s>>>(p, q, nzc, nr, m.coef.as<double>(), sc, mode, sub);
  count_launch();
  LAG_LAUNCH_CHECK();
}

}  // namespace lag
