// Axisymmetric elastic operator (Sec. 2.2 Eqs. 10-12 in cylindrical coordinates (r, z)), the
// gradient of a discrete strain energy, so that C is symmetric and the traction-free surface is the
// energy's natural condition.  Kernel layout: rows = radii i (nr), row length = depth nodes k (nzc);
// fields [rhs][comp][nr][nzc], comp 0 = Q (u_r), comp 1 = U (u_z).  With r_i = (i + 1/2) hr and
// rbar_i = (i + 1) hr (the face between radii i and i + 1):
//   r-faces (i+1/2, k), weight rbar: (l+2m) e_rr^2 + m U_r^2 + 2 l e_rr <e_tt>,
//   z-faces (i, k+1/2), weight r:    (l+2m) e_zz^2 + m Q_z^2 + 2 l e_zz <e_tt>,
//   nodes, weight r:                 (l+2m) e_tt^2 (e_tt = Q / r),
//   corners (i+1/2, k+1/2), weight rbar: 2 l <e_rr> <e_zz> + 2 m <Q_z> <U_r>,
// with <.> the mean of the two neighbouring values, e_rr = dQ/dr and U_r across r-faces, e_zz = dU/dz
// and Q_z across z-faces; Q = U = 0 on the ghost radius nr; no faces on the axis (rbar = 0), at
// z = 0 or at the bottom.  Each thread forms the two components of one node from the quadrature
// points around it (2 r-faces, 2 z-faces, 4 corners, the node), plus the mass r rho h^2/4.
#include "internal.h"

namespace lag {

// coef layout (each [nr][nzc]): p_r, m_r, l_r | p_z, m_z, l_z | p_n | l_c, m_c
struct CylElasticCoef {
  const double *p_r, *m_r, *l_r, *p_z, *m_z, *l_z, *p_n, *l_c, *m_c;
};

static CylElasticCoef cyl_elastic_coef(const lag_medium &m) {
  const size_t n = (size_t)m.grid.nx * m.grid.nz;
  const double *b = m.coef.as<double>();
  CylElasticCoef c;
  c.p_r = b;
  c.m_r = b + n;
  c.l_r = b + 2 * n;
  c.p_z = b + 3 * n;
  c.m_z = b + 4 * n;
  c.l_z = b + 5 * n;
  c.p_n = b + 6 * n;
  c.l_c = b + 7 * n;
  c.m_c = b + 8 * n;
  return c;
}

// face / corner means of the nodal lambda, mu (the ghost radius takes the last node's values)
__global__ void cyl_elastic_coef_kernel(const double *__restrict__ vp, const double *__restrict__ vs,
                                        const double *__restrict__ rho, int nzc, int nr, double hr, double h2,
                                        double *out, double *rh2, double *p2m, double *mu_n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (k >= nzc || i >= nr) return;
  const size_t n = (size_t)nr * nzc;
  auto LM = [&](int ii, int kk, double &l, double &m) {
    ii = min(ii, nr - 1);
    const size_t o = (size_t)ii * nzc + kk;
    const double r = rho[o], a = vp[o], b = vs[o];
    m = r * b * b;
    l = r * (a * a - 2.0 * b * b);
  };
  double l0, m0, l1, m1;
  LM(i, k, l0, m0);
  LM(i + 1, k, l1, m1);  // the ghost radius repeats the last node
  const size_t o = (size_t)i * nzc + k;
  const double lr = 0.5 * (l0 + l1), mr = 0.5 * (m0 + m1);
  out[o] = lr + 2.0 * mr;           // p_r
  out[n + o] = mr;                  // m_r
  out[2 * n + o] = lr;              // l_r
  out[6 * n + o] = l0 + 2.0 * m0;   // p_n
  if (k + 1 < nzc) {
    double l2, m2, l3, m3;
    LM(i, k + 1, l2, m2);
    LM(i + 1, k + 1, l3, m3);
    const double lz = 0.5 * (l0 + l2), mz = 0.5 * (m0 + m2);
    out[3 * n + o] = lz + 2.0 * mz;                         // p_z
    out[4 * n + o] = mz;                                    // m_z
    out[5 * n + o] = lz;                                    // l_z
    out[7 * n + o] = 0.5 * (lr + 0.5 * (l2 + l3));          // l_c: mean of the two r-face means
    out[8 * n + o] = 0.5 * (mr + 0.5 * (m2 + m3));          // m_c
  } else {
    out[3 * n + o] = out[4 * n + o] = out[5 * n + o] = out[7 * n + o] = out[8 * n + o] = 0.0;
  }
  const double r_i = (i + 0.5) * hr;
  rh2[o] = r_i * rho[o] * h2;
  p2m[o] = l0 + 2.0 * m0;
  mu_n[o] = m0;
}

// mode 0: every rhs (or those running when sc is given); mode 2: rhs running or ST_MET
__global__ void __launch_bounds__(256) cyl_elastic_apply_kernel(const double *__restrict__ X, double *__restrict__ Y,
                                                                int nzc, int nr, double hr, double hz,
                                                                CylElasticCoef c, const double *__restrict__ rh2,
                                                                const KrylovScalars *__restrict__ sc, int mode) {
  const int b = blockIdx.z;
  if (sc != nullptr) {
    const int st = sc[b].state;
    if (!(st == ST_RUN || (mode == 2 && st == ST_MET))) return;
  }
  const int k = blockIdx.x * 32 + (threadIdx.x & 31);
  const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (k >= nzc || i >= nr) return;
  const size_t plane = (size_t)nr * nzc;
  const double *Qf = X + (size_t)b * 2 * plane, *Uf = Qf + plane;
  double *yq = Y + (size_t)b * 2 * plane, *yu = yq + plane;
  auto Q = [&](int ii, int kk) -> double { return (ii < nr && kk >= 0 && kk < nzc) ? Qf[(size_t)ii * nzc + kk] : 0.0; };
  auto U = [&](int ii, int kk) -> double { return (ii < nr && kk >= 0 && kk < nzc) ? Uf[(size_t)ii * nzc + kk] : 0.0; };
  auto rr = [&](int ii) { return (ii + 0.5) * hr; };
  const double ihr = 1.0 / hr, ihz = 1.0 / hz;
  // r-face (ii+1/2, k): s_rr, s_tt, s_ur (0 outside 0 <= ii < nr)
  auto rface = [&](int ii, double &srr, double &stt, double &sur) {
    srr = stt = sur = 0.0;
    if (ii < 0 || ii >= nr) return;
    const size_t o = (size_t)ii * nzc + k;
    const double qa = Q(ii, k), qb = Q(ii + 1, k), ua = U(ii, k), ub = U(ii + 1, k);
    const double err = (qb - qa) * ihr;
    const double ett = 0.5 * (qa / rr(ii) + qb / rr(ii + 1));
    const double rb = (ii + 1.0) * hr;
    srr = rb * (c.p_r[o] * err + c.l_r[o] * ett);
    stt = rb * c.l_r[o] * err;
    sur = rb * c.m_r[o] * (ub - ua) * ihr;
  };
  // z-face (i, kk+1/2): s_zz, s_tz, s_qz (0 outside 0 <= kk < nzc - 1)
  auto zface = [&](int kk, double &szz, double &stz, double &sqz) {
    szz = stz = sqz = 0.0;
    if (kk < 0 || kk + 1 >= nzc) return;
    const size_t o = (size_t)i * nzc + kk;
    const double qa = Q(i, kk), qb = Q(i, kk + 1), ua = U(i, kk), ub = U(i, kk + 1);
    const double ezz = (ub - ua) * ihz;
    const double ett = 0.5 * (qa + qb) / rr(i);
    const double r = rr(i);
    szz = r * (c.p_z[o] * ezz + c.l_z[o] * ett);
    stz = r * c.l_z[o] * ezz;
    sqz = r * c.m_z[o] * (qb - qa) * ihz;
  };
  // corner (ii+1/2, kk+1/2): X = rbar l <e_zz>, X2 = rbar l <e_rr>, Y = rbar m <U_r>, Y2 = rbar m <Q_z>
  auto corner = [&](int ii, int kk, double &x1, double &x2, double &y1, double &y2) {
    x1 = x2 = y1 = y2 = 0.0;
    if (ii < 0 || ii >= nr || kk < 0 || kk + 1 >= nzc) return;
    const size_t o = (size_t)ii * nzc + kk;
    const double q00 = Q(ii, kk), q10 = Q(ii + 1, kk), q01 = Q(ii, kk + 1), q11 = Q(ii + 1, kk + 1);
    const double u00 = U(ii, kk), u10 = U(ii + 1, kk), u01 = U(ii, kk + 1), u11 = U(ii + 1, kk + 1);
    const double err = 0.5 * ((q10 - q00) + (q11 - q01)) * ihr;
    const double ezz = 0.5 * ((u01 - u00) + (u11 - u10)) * ihz;
    const double qz = 0.5 * ((q01 - q00) + (q11 - q10)) * ihz;
    const double ur = 0.5 * ((u10 - u00) + (u11 - u01)) * ihr;
    const double rb = (ii + 1.0) * hr;
    const double lc = rb * c.l_c[o], mc = rb * c.m_c[o];
    x1 = lc * ezz;
    x2 = lc * err;
    y1 = mc * ur;
    y2 = mc * qz;
  };
  const double ri = rr(i);
  double srr0, stt0, sur0, srr1, stt1, sur1;
  rface(i - 1, srr0, stt0, sur0);
  rface(i, srr1, stt1, sur1);
  double szz0, stz0, sqz0, szz1, stz1, sqz1;
  zface(k - 1, szz0, stz0, sqz0);
  zface(k, szz1, stz1, sqz1);
  // corners around the node: (i-1, k-1), (i-1, k), (i, k-1), (i, k)
  double xa[4], xb[4], ya[4], yb[4];
  corner(i - 1, k - 1, xa[0], xb[0], ya[0], yb[0]);
  corner(i - 1, k, xa[1], xb[1], ya[1], yb[1]);
  corner(i, k - 1, xa[2], xb[2], ya[2], yb[2]);
  corner(i, k, xa[3], xb[3], ya[3], yb[3]);
  const size_t o = (size_t)i * nzc + k;
  const double q = Qf[o], u = Uf[o];
  const double w = 0.25 * rh2[o];
  double gq = (srr0 - srr1) * ihr + 0.5 * (stt1 + stt0) / ri;
  gq += 0.5 * (stz0 + stz1) / ri + (sqz0 - sqz1) * ihz;
  gq += c.p_n[o] * q / ri;
  // dr^T(avz^T(X)) and dz^T(avr^T(Y))
  gq += (0.5 * (xa[0] + xa[1]) - 0.5 * (xa[2] + xa[3])) * ihr;
  gq += (0.5 * (ya[2] + ya[0]) - 0.5 * (ya[3] + ya[1])) * ihz;
  double gu = (sur0 - sur1) * ihr + (szz0 - szz1) * ihz;
  // dz^T(avr^T(X2)) and dr^T(avz^T(Y2))
  gu += (0.5 * (xb[2] + xb[0]) - 0.5 * (xb[3] + xb[1])) * ihz;
  gu += (0.5 * (yb[0] + yb[1]) - 0.5 * (yb[2] + yb[3])) * ihr;
  yq[o] = gq + w * q;
  yu[o] = gu + w * u;
}

void medium_build_elastic_cylindrical(lag_medium &m, const double *vp_host, const double *vs_host,
                                      const double *rho_host, cudaStream_t s) {
  const int nzc = m.grid.nx, nr = m.grid.nz;  // kernel layout: rows = radii
  const size_t n = (size_t)nzc * nr;
  m.ncoef = 9 * n;
  m.coef.alloc(m.ctx, m.ncoef * sizeof(double));
  m.rho_h2.alloc(m.ctx, n * sizeof(double));
  DevBuf tmp;
  tmp.alloc(m.ctx, (5 * n + 8) * sizeof(double));
  double *dvp = tmp.as<double>(), *dvs = dvp + n, *drho = dvs + n, *p2m = drho + n, *mun = p2m + n, *mm = mun + n;
  LAG_CUDA_CHECK(cudaMemcpyAsync(dvp, vp_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(dvs, vs_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  LAG_CUDA_CHECK(cudaMemcpyAsync(drho, rho_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  dim3 g((nzc + 127) / 128, nr);
  cyl_elastic_coef_kernel<<<g, 128, 0, s>>>(dvp, dvs, drho, nzc, nr, m.grid.dz, m.h * m.h, m.coef.as<double>(),
                                            m.rho_h2.as<double>(), p2m, mun);
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
                       cudaStream_t s) {
  const int nzc = m.grid.nx, nr = m.grid.nz;
  dim3 g((nzc + 31) / 32, (nr + 7) / 8, nrhs);
  ProfScope prof(KC_STENCIL_E, s);
  cyl_elastic_apply_kernel<<<g, 256, 0, s>>>(p, q, nzc, nr, m.grid.dz, m.grid.dx, cyl_elastic_coef(m),
                                             m.rho_h2.as<double>(), sc, mode);
  count_launch();
  LAG_LAUNCH_CHECK();
}

}  // namespace lag
