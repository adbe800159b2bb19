// Shots: the whole Laguerre harmonic loop of Sec. 2.1 (acoustic) / Sec. 2.2 (elastic) on the device.
//
// For m = 0, 1, ..., n-1 (sequential: the right-hand side of m needs R_0..R_{m-1}):
//   b_m = delta_s f_m - rho h^2 c_m S_m            (Eq. 9 / Eq. 12 in SPD form)
//   solve A R_m = b_m (PCG) or C R_m = b_m (FGMRES) to the tolerance, zero initial guess
//   T += c^_m R_m, S += T                          (so that S_{m+1} = sum_{k<=m} (m+1-k) c^_k R_k)
//   keep R_m at the receivers
// and at the end u(t_j) = sum_m R_m(rcv) (h t_j)^{alpha/2} l_m(h t_j) (Eq. 8).  The history of
// the series is carried in two running sums per source instead of all earlier harmonics.
#include <cmath>
#include <cstring>
#include <vector>

#include "solver.h"

using namespace lag;

lag_shot::~lag_shot() {
  if (stream) cudaStreamSynchronize(stream);
  delete p1;
  delete p2;
  delete medium;
  if (stream) cudaStreamDestroy(stream);
}

static void validate_shot(const lag_grid &g, const lag_laguerre &lag, const lag_solver &s, const lag_wavelet &w,
                          int nsrc, const lag_point *src, int nrcv, const lag_point *rcv, int nt, const double *t,
                          bool elastic) {
  if (g.nx < 1 || g.nz < 1 || !(g.dx > 0) || !(g.dz > 0)) throw Error(LAG_EINVAL, "bad grid");
  if (lag.n_harm < 1 || lag.alpha < 0 || !(lag.h > 0)) throw Error(LAG_EINVAL, "bad Laguerre parameters");
  check_solver(s, elastic);
  if (!(w.f0 > 0) || (w.kind != LAG_WAVELET_RICKER && w.kind != LAG_WAVELET_PAPER) ||
      (w.kind == LAG_WAVELET_PAPER && !(w.gamma > 0)))
    throw Error(LAG_EINVAL, "bad wavelet");
  if (nsrc < 1 || src == nullptr) throw Error(LAG_EINVAL, "need at least one source");
  if (nrcv < 0 || (nrcv > 0 && rcv == nullptr) || nt < 0 || (nt > 0 && t == nullptr))
    throw Error(LAG_EINVAL, "bad receivers / output times");
  for (int i = 0; i < nsrc; ++i)
    if (src[i].ix < 0 || src[i].ix >= g.nx || src[i].iz < 0 || src[i].iz >= g.nz)
      throw Error(LAG_EINVAL, "source outside the grid");
  for (int i = 0; i < nrcv; ++i)
    if (rcv[i].ix < 0 || rcv[i].ix >= g.nx || rcv[i].iz < 0 || rcv[i].iz >= g.nz)
      throw Error(LAG_EINVAL, "receiver outside the grid");
}

lag_shot *shot_new(lag_ctx *ctx, const lag_grid &g, const double *c, const double *vs, const double *rho,
                   const lag_laguerre &lag, const lag_solver &s, const lag_wavelet &w, int nsrc, const lag_point *src,
                   int nrcv, const lag_point *rcv, int nt, const double *t_out) {
  const bool elastic = vs != nullptr;
  validate_shot(g, lag, s, w, nsrc, src, nrcv, rcv, nt, t_out, elastic);
  const size_t before = ctx->in_use.load();
  std::unique_ptr<lag_shot> sh(new lag_shot());
  sh->ctx = ctx;
  sh->grid = g;
  sh->lag = lag;
  sh->solver = s;
  sh->wavelet = w;
  sh->elastic = elastic;
  sh->nsrc = nsrc;
  sh->nrcv = nrcv;
  sh->nt = nt;
  sh->ncomp = elastic ? 2 : 1;
  sh->t_start = now_seconds();
  LAG_CUDA_CHECK(cudaStreamCreateWithFlags(&sh->stream, cudaStreamNonBlocking));
  cudaStream_t st = sh->stream;
  sh->medium = medium_new(ctx, g, c, vs, rho, lag.h, st);
  const double *mid = sh->medium->mid;
  if (g.cylindrical && elastic && s.layered)
    throw Error(LAG_EINVAL, "the layered preconditioner is acoustic only on cylindrical grids");
  if (!elastic && s.layered) {
    // per-row midranges kappa~(z), rho~(z): ax = az = kappa~(z), d = rho~(z) h^2 / 4 (cylindrical
    // grids: per radius, the rows of the kernel grid)
    const int nz = g.cylindrical ? g.nx : g.nz;
    std::vector<double> mm(4 * (size_t)nz), rows(3 * (size_t)nz);
    LAG_CUDA_CHECK(cudaMemcpyAsync(mm.data(), sh->medium->rowmm.ptr, mm.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    LAG_CUDA_CHECK(cudaStreamSynchronize(st));
    for (int k = 0; k < nz; ++k) {
      const double kz = 0.5 * (mm[2 * k] + mm[2 * k + 1]);
      const double rz = 0.5 * (mm[2 * (nz + k)] + mm[2 * (nz + k) + 1]);
      rows[k] = rows[nz + k] = kz;
      rows[2 * nz + k] = rz * lag.h * lag.h / 4.0;
    }
    sh->p1 = precond_new(ctx, g, 0.0, 0.0, 0.0, s.prec, s.partitions, st, rows.data());
  } else if (!elastic) {
    sh->p1 = precond_new(ctx, g, mid[0], mid[0], mid[1] * lag.h * lag.h / 4.0, s.prec, s.partitions, st);
  } else if (s.layered) {
    // Eq. (22)'s K with per-row midranges: B1 (ax, az) = ((l+2m)~(z), mu~(z)), B2 = (mu~(z),
    // (l+2m)~(z)), d = rho~(z) h^2 / 4
    const int nz = g.nz;
    std::vector<double> mm(6 * (size_t)nz), r1(3 * (size_t)nz), r2(3 * (size_t)nz);
    LAG_CUDA_CHECK(cudaMemcpyAsync(mm.data(), sh->medium->rowmm.ptr, mm.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    LAG_CUDA_CHECK(cudaStreamSynchronize(st));
    for (int k = 0; k < nz; ++k) {
      const double pz = 0.5 * (mm[2 * k] + mm[2 * k + 1]);
      const double uz = 0.5 * (mm[2 * (nz + k)] + mm[2 * (nz + k) + 1]);
      const double rz = 0.5 * (mm[2 * (2 * nz + k)] + mm[2 * (2 * nz + k) + 1]);
      r1[k] = pz;
      r1[nz + k] = uz;
      r2[k] = uz;
      r2[nz + k] = pz;
      r1[2 * nz + k] = r2[2 * nz + k] = rz * lag.h * lag.h / 4.0;
    }
    sh->p1 = precond_new(ctx, g, 0.0, 0.0, 0.0, s.prec, s.partitions, st, r1.data());
    sh->p2 = precond_new(ctx, g, 0.0, 0.0, 0.0, s.prec, s.partitions, st, r2.data());
  } else {  // K = diag(B1, B2), Eq. (22): B1 (ax, az) = ((l+2m)~, mu~), B2 = (mu~, (l+2m)~)
    const double d = mid[2] * lag.h * lag.h / 4.0;
    // cylindrical grids: B1 also holds the hoop term (l+2m)~/r (Eq. 22)
    sh->p1 = precond_new(ctx, g, mid[0], mid[1], d, s.prec, s.partitions, st, nullptr, g.cylindrical ? mid[0] : 0.0);
    sh->p2 = precond_new(ctx, g, mid[1], mid[0], d, s.prec, s.partitions, st);
  }
  if (s.tune) {  // the autotuner issues on the context stream: the plans are complete already
    for (lag_precond *q : {sh->p1, sh->p2}) {
      if (q == nullptr) continue;
      const int rc = lag_precond_autotune(q, nsrc * sh->ncomp, nullptr, nullptr, nullptr, nullptr);
      if (rc != LAG_OK) throw Error(rc, std::string("autotune: ") + ctx->last_error);
    }
  }
  sh->wk.setup(ctx, sh->medium, sh->p1, sh->p2, s, nsrc, st);
  const size_t n = sh->wk.n;
  sh->hist.alloc(ctx, 2 * n * nsrc * sizeof(double), true);
  const size_t rows = (size_t)nsrc * sh->ncomp * nrcv;
  const size_t ntab = (size_t)lag.n_harm + (size_t)lag.n_harm * nt + nt + (size_t)lag.n_harm * rows + rows * nt;
  sh->tables.alloc(ctx, ntab * sizeof(double), true);
  sh->idx.alloc(ctx, (size_t)(nsrc + nrcv + 1) * sizeof(int));
  std::vector<int> hidx(nsrc + nrcv + 1, 0);
  // node offsets in the field layout: [nz][nx] (Cartesian) or [nx][nz] (cylindrical)
  auto offset = [&](const lag_point &q) { return g.cylindrical ? q.ix * g.nz + q.iz : q.iz * g.nx + q.ix; };
  for (int i = 0; i < nsrc; ++i) hidx[i] = offset(src[i]);
  for (int i = 0; i < nrcv; ++i) hidx[nsrc + i] = offset(rcv[i]);
  LAG_CUDA_CHECK(cudaMemcpyAsync(sh->idx.ptr, hidx.data(), hidx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  source_coeffs_device(lag, w, sh->fm(), sh->fm_scratch, ctx, st);
  if (nt > 0) {
    LAG_CUDA_CHECK(cudaMemcpyAsync(sh->tout(), t_out, nt * sizeof(double), cudaMemcpyHostToDevice, st));
    laguerre_table_device(lag, nt, sh->tout(), sh->tab(), st);
  }
  sh->cm.resize(lag.n_harm);
  sh->chat.resize(lag.n_harm);
  for (int m = 0; m < lag.n_harm; ++m) {
    const double lc = 0.5 * (std::lgamma((double)m + 1.0) - std::lgamma((double)m + lag.alpha + 1.0));
    sh->cm[m] = std::exp(lc);      // c_m = sqrt(m!/(m+alpha)!)
    sh->chat[m] = std::exp(-lc);   // c^_m = sqrt((m+alpha)!/m!)
  }
  sh->iters.assign((size_t)nsrc * lag.n_harm, 0);
  sh->relres.assign((size_t)nsrc * lag.n_harm, 0.0);
  LAG_CUDA_CHECK(cudaStreamSynchronize(st));
  sh->fm_scratch.release();
  sh->device_bytes = ctx->in_use.load() - before;
  return sh.release();
}

int lag_shot::pump(bool block) {
  const size_t n = wk.n;
  const size_t nplane = wk.nplane;
  const int *src_idx = idx.as<int>(), *rcv_idx = src_idx + nsrc;
  double *T = hist.as<double>(), *S = T + n * nsrc;
  for (;;) {
    if (failed) return 1;
    if (m >= lag.n_harm) return 1;
    if (phase == 0) {
      // point source per unit cell: 1/(dx dz); cylindrical: 1/(2 pi dr dz) (Eq. 1's delta / (2 pi r)
      // in the r-weighted equation)
      const double inv_cell = grid.cylindrical ? 1.0 / (2.0 * M_PI * grid.dx * grid.dz) : 1.0 / (grid.dx * grid.dz);
      laguerre_rhs(medium->rho_h2.as<double>(), S, cm[m], fm(), m, src_idx, elastic ? 1 : 0,
                   inv_cell, ncomp, nplane, nsrc, wk.r(), wk.x(), elastic ? nullptr : wk.vec(3), solver.tol, wk.sc(),
                   wk.red.get(), stream);
      wk.start_from_r();
      wk.enqueue_chunk();
      phase = 1;
    }
    const int st = wk.poll(block);
    if (st < 0) return 0;
    if (st == 0) {
      wk.enqueue_chunk();
      if (!block) return 0;
      continue;
    }
    if (elastic && wk.cycle_open) wk.cycle_open = false;
    const int fs = wk.finish_status();
    for (int i = 0; i < nsrc; ++i) {
      const KrylovScalars &k = wk.hsc[i];
      iters[(size_t)i * lag.n_harm + m] = k.iters;
      relres[(size_t)i * lag.n_harm + m] = k.bb > 0 ? std::sqrt(k.rr / k.bb) : 0.0;
      total_iters += k.iters;
    }
    if (fs == LAG_ENUMERIC) {
      failed = true;
      last_status = LAG_ENUMERIC;
      return 1;
    }
    if (fs == LAG_ENOTCONV) last_status = LAG_ENOTCONV;
    laguerre_accumulate(wk.x(), T, S, chat[m], n, nsrc, stream);
    gather_receivers(wk.x(), rcv_idx, nrcv, ncomp, nplane, nsrc, rrcv() + (size_t)m * nsrc * ncomp * nrcv, stream);
    ++m;
    phase = 0;
    if (m >= lag.n_harm) return 1;
    if (block) return 0;  // a blocking caller counts harmonics itself
  }
}

static thread_local std::string g_shot_err;

template <typename F>
static int guarded_shot(lag_ctx *ctx, F &&f) {
  try {
    return f();
  } catch (const Error &e) {
    if (ctx) ctx->last_error = e.what();
    return e.status;
  } catch (const std::exception &e) {
    if (ctx) ctx->last_error = e.what();
    return LAG_ECUDA;
  }
}

extern "C" {

int lag_shot_create(lag_ctx *ctx, const lag_grid *grid, const double *c, const double *vs, const double *rho,
                    const lag_laguerre *lag, const lag_solver *s, const lag_wavelet *w, int nsrc, const lag_point *src,
                    int nrcv, const lag_point *rcv, int nt, const double *t_out, lag_shot **out) {
  if (!ctx || !grid || !c || !rho || !lag || !s || !w || !out) return LAG_EINVAL;
  *out = nullptr;
  return guarded_shot(ctx, [&] {
    LAG_CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = shot_new(ctx, *grid, c, vs, rho, *lag, *s, *w, nsrc, src, nrcv, rcv, nt, t_out);
    return LAG_OK;
  });
}

void lag_shot_destroy(lag_shot *sh) {
  if (!sh) return;
  cudaSetDevice(sh->ctx->device);
  delete sh;
}

int lag_shot_step(lag_shot *sh, int nharm) {
  if (!sh || nharm < 0) return LAG_EINVAL;
  return guarded_shot(sh->ctx, [&] {
    LAG_CUDA_CHECK(cudaSetDevice(sh->ctx->device));
    const double t0 = now_seconds();
    const int target = std::min(sh->lag.n_harm, sh->m + nharm);
    while (sh->m < target && !sh->failed) sh->pump(true);
    LAG_CUDA_CHECK(cudaStreamSynchronize(sh->stream));
    sh->t_busy += now_seconds() - t0;
    return sh->failed ? sh->last_status : sh->last_status;
  });
}

int lag_shot_pump(lag_shot *sh, int *done) {
  if (!sh) return LAG_EINVAL;
  return guarded_shot(sh->ctx, [&] {
    const int d = sh->pump(false);
    if (done) *done = d;
    return sh->failed ? sh->last_status : LAG_OK;
  });
}

int lag_shot_harmonic(const lag_shot *sh) { return sh ? sh->m : 0; }
void *lag_shot_stream(const lag_shot *sh) { return sh ? (void *)sh->stream : nullptr; }

int lag_shot_traces(lag_shot *sh, double *traces_host) {
  if (!sh || !traces_host) return LAG_EINVAL;
  return guarded_shot(sh->ctx, [&] {
    const int rows = sh->nsrc * sh->ncomp * sh->nrcv;
    if (rows == 0 || sh->nt == 0) return LAG_OK;
    inverse_sum(sh->rrcv(), sh->tab(), sh->m, rows, sh->nt, sh->traces(), sh->stream);
    LAG_CUDA_CHECK(cudaMemcpyAsync(traces_host, sh->traces(), (size_t)rows * sh->nt * sizeof(double),
                                   cudaMemcpyDeviceToHost, sh->stream));
    LAG_CUDA_CHECK(cudaStreamSynchronize(sh->stream));
    return LAG_OK;
  });
}

int lag_shot_receiver_harmonics(lag_shot *sh, double *out) {
  if (!sh || !out) return LAG_EINVAL;
  return guarded_shot(sh->ctx, [&] {
    const size_t cnt = (size_t)sh->lag.n_harm * sh->nsrc * sh->ncomp * sh->nrcv;
    if (cnt == 0) return LAG_OK;
    LAG_CUDA_CHECK(cudaMemcpyAsync(out, sh->rrcv(), cnt * sizeof(double), cudaMemcpyDeviceToHost, sh->stream));
    LAG_CUDA_CHECK(cudaStreamSynchronize(sh->stream));
    return LAG_OK;
  });
}

const double *lag_shot_field(const lag_shot *sh) { return sh ? sh->wk.x() : nullptr; }

int lag_shot_copy_field(lag_shot *sh, double *out) {
  if (!sh || !out) return LAG_EINVAL;
  return guarded_shot(sh->ctx, [&] {
    LAG_CUDA_CHECK(cudaMemcpyAsync(out, sh->wk.x(), sh->wk.n * sh->nsrc * sizeof(double), cudaMemcpyDeviceToDevice,
                                   sh->stream));
    LAG_CUDA_CHECK(cudaStreamSynchronize(sh->stream));
    return LAG_OK;
  });
}

int lag_shot_stats(const lag_shot *sh, lag_stats *st) {
  if (!sh || !st) return LAG_EINVAL;
  const int n = sh->lag.n_harm;
  for (int i = 0; i < sh->nsrc; ++i)
    for (int m = 0; m < n; ++m) {
      if (st->iters) st->iters[(size_t)i * n + m] = sh->iters[(size_t)i * n + m];
      if (st->relres) st->relres[(size_t)i * n + m] = sh->relres[(size_t)i * n + m];
    }
  st->total_iters = sh->total_iters;
  st->seconds = sh->t_busy;
  return LAG_OK;
}

static int solve_whole(lag_ctx *ctx, const lag_grid *grid, const double *c, const double *vs, const double *rho,
                       const lag_laguerre *lag, const lag_solver *s, const lag_wavelet *w, int nsrc,
                       const lag_point *src, int nrcv, const lag_point *rcv, int nt, const double *t_out,
                       double *traces, lag_stats *stats) {
  const double t0 = now_seconds();
  lag_shot *sh = nullptr;
  int rc = lag_shot_create(ctx, grid, c, vs, rho, lag, s, w, nsrc, src, nrcv, rcv, nt, t_out, &sh);
  if (rc != LAG_OK) return rc;
  rc = lag_shot_step(sh, lag->n_harm);
  if (rc == LAG_OK || rc == LAG_ENOTCONV) {
    const int rc2 = (traces != nullptr) ? lag_shot_traces(sh, traces) : LAG_OK;
    if (rc2 != LAG_OK) rc = rc2;
  }
  if (stats) {
    lag_shot_stats(sh, stats);
    stats->seconds = now_seconds() - t0;
  }
  lag_shot_destroy(sh);
  return rc;
}

int lag_solve_acoustic(lag_ctx *ctx, const lag_grid *grid, const double *c, const double *rho, const lag_laguerre *lag,
                       const lag_solver *s, const lag_wavelet *w, int nsrc, const lag_point *src, int nrcv,
                       const lag_point *rcv, int nt, const double *t_out, double *traces, lag_stats *stats) {
  if (!ctx || !c || !rho) return LAG_EINVAL;
  return solve_whole(ctx, grid, c, nullptr, rho, lag, s, w, nsrc, src, nrcv, rcv, nt, t_out, traces, stats);
}

int lag_solve_elastic(lag_ctx *ctx, const lag_grid *grid, const double *vp, const double *vs, const double *rho,
                      const lag_laguerre *lag, const lag_solver *s, const lag_wavelet *w, int nsrc,
                      const lag_point *src, int nrcv, const lag_point *rcv, int nt, const double *t_out,
                      double *traces, lag_stats *stats) {
  if (!ctx || !vp || !vs || !rho) return LAG_EINVAL;
  return solve_whole(ctx, grid, vp, vs, rho, lag, s, w, nsrc, src, nrcv, rcv, nt, t_out, traces, stats);
}

}  // extern "C"
