// C ABI of the library: contexts, media, preconditioner plans, Krylov drivers and shots.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "solver.h"

using namespace lag;

namespace lag {

double now_seconds() {
  using namespace std::chrono;
  return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

void DevBuf::alloc(lag_ctx *c, size_t nbytes, bool zero) {
  release();
  ctx = c;
  if (nbytes == 0) return;
  if (ctx != nullptr && ctx->budget != 0 && ctx->in_use.load() + nbytes > ctx->budget)
    throw Error(LAG_ENOMEM, "HBM budget exceeded: " + std::to_string(ctx->in_use.load() + nbytes) + " > " +
                                std::to_string(ctx->budget) + " bytes");
  cudaError_t e = cudaMalloc(&ptr, nbytes);
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    throw Error(LAG_ENOMEM, std::string("cudaMalloc(") + std::to_string(nbytes) + "): " + cudaGetErrorString(e));
  }
  bytes = nbytes;
  if (ctx != nullptr) ctx->in_use += nbytes;
  if (zero) LAG_CUDA_CHECK(cudaMemset(ptr, 0, nbytes));
}

void DevBuf::release() {
  if (ptr != nullptr) {
    cudaFree(ptr);
    if (ctx != nullptr) ctx->in_use -= bytes;
  }
  ptr = nullptr;
  bytes = 0;
}

// ------------------------------------------------------------------------------ reduction scratch
void ReduceBuf::ensure(lag_ctx *ctx, int nrhs_, int cap_, int nv_) {
  if (nrhs_ <= nrhs && cap_ <= cap && nv_ <= nv) return;
  nrhs = std::max(nrhs, nrhs_);
  cap = std::max(cap, cap_);
  nv = std::max(nv, nv_);
  part.alloc(ctx, (size_t)nrhs * nv * cap * sizeof(double));
  count.alloc(ctx, (size_t)nrhs * sizeof(unsigned int), true);
}

Reduce ReduceBuf::get() const { return Reduce{part.as<double>(), count.as<unsigned int>(), cap, nv * cap}; }

int stencil_blocks(const lag_grid &g) { return ((g.nx + 31) / 32) * ((g.nz + 7) / 8); }

}  // namespace lag

// ------------------------------------------------------------------------------ preconditioner
void lag_precond::ensure_scratch(int nrhs) {
  if (nrhs <= scratch_rhs) return;
  const size_t per = (size_t)grid.nx * grid.nz;
  scratch.alloc(ctx, per * nrhs * (prec == LAG_FP64 ? sizeof(double) : sizeof(float)));
  if (use_tc) {
    tc_scratch.alloc(ctx, dst_tc_scratch_bytes(dst, nrhs * grid.nz));
    dst.tc_scratch = tc_scratch.as<uint8_t>();
  } else if (dst.oz) {
    tc_scratch.alloc(ctx, dst_oz_scratch_bytes(dst, nrhs * grid.nz), true);  // stream-K counters start at 0
    dst.tc_scratch = tc_scratch.as<uint8_t>();
  }
  scratch_rhs = nrhs;
}

void lag_precond::apply(const double *r, double *z, int nrhs, const KrylovScalars *sc, cudaStream_t s,
                        bool rscale) {
  ensure_scratch(nrhs);
  const int rows = nrhs * grid.nz;
  if (prec == LAG_FP64) {
    double *w = scratch.as<double>();
    dst_apply_f64(dst, r, w, rows, grid.nz, sc, s);
    tri_solve_f64(tri64, w, w, nrhs, sc, s);
    dst_inverse_f64(dst, w, z, rows, grid.nz, sc, s);
  } else {
    float *w = scratch.as<float>();
    if (use_tc) dst_apply_tc_d2f(dst, r, w, rows, grid.nz, sc, s, rscale);
    else dst_apply_f32_d2f(dst, r, w, rows, grid.nz, sc, s, rscale);
    tri_solve_f32(tri32, w, w, nrhs, sc, s);
    if (use_tc) dst_apply_tc_f2d(dst, w, z, rows, grid.nz, sc, s, rscale);
    else dst_inverse_f32_f2d(dst, w, z, rows, grid.nz, sc, s, rscale);
  }
}

lag::TriCoef lag_precond::coef() const {
  lag::TriCoef k;
  k.ax = ax;
  k.az = az;
  k.d = d;
  k.zrows = zrows.ptr ? zrows.as<double>() : nullptr;
  k.free_surface = grid.free_surface != 0;
  k.dct = grid.cylindrical != 0;
  return k;
}

lag_grid lag::kernel_grid(const lag_grid &g) {
  if (g.nx < 1 || g.nz < 1 || !(g.dx > 0) || !(g.dz > 0)) throw Error(LAG_EINVAL, "bad grid");
  if ((g.free_surface != 0 && g.free_surface != 1) || (g.cylindrical != 0 && g.cylindrical != 1))
    throw Error(LAG_EINVAL, "free_surface and cylindrical must be 0 or 1");
  if (!g.cylindrical) return g;
  if (!g.free_surface) throw Error(LAG_EINVAL, "cylindrical grids have a free surface on top: set free_surface = 1");
  lag_grid k{};
  k.nx = g.nz;
  k.nz = g.nx;
  k.dx = g.dz;
  k.dz = g.dx;
  k.free_surface = 0;  // the zero-flux faces are part of the cylindrical coefficients
  k.cylindrical = 1;
  return k;
}

lag_precond *lag::precond_new(lag_ctx *ctx, const lag_grid &gu, double ax, double az, double d, int prec,
                              int partitions, cudaStream_t s, const double *layered, double hoop) {
  const lag_grid g = kernel_grid(gu);
  std::vector<double> zr;
  if (g.cylindrical) {
    // Eq. 21 with the cylindrical coefficients a1 = rbar ax, a2 = r az, d(r) = r d: after the
    // DCT-II along z, per z-mode q the system along r has the rows
    //   (-ax i/dr, ax (2i+1)/dr + r_i az mu_q + r_i d, -ax (i+1)/dr)   (r_i = (i + 1/2) dr)
    // With per-radius rows (the radial variant: coefficients independent of z keep the DCT's
    // separation) ax, az, d come from layered = [ax(r) | az(r) | d(r)], the r faces taking the
    // mean of their two radii (the outer face its radius's value).
    const int nr = g.nz;
    const double dr = g.dz;
    if (!(hoop >= 0) || !std::isfinite(hoop)) throw Error(LAG_EINVAL, "preconditioner coefficients must be positive and finite");
    if (layered == nullptr && (!(ax > 0) || !(az > 0) || !(d >= 0) || !std::isfinite(ax + az + d)))
      throw Error(LAG_EINVAL, "preconditioner coefficients must be positive and finite");
    auto AX = [&](int i) { return layered ? layered[i] : ax; };
    auto AZ = [&](int i) { return layered ? layered[nr + i] : az; };
    auto D = [&](int i) { return layered ? layered[2 * (size_t)nr + i] : d; };
    if (layered)
      for (int i = 0; i < nr; ++i)
        if (!(AX(i) > 0) || !(AZ(i) > 0) || !(D(i) >= 0) || !std::isfinite(AX(i) + AZ(i) + D(i)))
          throw Error(LAG_EINVAL, "per-radius preconditioner coefficients must be positive and finite");
    zr.resize(3 * (size_t)nr + 1);
    zr[0] = 0.0;  // the axis face: rbar = 0
    for (int i = 1; i <= nr; ++i) {  // rbar a_face / dr^2 with rbar = i dr
      const double af = (i < nr) ? 0.5 * (AX(i - 1) + AX(i)) : AX(nr - 1);
      zr[i] = af * (double)i / dr;
    }
    for (int i = 0; i < nr; ++i) {
      const double ri = (i + 0.5) * dr;
      zr[nr + 1 + i] = ri * AZ(i);
      zr[2 * nr + 1 + i] = ri * D(i) + hoop / ri;
    }
  } else if (hoop != 0.0) {
    throw Error(LAG_EINVAL, "the hoop term belongs to cylindrical grids");
  } else if (layered != nullptr) {
    // per-row coefficients -> z faces (mean of the two rows; a boundary face takes its row's value,
    // the top face carries no flux under a free surface), each over dz^2
    const int nz = g.nz;
    const double *lax = layered, *laz = layered + nz, *ld = layered + 2 * nz;
    for (int k = 0; k < nz; ++k)
      if (!(lax[k] > 0) || !(laz[k] > 0) || !(ld[k] >= 0) || !std::isfinite(lax[k] + laz[k] + ld[k]))
        throw Error(LAG_EINVAL, "layered preconditioner coefficients must be positive and finite");
    const double dz2 = g.dz * g.dz;
    zr.resize(3 * (size_t)nz + 1);
    zr[0] = g.free_surface ? 0.0 : laz[0] / dz2;
    for (int k = 1; k < nz; ++k) zr[k] = 0.5 * (laz[k - 1] + laz[k]) / dz2;
    zr[nz] = laz[nz - 1] / dz2;
    for (int k = 0; k < nz; ++k) {
      zr[nz + 1 + k] = lax[k];
      zr[2 * nz + 1 + k] = ld[k];
    }
    ax = az = d = 0.0;
  }
  if (!g.cylindrical && layered == nullptr && (!(ax > 0) || !(az > 0) || !(d >= 0) || !std::isfinite(ax + az + d))) {
    throw Error(LAG_EINVAL, "preconditioner coefficients must be positive and finite");
  }
  if (prec != LAG_FP64 && prec != LAG_MIXED) throw Error(LAG_EINVAL, "prec must be LAG_FP64 or LAG_MIXED");
  std::unique_ptr<lag_precond> p(new lag_precond());
  p->ctx = ctx;
  p->grid = g;
  p->prec = prec;
  p->ax = ax;
  p->az = az;
  p->d = d;
  p->dst_store.ctx = p->tri_store.ctx = p->tri32_store.ctx = p->scratch.ctx = p->tc_scratch.ctx = ctx;
  p->zrows.ctx = ctx;
  p->layered = layered != nullptr;
  const bool gen = !zr.empty();
  if (gen) {
    p->zrows.alloc(ctx, zr.size() * sizeof(double));
    LAG_CUDA_CHECK(cudaMemcpyAsync(p->zrows.ptr, zr.data(), zr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // DCT-II plans share the tensor-core paths: same fold, inverse operands su^T / sv^T = ie / io
  p->use_tc = (prec == LAG_MIXED) && dst_tc_supported(g.nx) && !tc_disabled();
  const bool oz = (prec == LAG_FP64) && dst_oz_supported(g.nx) && !tc_disabled();
  dst_build(p->dst, p->dst_store, g.nx, p->use_tc ? 1 : (oz ? 2 : 0), s, g.cylindrical ? 1 : 0);
  if (p->use_tc || p->dst.oz) {
    p->dst.tc_err = reinterpret_cast<int *>(p->dst_store.as<uint8_t>() + p->dst_store.bytes - 256);
    const char *ev = std::getenv("LAGWAVE_DST_PRODUCTS");  // default split-product count
    if (ev != nullptr && (ev[0] == '1' || ev[0] == '2' || ev[0] == '3') && ev[1] == 0) p->dst.tc_products = ev[0] - '0';
  }
  p->tri64.nx = g.nx;
  p->tri64.nz = g.nz;
  tri_choose_layout(p->tri64, 8, partitions, 0, gen);
  tri_build_factors(p->tri64, p->tri_store, p->coef(), g.dx, g.dz, s, 0);
  if (prec == LAG_MIXED) {
    p->tri32.nx = g.nx;
    p->tri32.nz = g.nz;
    tri_choose_layout(p->tri32, 4, partitions, 0, gen);
    if (p->use_tc) {  // the tensor-core DST leaves the spectrum parity-permuted: permuted factors
      TriFactors tp = p->tri64;
      DevBuf tmp;
      tmp.ctx = ctx;
      tri_build_factors(tp, tmp, p->coef(), g.dx, g.dz, s, p->dst.ku);
      tri_make_f32(tp, p->tri32, p->tri32_store, s);
      LAG_CUDA_CHECK(cudaStreamSynchronize(s));
    } else {
      tri_make_f32(p->tri64, p->tri32, p->tri32_store, s);
    }
  }
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
  return p.release();
}

// ------------------------------------------------------------------------------ medium
void lag_medium::apply(const double *p, double *q, int nrhs, const KrylovScalars *sc, const Reduce *red, int mode,
                       cudaStream_t s, const double *sub) {
  if (elastic) elastic_apply(*this, p, q, nrhs, sc, red, mode, s, sub);
  else if (sub != nullptr) throw Error(LAG_EINVAL, "acoustic operator: no subtrahend");
  else acoustic_apply(*this, p, q, nrhs, sc, red, mode, s);
}

lag_medium *lag::medium_new(lag_ctx *ctx, const lag_grid &gu, const double *c, const double *vs, const double *rho,
                            double h, cudaStream_t s) {
  const lag_grid g = kernel_grid(gu);
  if (c == nullptr || rho == nullptr) throw Error(LAG_EINVAL, "null medium array");
  if (!(h > 0)) throw Error(LAG_EINVAL, "Laguerre h must be positive");
  std::unique_ptr<lag_medium> m(new lag_medium());
  m->ctx = ctx;
  m->grid = g;
  m->h = h;
  m->coef.ctx = m->rho_h2.ctx = m->rowmm.ctx = ctx;
  if (vs == nullptr) {
    m->elastic = false;
    if (g.cylindrical) medium_build_cylindrical(*m, c, rho, s);
    else medium_build_acoustic(*m, c, rho, s);
  } else {
    if (g.cylindrical) {  // the axisymmetric elastic operator (k_elastic_cyl.cu)
      m->elastic = true;
      medium_build_elastic_cylindrical(*m, c, vs, rho, s);
      return m.release();
    }
    if (g.free_surface)
      throw Error(LAG_EINVAL, "free_surface applies to acoustic media only (the elastic traction-free surface is not built)");
    m->elastic = true;
    medium_build_elastic(*m, c, vs, rho, s);
  }
  return m.release();
}

// ------------------------------------------------------------------------------ C ABI helpers
static thread_local std::string g_tls_error;

template <typename F>
static int guarded(lag_ctx *ctx, F &&f) {
  try {
    f();
    return LAG_OK;
  } catch (const Error &e) {
    if (ctx) ctx->last_error = e.what();
    g_tls_error = e.what();
    return e.status;
  } catch (const std::bad_alloc &) {
    if (ctx) ctx->last_error = "host allocation failed";
    return LAG_ENOMEM;
  } catch (const std::exception &e) {
    if (ctx) ctx->last_error = e.what();
    g_tls_error = e.what();
    return LAG_ECUDA;
  }
}

static void set_device(lag_ctx *ctx) { LAG_CUDA_CHECK(cudaSetDevice(ctx->device)); }

extern "C" {

const char *lag_strerror(int status) {
  switch (status) {
    case LAG_OK: return "ok";
    case LAG_EINVAL: return "invalid argument";
    case LAG_ENOMEM: return "out of device memory or HBM budget";
    case LAG_ENOTCONV: return "Krylov solve did not converge within max_iter";
    case LAG_ENUMERIC: return "NaN or Inf in a residual";
    case LAG_ECUDA: return "CUDA error";
    case LAG_EAGAIN: return "not finished yet";
    case LAG_ETIMEDOUT: return "bounded device wait timed out";
    case LAG_ECANCELED: return "cancelled";
    default: return "unknown status";
  }
}

const char *lag_last_error(const lag_ctx *ctx) { return ctx ? ctx->last_error.c_str() : g_tls_error.c_str(); }
int lag_version(void) { return 100; }

int lag_create(lag_ctx **out, int device, size_t budget, void *stream) {
  if (out == nullptr) return LAG_EINVAL;
  *out = nullptr;
  return guarded(nullptr, [&] {
    int ndev = 0;
    LAG_CUDA_CHECK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) throw Error(LAG_EINVAL, "no such CUDA device");
    std::unique_ptr<lag_ctx> c(new lag_ctx());
    c->device = device;
    c->budget = budget;
    c->t_created = now_seconds();
    LAG_CUDA_CHECK(cudaSetDevice(device));
    if (stream != nullptr) {
      c->stream = static_cast<cudaStream_t>(stream);
    } else {
      LAG_CUDA_CHECK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    *out = c.release();
  });
}

void lag_destroy(lag_ctx *ctx) {
  if (ctx == nullptr) return;
  server_destroy(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->own_stream && ctx->stream) {
    cudaStreamSynchronize(ctx->stream);
    cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
}

int lag_synchronize(lag_ctx *ctx) {
  if (!ctx) return LAG_EINVAL;
  return guarded(ctx, [&] { LAG_CUDA_CHECK(cudaStreamSynchronize(ctx->stream)); });
}

size_t lag_bytes_in_use(const lag_ctx *ctx) { return ctx ? ctx->in_use.load() : 0; }
long long lag_kernel_launches(const lag_ctx *) { return (long long)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// ------------------------------------------------------------------------------ preconditioner
int lag_precond_create(lag_ctx *ctx, const lag_grid *grid, double kappa_t, double rho_t, double h_lag, int prec,
                       lag_precond **out) {
  if (!ctx || !grid || !out) return LAG_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    set_device(ctx);
    *out = precond_new(ctx, *grid, kappa_t, kappa_t, rho_t * h_lag * h_lag / 4.0, prec, 0, ctx->stream);
  });
}

int lag_precond_create_sep(lag_ctx *ctx, const lag_grid *grid, double ax, double az, double d, int prec,
                           int partitions, lag_precond **out) {
  if (!ctx || !grid || !out) return LAG_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    set_device(ctx);
    if (partitions < 0 || partitions > 32) throw Error(LAG_EINVAL, "partitions must be 0..32");
    *out = precond_new(ctx, *grid, ax, az, d, prec, partitions, ctx->stream);
  });
}

int lag_precond_create_layered(lag_ctx *ctx, const lag_grid *grid, const double *ax_z, const double *az_z,
                               const double *d_z, int prec, int partitions, lag_precond **out) {
  if (!ctx || !grid || !out || !ax_z || !az_z || !d_z) return LAG_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    set_device(ctx);
    if (partitions < 0 || partitions > 32) throw Error(LAG_EINVAL, "partitions must be 0..32");
    // rows: depths of a Cartesian grid, radii (grid->nx) of a cylindrical one
    const int nrow = grid->cylindrical ? grid->nx : grid->nz;
    if (nrow < 1) throw Error(LAG_EINVAL, "bad grid");
    std::vector<double> rows(3 * (size_t)nrow);
    std::copy(ax_z, ax_z + nrow, rows.begin());
    std::copy(az_z, az_z + nrow, rows.begin() + nrow);
    std::copy(d_z, d_z + nrow, rows.begin() + 2 * (size_t)nrow);
    *out = precond_new(ctx, *grid, 0.0, 0.0, 0.0, prec, partitions, ctx->stream, rows.data());
  });
}

int lag_precond_create_cyl(lag_ctx *ctx, const lag_grid *grid, double ax_t, double az_t, double d_t, double hoop_t,
                           int prec, int partitions, lag_precond **out) {
  if (!ctx || !grid || !out) return LAG_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    set_device(ctx);
    if (!grid->cylindrical) throw Error(LAG_EINVAL, "lag_precond_create_cyl needs a cylindrical grid");
    if (partitions < 0 || partitions > 32) throw Error(LAG_EINVAL, "partitions must be 0..32");
    *out = precond_new(ctx, *grid, ax_t, az_t, d_t, prec, partitions, ctx->stream, nullptr, hoop_t);
  });
}

int lag_precond_is_layered(const lag_precond *p) { return (p && p->layered) ? 1 : 0; }

void lag_precond_destroy(lag_precond *p) {
  if (!p) return;
  cudaSetDevice(p->ctx->device);
  cudaStreamSynchronize(p->ctx->stream);
  delete p;
}

int lag_precond_status(lag_precond *p) {
  if (!p) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    LAG_CUDA_CHECK(cudaStreamSynchronize(p->ctx->stream));
    if (!(p->use_tc || p->dst.oz) || p->dst.tc_err == nullptr) return;
    int h = 0;
    LAG_CUDA_CHECK(cudaMemcpy(&h, p->dst.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0)
      throw Error(LAG_ETIMEDOUT, "tensor-core DST: a bounded pipeline wait gave up (code " + std::to_string(h) +
                                     ": 1-4 split-bf16 GEMM, 11-14 exact-slice GEMM, 21-24 its two-SM pairs, "
                                     "31-36 its stream-K variant)");
  });
}

int lag_precond_apply(lag_precond *p, const double *r, double *z, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!r || !z))) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    if (nrhs == 0) return;
    p->apply(r, z, nrhs, nullptr, p->ctx->stream);
  });
}

int lag_precond_dst(lag_precond *p, const double *x, double *y, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!x || !y))) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    if (nrhs == 0) return;
    const int rows = nrhs * p->grid.nz;
    if (p->prec == LAG_FP64) {
      p->ensure_scratch(nrhs);
      dst_apply_f64(p->dst, x, y, rows, p->grid.nz, nullptr, p->ctx->stream);
    } else {  // float64 -> float32 spectrum -> float64 (both mixed-path kernels, back to back)
      p->ensure_scratch(nrhs);
      float *w = p->scratch.as<float>();
      if (p->use_tc) {
        dst_apply_tc_d2f(p->dst, x, w, rows, p->grid.nz, nullptr, p->ctx->stream);
        spectrum_unpermute_widen(w, y, rows, p->grid.nx, p->dst.ku, p->ctx->stream);
      } else {
        dst_apply_f32_d2f(p->dst, x, w, rows, p->grid.nz, nullptr, p->ctx->stream);
        widen_f32(w, y, (size_t)rows * p->grid.nx, p->ctx->stream);
      }
    }
  });
}

int lag_precond_dst_inverse(lag_precond *p, const double *x, double *y, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!x || !y)) || p->prec != LAG_FP64) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    if (nrhs == 0) return;
    p->ensure_scratch(nrhs);
    dst_inverse_f64(p->dst, x, y, nrhs * p->grid.nz, p->grid.nz, nullptr, p->ctx->stream);
  });
}

int lag_precond_dst_f32(lag_precond *p, const float *x, double *y, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!x || !y)) || p->prec != LAG_MIXED) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    if (nrhs == 0) return;
    const int rows = nrhs * p->grid.nz;
    if (p->use_tc) {  // the tensor-core inverse reads a parity-permuted spectrum
      p->ensure_scratch(nrhs);
      float *w = p->scratch.as<float>();
      spectrum_permute(x, w, rows, p->grid.nx, p->dst.ku, true, p->ctx->stream);
      dst_apply_tc_f2d(p->dst, w, y, rows, p->grid.nz, nullptr, p->ctx->stream);
    } else {
      dst_apply_f32_f2d(p->dst, x, y, rows, p->grid.nz, nullptr, p->ctx->stream);
    }
  });
}

int lag_precond_tridiag(lag_precond *p, const double *d, double *y, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!d || !y))) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    if (nrhs > 0) tri_solve_f64(p->tri64, d, y, nrhs, nullptr, p->ctx->stream);
  });
}

int lag_precond_tridiag_f32(lag_precond *p, const float *d, float *y, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!d || !y)) || p->prec != LAG_MIXED) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    if (nrhs == 0) return;
    if (p->use_tc) {  // factors are stored for parity-permuted spectra
      p->ensure_scratch(nrhs);
      float *w = p->scratch.as<float>();
      const int rows = nrhs * p->grid.nz;
      spectrum_permute(d, w, rows, p->grid.nx, p->dst.ku, true, p->ctx->stream);
      tri_solve_f32(p->tri32, w, w, nrhs, nullptr, p->ctx->stream);
      spectrum_permute(w, y, rows, p->grid.nx, p->dst.ku, false, p->ctx->stream);
    } else {
      tri_solve_f32(p->tri32, d, y, nrhs, nullptr, p->ctx->stream);
    }
  });
}

int lag_precond_info(const lag_precond *p, int *P, int *L, int *mt) {
  if (!p) return LAG_EINVAL;
  const TriFactors &t = (p->prec == LAG_FP64) ? p->tri64 : p->tri32;
  if (P) *P = t.P;
  if (L) *L = t.L;
  if (mt) *mt = t.mt;
  return LAG_OK;
}

int lag_dst_f64_slice_products(int n) {
  if (!dst_oz_supported(n)) return 0;
  return dst_oz_products(n);
}

int lag_precond_uses_tensor_cores(const lag_precond *p) { return p ? ((p->use_tc || p->dst.oz) ? 1 : 0) : 0; }

int lag_precond_dst_gemm(lag_precond *p, int nrhs) {
  if (!p || nrhs < 1) return LAG_EINVAL;
  if (p->use_tc) return LAG_GEMM_SPLIT_BF16;
  if (!p->dst.oz) return LAG_GEMM_SIMT;
  int v = LAG_GEMM_SLICE_TILES;
  const int rc = guarded(p->ctx, [&] {
    set_device(p->ctx);
    v = dst_oz_gemm_variant(p->dst, nrhs * p->grid.nz, p->grid.nz, 0);
  });
  return rc == LAG_OK ? v : rc;
}

int lag_precond_set_layout(lag_precond *p, int partitions, int modes_per_cta) {
  if (!p || partitions < 0 || partitions > 32 || modes_per_cta < 0) return LAG_EINVAL;
  return guarded(p->ctx, [&] {
    set_device(p->ctx);
    const int eb = (p->prec == LAG_FP64) ? 8 : 4;
    TriFactors probe;
    probe.nx = p->grid.nx;
    probe.nz = p->grid.nz;
    tri_choose_layout(probe, eb, partitions, 0);
    if (modes_per_cta != 0 && (!probe.reg || !tri_mode_tile_ok(eb, probe.L, modes_per_cta)))
      throw Error(LAG_EINVAL, "mode tile not available for this layout (float32: 8, 16, 32 (L <= 32); "
                              "float64: 4, 8; register kernel only)");
    LAG_CUDA_CHECK(cudaStreamSynchronize(p->ctx->stream));
    precond_rebuild_tri(p, partitions, modes_per_cta, p->ctx->stream);
  });
}

int lag_precond_set_dst_products(lag_precond *p, int products) {
  if (!p || products < 1 || products > 3) return LAG_EINVAL;
  if (!p->use_tc) return products == 3 ? LAG_OK : LAG_EINVAL;
  p->dst.tc_products = products;
  return LAG_OK;
}

// ------------------------------------------------------------------------------ medium
int lag_medium_create_acoustic(lag_ctx *ctx, const lag_grid *g, const double *c, const double *rho, double h,
                               lag_medium **out) {
  if (!ctx || !g || !out) return LAG_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    set_device(ctx);
    *out = medium_new(ctx, *g, c, nullptr, rho, h, ctx->stream);
  });
}

int lag_medium_create_elastic(lag_ctx *ctx, const lag_grid *g, const double *vp, const double *vs,
                              const double *rho, double h, lag_medium **out) {
  if (!ctx || !g || !out || !vs) return LAG_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    set_device(ctx);
    *out = medium_new(ctx, *g, vp, vs, rho, h, ctx->stream);
  });
}

void lag_medium_destroy(lag_medium *m) {
  if (!m) return;
  cudaSetDevice(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  delete m;
}

int lag_medium_midranges(lag_medium *m, double *out) {
  if (!m || !out) return LAG_EINVAL;
  out[0] = m->mid[0];
  out[1] = m->mid[1];
  if (m->elastic) out[2] = m->mid[2];
  return LAG_OK;
}

int lag_apply_operator(lag_medium *m, const double *p, double *q, int nrhs) {
  if (!m || nrhs < 0 || (nrhs > 0 && (!p || !q))) return LAG_EINVAL;
  return guarded(m->ctx, [&] {
    set_device(m->ctx);
    if (nrhs > 0) m->apply(p, q, nrhs, nullptr, nullptr, 0, m->ctx->stream);
  });
}

// ------------------------------------------------------------------------------ one system
int lag_solve_system(lag_medium *m, lag_precond *p1, lag_precond *p2, const double *b, double *x, int nrhs,
                     const lag_solver *s, int *iters, double *relres) {
  if (!m || !p1 || !s || nrhs < 0 || (nrhs > 0 && (!b || !x))) return LAG_EINVAL;
  int status = LAG_OK;
  int rc = guarded(m->ctx, [&] {
    set_device(m->ctx);
    if (nrhs == 0) return;
    check_solver(*s, m->elastic);
    if (p1->grid.nx != m->grid.nx || p1->grid.nz != m->grid.nz) throw Error(LAG_EINVAL, "plan/medium grid mismatch");
    if (p1->prec != s->prec) throw Error(LAG_EINVAL, "plan precision differs from solver precision");
    if (m->elastic && (!p2 || p2->prec != s->prec || p2->grid.nx != m->grid.nx || p2->grid.nz != m->grid.nz))
      throw Error(LAG_EINVAL, "elastic solve needs a second matching plan (B2)");
    KrylovWork wk;
    wk.setup(m->ctx, m, p1, p2, *s, nrhs, m->ctx->stream);
    LAG_CUDA_CHECK(cudaMemcpyAsync(wk.b(), b, wk.n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, m->ctx->stream));
    status = wk.solve_blocking();
    wk.copy_result(x);
    wk.report(iters, relres);
  });
  return rc != LAG_OK ? rc : status;
}

// ------------------------------------------------------------------------------ Laguerre pieces
int lag_source_coeffs(lag_ctx *ctx, const lag_laguerre *lag, const lag_wavelet *w, double *fm_host) {
  if (!ctx || !lag || !w || !fm_host || lag->n_harm < 1 || lag->alpha < 0 || !(lag->h > 0) || !(w->f0 > 0))
    return LAG_EINVAL;
  return guarded(ctx, [&] {
    set_device(ctx);
    DevBuf fm, scratch;
    fm.alloc(ctx, lag->n_harm * sizeof(double));
    source_coeffs_device(*lag, *w, fm.as<double>(), scratch, ctx, ctx->stream);
    LAG_CUDA_CHECK(cudaMemcpyAsync(fm_host, fm.ptr, lag->n_harm * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LAG_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  });
}

int lag_laguerre_table(lag_ctx *ctx, const lag_laguerre *lag, int nt, const double *t_host, double *tab_host) {
  if (!ctx || !lag || nt < 0 || (nt > 0 && (!t_host || !tab_host)) || lag->n_harm < 1 || !(lag->h > 0))
    return LAG_EINVAL;
  return guarded(ctx, [&] {
    set_device(ctx);
    if (nt == 0) return;
    DevBuf t, tab;
    t.alloc(ctx, nt * sizeof(double));
    tab.alloc(ctx, (size_t)nt * lag->n_harm * sizeof(double));
    LAG_CUDA_CHECK(cudaMemcpyAsync(t.ptr, t_host, nt * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    laguerre_table_device(*lag, nt, t.as<double>(), tab.as<double>(), ctx->stream);
    LAG_CUDA_CHECK(cudaMemcpyAsync(tab_host, tab.ptr, (size_t)nt * lag->n_harm * sizeof(double),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    LAG_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  });
}

}  // extern "C"
