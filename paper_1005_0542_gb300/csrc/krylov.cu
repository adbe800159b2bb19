// Krylov drivers: preconditioned CG (acoustic) and right-preconditioned flexible GMRES(k)
// (elastic), Sec. 2.3.  Every scalar stays on the device; the host enqueues chunks of iterations
// and looks at a pinned copy of the per-system state between chunks.  Systems that have
// converged are skipped by every kernel, so a chunk that overshoots costs only launches.
#include <cstdlib>
#include <cstring>

#include "solver.h"

namespace lag {

bool tc_disabled() {
  // kernel selection for the mixed path's DST: "simt" forces the float32 SIMT kernel
  const char *v = std::getenv("LAGWAVE_DST_KERNEL");
  return v != nullptr && std::strcmp(v, "simt") == 0;
}

__global__ void widen_kernel(const float *a, double *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

void widen_f32(const float *a, double *b, size_t n, cudaStream_t s) {
  widen_kernel<<<1024, 256, 0, s>>>(a, b, n);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void check_solver(const lag_solver &s, bool elastic) {
  if (!(s.tol > 0) || !(s.tol < 1)) throw Error(LAG_EINVAL, "tol must be in (0, 1)");
  if (s.max_iter < 1) throw Error(LAG_EINVAL, "max_iter must be >= 1");
  if (s.prec != LAG_FP64 && s.prec != LAG_MIXED) throw Error(LAG_EINVAL, "prec must be LAG_FP64 or LAG_MIXED");
  if (elastic && (s.restart_k < 1 || s.restart_k > 64)) throw Error(LAG_EINVAL, "restart_k must be 1..64");
  if (s.partitions < 0 || s.partitions > 32) throw Error(LAG_EINVAL, "partitions must be 0..32");
  if (s.tune != 0 && s.tune != 1) throw Error(LAG_EINVAL, "tune must be 0 or 1");
  if (s.layered != 0 && s.layered != 1) throw Error(LAG_EINVAL, "layered must be 0 or 1");
}

void precond_apply_multi(lag_precond *p1, lag_precond *p2, const double *r, double *z, int nrhs, int ncomp,
                         const KrylovScalars *sc, cudaStream_t s) {
  if (ncomp == 1) {  // PCG: r is the residual whose norm sc[b].rr holds
    p1->apply(r, z, nrhs, sc, s, true);
    return;
  }
  // two components share the DST (same nx); the tridiagonal factors differ per component
  const int planes = nrhs * ncomp;
  p1->ensure_scratch(planes);
  const int rows = planes * p1->grid.nz;
  const int rpr = p1->grid.nz * ncomp;
  if (p1->prec == LAG_FP64) {
    double *w = p1->scratch.as<double>();
    dst_apply_f64(p1->dst, r, w, rows, rpr, sc, s);
    tri_solve_f64(p1->tri64, w, w, nrhs, sc, s, ncomp, 0, ncomp);
    tri_solve_f64(p2->tri64, w, w, nrhs, sc, s, ncomp, 1, ncomp);
    dst_inverse_f64(p1->dst, w, z, rows, rpr, sc, s);
  } else {
    float *w = p1->scratch.as<float>();
    if (p1->use_tc) dst_apply_tc_d2f(p1->dst, r, w, rows, rpr, sc, s);
    else dst_apply_f32_d2f(p1->dst, r, w, rows, rpr, sc, s);
    tri_solve_f32(p1->tri32, w, w, nrhs, sc, s, ncomp, 0, ncomp);
    tri_solve_f32(p2->tri32, w, w, nrhs, sc, s, ncomp, 1, ncomp);
    if (p1->use_tc) dst_apply_tc_f2d(p1->dst, w, z, rows, rpr, sc, s);
    else dst_inverse_f32_f2d(p1->dst, w, z, rows, rpr, sc, s);
  }
}

KrylovWork::~KrylovWork() {
  if (hsc) cudaFreeHost(hsc);
  for (auto &g : gexec)
    if (g) cudaGraphExecDestroy(g);
  if (ev) cudaEventDestroy(ev);
}

void KrylovWork::setup(lag_ctx *c, lag_medium *med, lag_precond *q1, lag_precond *q2, const lag_solver &sol,
                       int nr, cudaStream_t st) {
  for (auto &g : gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  eager_done = false;
  ctx = c;
  m = med;
  p1 = q1;
  p2 = q2;
  s = sol;
  nrhs = nr;
  stream = st;
  elastic = med->elastic;
  ncomp = elastic ? 2 : 1;
  nplane = (size_t)med->grid.nx * med->grid.nz;
  n = nplane * ncomp;
  vecs.ctx = scal.ctx = gm.ctx = red.part.ctx = red.count.ctx = ctx;
  const int nvec = elastic ? (3 + (s.restart_k + 1) + s.restart_k) : 6;
  vecs.alloc(ctx, (size_t)nvec * n * nrhs * sizeof(double));
  scal.alloc(ctx, (size_t)nrhs * sizeof(KrylovScalars), true);
  const int cap = std::max(std::max(reduce_blocks(n), stencil_blocks(med->grid)), 1);
  red.ensure(ctx, nrhs, cap, elastic ? s.restart_k + 1 : 2);
  if (elastic) {
    gk = s.restart_k;
    const int k = gk;
    const size_t per = (size_t)(k + 1) * k + k + k + (k + 1) + k + (k + 1);
    gm.alloc(ctx, per * nrhs * sizeof(double), true);
    double *g0 = gm.as<double>();
    gdev.k = k;
    gdev.H = g0;
    gdev.cs = gdev.H + (size_t)nrhs * (k + 1) * k;
    gdev.sn = gdev.cs + (size_t)nrhs * k;
    gdev.g = gdev.sn + (size_t)nrhs * k;
    gdev.y = gdev.g + (size_t)nrhs * (k + 1);
    gdev.hcol = gdev.y + (size_t)nrhs * k;
  }
  // pinned mirror: the scalars, then the error words of the two plans' tensor-core kernels
  LAG_CUDA_CHECK(cudaMallocHost(&hsc, (size_t)nrhs * sizeof(KrylovScalars) + 2 * sizeof(int)));
  std::memset(hsc, 0, (size_t)nrhs * sizeof(KrylovScalars) + 2 * sizeof(int));
  LAG_CUDA_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
}

void KrylovWork::precond(const double *rr, double *zz) { precond_apply_multi(p1, p2, rr, zz, nrhs, ncomp, sc(), stream); }

void KrylovWork::start_from_b() {
  if (elastic) {
    LAG_CUDA_CHECK(cudaMemsetAsync(x(), 0, n * nrhs * sizeof(double), stream));
    gmres_begin_cycle(true);
    return;
  }
  pcg_start(b(), x(), r(), n, nrhs, s.tol, sc(), red.get(), stream);
  start_from_r();
}

void KrylovWork::start_from_r() {
  iters_this_solve = 0;
  chunk = 2;
  if (elastic) {
    // r holds the right-hand side: copy it to b, x = 0 (set by the right-hand side kernel)
    LAG_CUDA_CHECK(cudaMemcpyAsync(b(), r(), n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    gmres_begin_cycle(true);
    return;
  }
  double *z = vec(5), *p = vec(3);
  precond(r(), z);
  pcg_rz_p(r(), z, p, n, nrhs, sc(), red.get(), stream);
}

void KrylovWork::pcg_iteration() {
  double *p = vec(3), *q = vec(4), *z = vec(5);
  Reduce rd = red.get();
  const int flexible = s.prec == LAG_MIXED ? 1 : 0;
  m->apply(p, q, nrhs, sc(), &rd, 1, stream);                        // q = A p, alpha
  pcg_update_xr(x(), r(), p, q, n, nrhs, s.max_iter, sc(), rd, stream);  // x, r, ||r||, state
  if (p1->use_tc) {
    // mixed path: forward DST, tridiagonal solve, then the inverse DST whose butterfly also forms
    // (r, z), (z, q) and beta
    const int rows = nrhs * p1->grid.nz;
    p1->ensure_scratch(nrhs);
    float *w = p1->scratch.as<float>();
    dst_apply_tc_d2f(p1->dst, r(), w, rows, p1->grid.nz, sc(), stream, true);
    tri_solve_f32(p1->tri32, w, w, nrhs, sc(), stream);
    dst_apply_tc_f2d_beta(p1->dst, w, z, nrhs, p1->grid.nz, r(), q, flexible, sc(), rd, stream);
  } else {
    precond(r(), z);                                                 // z = B^{-1} r
    pcg_beta(r(), z, q, n, nrhs, flexible, sc(), rd, stream);
  }
  pcg_update_p(p, z, n, nrhs, sc(), stream);                         // p = z + beta p
}

static bool graphs_disabled() {
  const char *e = std::getenv("LAGWAVE_GRAPHS");
  return e != nullptr && e[0] == '0';
}

void KrylovWork::pcg_chunk(int iters) {
  int idx = 0;
  while ((1 << idx) < iters && idx < 4) ++idx;
  // the first chunk runs eagerly: it also performs the one-time kernel attribute setup, which
  // must not happen inside a capture
  // (the legacy default stream cannot be captured)
  const bool capturable = stream != nullptr && stream != cudaStreamLegacy && stream != cudaStreamPerThread;
  if (!eager_done || (1 << idx) != iters || !capturable || profiling_on() || graphs_disabled()) {
    for (int i = 0; i < iters; ++i) pcg_iteration();
    eager_done = true;
    return;
  }
  p1->ensure_scratch(nrhs);
  const void *key[3] = {p1->scratch.ptr, p1->tc_scratch.ptr, vecs.ptr};
  const int prod = p1->dst.tc_products;
  if (gexec[idx] != nullptr && (std::memcmp(key, gkey[idx], sizeof(key)) != 0 || prod != gprod[idx])) {
    cudaGraphExecDestroy(gexec[idx]);
    gexec[idx] = nullptr;
  }
  if (gexec[idx] == nullptr) {
    cudaGraph_t g = nullptr;
    LAG_CUDA_CHECK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      for (int i = 0; i < iters; ++i) pcg_iteration();
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    g_capturing = false;
    LAG_CUDA_CHECK(cudaStreamEndCapture(stream, &g));
    size_t nodes = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nodes);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec[idx], g, 0);
    cudaGraphDestroy(g);
    LAG_CUDA_CHECK(e);
    gnodes[idx] = nodes;
    std::memcpy(gkey[idx], key, sizeof(key));
    gprod[idx] = prod;
  }
  LAG_CUDA_CHECK(cudaGraphLaunch(gexec[idx], stream));
  count_launch((int)gnodes[idx]);
}

void KrylovWork::enqueue_chunk() {
  if (!elastic) {
    pcg_chunk(chunk);
    iters_this_solve += chunk;
  } else {
    for (int i = 0; i < chunk; ++i) {
      if (!cycle_open) gmres_begin_cycle(false);
      gmres_step();
      if (gj >= gk) gmres_end_cycle();
    }
    iters_this_solve += chunk;
  }
  mirror_state();
  if (chunk < 16) chunk *= 2;
}

void KrylovWork::mirror_state() {
  LAG_CUDA_CHECK(cudaMemcpyAsync(hsc, sc(), (size_t)nrhs * sizeof(KrylovScalars), cudaMemcpyDeviceToHost, stream));
  int *herr = reinterpret_cast<int *>(hsc + nrhs);
  const lag_precond *pl[2] = {p1, p2};
  for (int i = 0; i < 2; ++i)
    if (pl[i] != nullptr && (pl[i]->use_tc || pl[i]->dst.oz) && pl[i]->dst.tc_err != nullptr)
      LAG_CUDA_CHECK(cudaMemcpyAsync(herr + i, pl[i]->dst.tc_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  LAG_CUDA_CHECK(cudaEventRecord(ev, stream));
  pending = true;
}

int KrylovWork::poll(bool block) {
  if (pending) {
    if (block) {
      LAG_CUDA_CHECK(cudaEventSynchronize(ev));
    } else {
      cudaError_t e = cudaEventQuery(ev);
      if (e == cudaErrorNotReady) return -1;
      LAG_CUDA_CHECK(e);
    }
    pending = false;
    const int *herr = reinterpret_cast<const int *>(hsc + nrhs);
    if (herr[0] != 0 || herr[1] != 0)
      throw Error(LAG_ETIMEDOUT, "tensor-core DST: a bounded pipeline wait gave up (code " +
                                     std::to_string(herr[0] ? herr[0] : herr[1]) + "); the preconditioner output is invalid");
  }
  bool any_run = false, any_met = false;
  for (int i = 0; i < nrhs; ++i) {
    if (hsc[i].state == ST_RUN) any_run = true;
    if (hsc[i].state == ST_MET) any_met = true;
  }
  if (any_run) return 0;
  if (!elastic) return 1;
  if (any_met) {
    // every open system met the tolerance estimate inside the cycle: close it (x += Z y) and
    // recheck the true residual; after the recheck no system is left in ST_MET
    if (cycle_open) gmres_end_cycle();
    gmres_begin_cycle(false);
    mirror_state();
    return poll(block);
  }
  cycle_open = false;  // systems stop only at a cycle start: no update is pending
  return 1;
}

int KrylovWork::finish_status() const {
  int st = LAG_OK;
  for (int i = 0; i < nrhs; ++i) {
    if (hsc[i].state == ST_NAN) return LAG_ENUMERIC;
    if (hsc[i].state == ST_STOP) st = LAG_ENOTCONV;
  }
  return st;
}

int KrylovWork::solve_blocking() {
  start_from_b();
  for (;;) {
    enqueue_chunk();
    if (poll(true) == 1) break;
  }
  if (elastic && cycle_open) gmres_end_cycle();
  LAG_CUDA_CHECK(cudaStreamSynchronize(stream));
  return finish_status();
}

void KrylovWork::copy_result(double *x_out) {
  LAG_CUDA_CHECK(cudaMemcpyAsync(x_out, x(), n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  LAG_CUDA_CHECK(cudaStreamSynchronize(stream));
}

void KrylovWork::report(int *iters, double *relres) const {
  for (int i = 0; i < nrhs; ++i) {
    if (iters) iters[i] = hsc[i].iters;
    if (relres) relres[i] = hsc[i].bb > 0 ? std::sqrt(hsc[i].rr / hsc[i].bb) : 0.0;
  }
}

// ------------------------------------------------------------------------------ FGMRES driver
// Cycle: r = b - C x, beta = ||r||, V_0 = r / beta, g = beta e_1; step j: Z_j = K^{-1} V_j,
// w = C Z_j, two classical Gram-Schmidt passes against V_0..V_j (the second one re-orthogonalises),
// h_{j+1,j} = ||w||, V_{j+1} = w / h_{j+1,j}, Givens rotation of the new column and of g; end:
// y = H^{-1} g (upper triangular), x += Z y.  State 4 marks a system whose residual estimate met
// the tolerance inside the open cycle; the true residual at the next cycle start decides.
void KrylovWork::gmres_begin_cycle(bool first) {
  double *w = r();
  double *V0 = vec(3);
  Reduce rd = red.get();
  if (!first) m->apply(x(), w, nrhs, sc(), nullptr, 2, stream);  // w = C x for systems still open
  gm_start(b(), w, V0, n, nrhs, first ? 1 : 0, s.tol, s.max_iter, sc(), gdev, rd, stream);
  gj = 0;
  cycle_open = true;
}

void KrylovWork::gmres_step() {
  const int k = gk, j = gj;
  double *V = vec(3), *Z = vec(3 + k + 1), *w = r();
  const size_t vs = n * (size_t)nrhs;
  Reduce rd = red.get();
  precond(V + (size_t)j * vs, Z + (size_t)j * vs);               // Z_j = K^{-1} V_j
  // shifted Arnoldi step: w = C Z_j - V_j spans the same Krylov space (C K^{-1} - I has the
  // Hessenberg matrix H - I), but for a good preconditioner C K^{-1} V_j lies close to V_j and the
  // shift removes that component before the projections, so the first Gram-Schmidt pass cancels
  // less and the second one (selective) is often skipped
  m->apply(Z + (size_t)j * vs, w, nrhs, sc(), nullptr, 0, stream, V + (size_t)j * vs);
  gm_orthogonalize(w, V, j, n, nrhs, vs, sc(), gdev, rd, 0, true, stream);
  gm_orthogonalize(w, V, j, n, nrhs, vs, sc(), gdev, rd, 1, true, stream);
  gm_normalize(w, V + (size_t)(j + 1) * vs, j, n, nrhs, sc(), gdev, rd, s.max_iter, stream);
  gj = j + 1;
}

void KrylovWork::gmres_end_cycle() {
  const int k = gk;
  double *Z = vec(3 + k + 1);
  gm_update_x(x(), Z, gj, n, nrhs, n * (size_t)nrhs, sc(), gdev, stream);
  cycle_open = false;
}

}  // namespace lag
