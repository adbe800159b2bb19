// Krylov drivers: preconditioned CG (acoustic) and right-preconditioned flexible GMRES(k)
// (elastic), Sec. 2.3.  Every scalar stays on the device.  PCG runs as one CUDA graph per solve
// whose conditional WHILE node repeats the iterations until every system has stopped (eager chunks
// of iterations where a graph cannot be used); GMRES is enqueued in chunks of steps.  The host looks
// at a pinned copy of the per-system state after each launch.  Systems that have converged are
// skipped by every kernel, so iterations past a system's convergence cost only launches.
#include <algorithm>
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
  if (wexec) cudaGraphExecDestroy(wexec);
  if (ev) cudaEventDestroy(ev);
}

void KrylovWork::setup(lag_ctx *c, lag_medium *med, lag_precond *q1, lag_precond *q2, const lag_solver &sol,
                       int nr, cudaStream_t st) {
  if (wexec) {
    cudaGraphExecDestroy(wexec);
    wexec = nullptr;
  }
  eager_done = false;
  pcur = 0;
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
  vecs.ctx = scal.ctx = gm.ctx = red.part.ctx = red.count.ctx = wcount.ctx = ctx;
  const int nvec = elastic ? (3 + (s.restart_k + 1) + s.restart_k) : 7;
  vecs.alloc(ctx, (size_t)nvec * n * nrhs * sizeof(double));
  scal.alloc(ctx, (size_t)nrhs * sizeof(KrylovScalars), true);
  // blocks per right-hand side of the reductions: the vector kernels, the stencil, and the float64
  // tridiagonal solve that also forms (r, z) (one CTA per 4 modes at most)
  const int cap = std::max(std::max(std::max(reduce_blocks(n), stencil_blocks(med->grid)), 1),
                           elastic ? 1 : (med->grid.nx + 3) / 4);
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
  if (!elastic) {
    wcount.alloc(ctx, 4 * sizeof(unsigned int), true);  // [0] repeats this launch, [2..3] bodies in total
    wbodies_seen = 0;
  }
  // pinned mirror: the scalars, the error words of the two plans' tensor-core kernels, then the
  // PCG graph's body count
  if (hsc) cudaFreeHost(hsc);
  hsc = nullptr;
  const size_t mbytes = (size_t)nrhs * sizeof(KrylovScalars) + 2 * sizeof(int) + sizeof(unsigned long long);
  LAG_CUDA_CHECK(cudaMallocHost(&hsc, mbytes));
  std::memset(hsc, 0, mbytes);
  LAG_CUDA_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
}

void KrylovWork::precond(const double *rr, double *zz) { precond_apply_multi(p1, p2, rr, zz, nrhs, ncomp, sc(), stream); }

void KrylovWork::start_from_b() {
  if (elastic) {
    LAG_CUDA_CHECK(cudaMemsetAsync(x(), 0, n * nrhs * sizeof(double), stream));
    gmres_begin_cycle(true);
    return;
  }
  pcg_start(b(), x(), r(), vec(3), n, nrhs, s.tol, sc(), red.get(), stream);
  start_from_r();
}

void KrylovWork::start_from_r() {
  iters_this_solve = 0;
  // an even count (the PCG graph's body starts from the first direction buffer), one below the
  // previous solve's
  predicted_first = predict > 3;
  chunk = predicted_first ? (predict - 1) & ~1 : 2;
  if (elastic) {
    // r holds the right-hand side: copy it to b, x = 0 (set by the right-hand side kernel)
    LAG_CUDA_CHECK(cudaMemcpyAsync(b(), r(), n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    gmres_begin_cycle(true);
    return;
  }
  // PCG: x = 0, r = b and p = 0 were set by the right-hand side kernel; the first iteration takes
  // beta = 0, so its direction is z = B^{-1} r
  pcur = 0;
}

// One PCG iteration (Sec. 2.3), in the order z = B^{-1} r, beta, p = z + beta p with q = A p and
// alpha = (r, z) / (p, q), then x += alpha p, r -= alpha q and the convergence test; beta is 0 on a
// system's first iteration.  The direction alternates between two buffers (vec 3 and vec 6).
void KrylovWork::pcg_iteration() {
  double *q = vec(4), *z = vec(5);
  double *pold = vec(pcur ? 6 : 3), *pnew = vec(pcur ? 3 : 6);
  Reduce rd = red.get();
  const int flexible = s.prec == LAG_MIXED ? 1 : 0;
  const int rpr = p1->grid.nz;
  if (p1->use_tc) {
    // mixed path: forward DST, tridiagonal solve, then the inverse DST whose butterfly also forms
    // (r, z), (z, q) and beta
    const int rows = nrhs * rpr;
    p1->ensure_scratch(nrhs);
    float *w = p1->scratch.as<float>();
    dst_apply_tc_d2f(p1->dst, r(), w, rows, rpr, sc(), stream, true);
    tri_solve_f32(p1->tri32, w, w, nrhs, sc(), stream);
    dst_apply_tc_f2d_beta(p1->dst, w, z, nrhs, rpr, r(), q, flexible, sc(), rd, stream);
  } else if (p1->prec == LAG_FP64 && p1->dst.kind == 0 && tri_rz_fusable(p1->tri64, rd)) {
    // float64 path: one symmetric DST-I S serves both transforms, so (r, z) = (S r, T^{-1} S r) and
    // the tridiagonal solve forms it from its input and output, with beta.  Its output goes to q,
    // whose previous content only the flexible beta reads; the direction update rewrites it.
    p1->ensure_scratch(nrhs);
    double *w = p1->scratch.as<double>();
    dst_apply_f64(p1->dst, r(), w, nrhs * rpr, rpr, sc(), stream);
    tri_solve_f64_rz(p1->tri64, w, q, nrhs, sc(), rd, stream);
    dst_inverse_f64(p1->dst, q, z, nrhs * rpr, rpr, sc(), stream);
  } else {
    precond(r(), z);                                                 // z = B^{-1} r
    pcg_beta(r(), z, q, n, nrhs, flexible, sc(), rd, stream);
  }
  acoustic_apply_dir(*m, z, pold, pnew, q, nrhs, sc(), rd, stream);   // p = z + beta p, q = A p, alpha
  pcg_update_xr(x(), r(), pnew, q, n, nrhs, s.max_iter, sc(), rd, stream);  // x, r, ||r||, state
  pcur ^= 1;
}

static bool graphs_disabled() {
  const char *e = std::getenv("LAGWAVE_GRAPHS");
  return e != nullptr && e[0] == '0';
}

void KrylovWork::pcg_chunk(int iters) {
  for (int i = 0; i < iters; ++i) pcg_iteration();
}

// Condition of the WHILE node: repeat while a system still runs, no tensor-core kernel reported
// a pipeline timeout, and this launch has repeated the body fewer than `cap` times (a bound on one
// launch; the host launches again if a system is still running then).  The counter is reset when
// the loop ends, for the next launch.
__global__ void pcg_loop_kernel(const KrylovScalars *sc, int nrhs, const int *err0, const int *err1,
                                unsigned int *count, unsigned int cap, cudaGraphConditionalHandle handle) {
  bool run = false;
  for (int b = threadIdx.x; b < nrhs; b += blockDim.x) run |= (sc[b].state == ST_RUN);
  run = __any_sync(0xffffffffu, run);
  if (threadIdx.x == 0) {
    // count[1..2]: bodies executed since the work was set up (64-bit), for launch accounting
    unsigned long long *total = reinterpret_cast<unsigned long long *>(count + 2);
    *total += 1ull;
    const unsigned int c = *count + 1;
    if ((err0 != nullptr && *err0 != 0) || (err1 != nullptr && *err1 != 0) || c >= cap) run = false;
    *count = run ? c : 0u;
    cudaGraphSetConditional(handle, run ? 1u : 0u);
  }
}

void KrylovWork::pcg_loop_condition(unsigned long long handle) {
  const int *e0 = (p1 != nullptr && (p1->use_tc || p1->dst.oz)) ? p1->dst.tc_err : nullptr;
  pcg_loop_kernel<<<1, 32, 0, stream>>>(sc(), nrhs, e0, nullptr, wcount.as<unsigned int>(), 1024u,
                                        (cudaGraphConditionalHandle)handle);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void KrylovWork::pcg_while() {
  p1->ensure_scratch(nrhs);
  const void *key[4] = {p1->scratch.ptr, p1->tc_scratch.ptr, vecs.ptr, red.part.ptr};
  const int prod = p1->dst.tc_products;
  if (wexec != nullptr && (std::memcmp(key, wkey, sizeof(key)) != 0 || prod != wprod)) {
    cudaGraphExecDestroy(wexec);
    wexec = nullptr;
  }
  if (wexec == nullptr) {
    cudaGraph_t g = nullptr;
    LAG_CUDA_CHECK(cudaGraphCreate(&g, 0));
    try {
      cudaGraphConditionalHandle h;
      LAG_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      LAG_CUDA_CHECK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      LAG_CUDA_CHECK(cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      g_capturing = true;
      const int pc = pcur;
      try {
        pcur = 0;
        pcg_iteration();
        pcg_iteration();
        pcg_loop_condition((unsigned long long)h);
      } catch (...) {
        g_capturing = false;
        pcur = pc;
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(stream, &dummy);
        throw;
      }
      g_capturing = false;
      pcur = pc;
      cudaGraph_t captured = nullptr;
      LAG_CUDA_CHECK(cudaStreamEndCapture(stream, &captured));
      size_t nodes = 0;
      LAG_CUDA_CHECK(cudaGraphGetNodes(body, nullptr, &nodes));
      LAG_CUDA_CHECK(cudaGraphInstantiate(&wexec, g, 0));
      wnodes = nodes;
    } catch (...) {
      cudaGraphDestroy(g);
      throw;
    }
    cudaGraphDestroy(g);
    std::memcpy(wkey, key, sizeof(key));
    wprod = prod;
  }
  if (pcur != 0) throw Error(LAG_ECUDA, "PCG graph: the direction buffers are out of step");
  LAG_CUDA_CHECK(cudaGraphLaunch(wexec, stream));  // its kernels are counted from the body count (poll)
}

void KrylovWork::enqueue_chunk() {
  if (!elastic) {
    // the legacy default stream cannot be captured; the first iterations on a stream run eagerly:
    // they also perform the one-time kernel attribute setup, which must not happen inside a capture
    const bool capturable = stream != nullptr && stream != cudaStreamLegacy && stream != cudaStreamPerThread;
    if (!eager_done || !capturable || profiling_on() || graphs_disabled()) {
      pcg_chunk(chunk);  // an even count: the graph's body starts from the first direction buffer
      iters_this_solve += chunk;
      eager_done = true;
    } else {
      pcg_while();
      iters_this_solve += 2;
    }
  } else {
    for (int i = 0; i < chunk; ++i) {
      if (!cycle_open) gmres_begin_cycle(false);
      gmres_step();
      if (gj >= gk) gmres_end_cycle();
    }
    iters_this_solve += chunk;
  }
  mirror_state();
  if (predicted_first) {
    chunk = 2;  // after the predicted count: small chunks up to convergence
    predicted_first = false;
  } else if (chunk < 16) {
    chunk *= 2;
  }
}

void KrylovWork::mirror_state() {
  LAG_CUDA_CHECK(cudaMemcpyAsync(hsc, sc(), (size_t)nrhs * sizeof(KrylovScalars), cudaMemcpyDeviceToHost, stream));
  int *herr = reinterpret_cast<int *>(hsc + nrhs);
  const lag_precond *pl[2] = {p1, p2};
  for (int i = 0; i < 2; ++i)
    if (pl[i] != nullptr && (pl[i]->use_tc || pl[i]->dst.oz) && pl[i]->dst.tc_err != nullptr)
      LAG_CUDA_CHECK(cudaMemcpyAsync(herr + i, pl[i]->dst.tc_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  if (wcount.ptr != nullptr)
    LAG_CUDA_CHECK(cudaMemcpyAsync(herr + 2, wcount.as<unsigned int>() + 2, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, stream));
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
    if (wcount.ptr != nullptr) {  // kernels the PCG graph ran: its body's nodes per repeat
      unsigned long long bodies;
      std::memcpy(&bodies, herr + 2, sizeof(bodies));
      if (bodies > wbodies_seen) count_launch((int)((bodies - wbodies_seen) * wnodes));
      wbodies_seen = bodies;
    }
    if (herr[0] != 0 || herr[1] != 0)
      throw Error(LAG_ETIMEDOUT, "tensor-core DST: a bounded pipeline wait gave up (code " +
                                     std::to_string(herr[0] ? herr[0] : herr[1]) + "); the preconditioner output is invalid");
  }
  bool any_run = false, any_met = false;
  int most = 0;
  for (int i = 0; i < nrhs; ++i) {
    if (hsc[i].state == ST_RUN) any_run = true;
    if (hsc[i].state == ST_MET) any_met = true;
    most = std::max(most, hsc[i].iters);
  }
  if (any_run) return 0;
  predict = most;
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
