// Krylov drivers (PCG / flexible GMRES(k)) and whole-shot state, host side.
#pragma once

#include "internal.h"

namespace lag {

struct ReduceBuf {
  DevBuf part, count;
  int nrhs = 0, cap = 0, nv = 0;
  void ensure(lag_ctx *ctx, int nrhs, int cap, int nv);
  Reduce get() const;
};

int stencil_blocks(const lag_grid &g);
void check_solver(const lag_solver &s, bool elastic);
bool tc_disabled();
void widen_f32(const float *a, double *b, size_t n, cudaStream_t s);

// Device-resident Krylov state for nrhs independent systems of one medium, driven in chunks of
// iterations with the convergence test on the device (KrylovScalars::state); the host looks at
// a pinned copy of the scalars only between chunks.
struct KrylovWork {
  lag_ctx *ctx = nullptr;
  lag_medium *m = nullptr;
  lag_precond *p1 = nullptr, *p2 = nullptr;
  lag_solver s{};
  int nrhs = 0, ncomp = 1;
  size_t nplane = 0, n = 0;  // values per component plane, per rhs
  cudaStream_t stream = nullptr;
  bool elastic = false;
  DevBuf vecs;               // see offsets below
  DevBuf scal;               // KrylovScalars[nrhs]
  DevBuf gm;                 // FGMRES small arrays
  ReduceBuf red;
  KrylovScalars *hsc = nullptr;   // pinned mirror
  cudaEvent_t ev = nullptr;
  bool pending = false;
  int chunk = 2;
  int iters_this_solve = 0;
  // iterations the last finished solve took (the most over its systems): the next solve's first
  // chunk runs just below that many at once, then small chunks, so that eagerly launched solves
  // issue few iterations past convergence (the next harmonic's count is within one or two)
  int predict = 0;
  bool predicted_first = false;
  // FGMRES bookkeeping (host): current cycle step j, restart length k
  int gj = 0, gk = 0;
  bool cycle_open = false;
  GmresDev gdev{};
  // PCG on the device: one CUDA graph whose conditional WHILE node repeats a body of two iterations
  // until no system runs (pcg_loop_kernel sets the condition from the systems' states), so a solve is
  // one graph launch with no host round trip and at most one iteration past convergence (whose
  // kernels skip the finished systems).  Captured again when a pointer or the DST product count
  // it baked in changes.
  cudaGraphExec_t wexec = nullptr;
  unsigned long long wnodes = 0;
  const void *wkey[4] = {};
  int wprod = 0;
  DevBuf wcount;             // the loop's repeat counter (a bound on one launch) and its body total
  unsigned long long wbodies_seen = 0;
  bool eager_done = false;
  int pcur = 0;              // which of the two direction buffers holds the current p

  ~KrylovWork();
  void setup(lag_ctx *ctx, lag_medium *m, lag_precond *p1, lag_precond *p2, const lag_solver &s, int nrhs,
             cudaStream_t stream);
  double *vec(int i) const { return vecs.as<double>() + (size_t)i * n * nrhs; }
  // acoustic: 0 b, 1 x, 2 r, 3 p (even iterations' old direction), 4 q, 5 z, 6 p (odd ones')
  // elastic:  0 b, 1 x, 2 r (= w work), 3..3+k V_0..V_k, 4+k.. Z_0..Z_{k-1}
  double *b() const { return vec(0); }
  double *x() const { return vec(1); }
  double *r() const { return vec(2); }
  KrylovScalars *sc() const { return scal.as<KrylovScalars>(); }

  void precond(const double *r, double *z);
  void start_from_b();        // x = 0, r = b, ||b||
  void start_from_r();        // r, x already set with ||b|| in the scalars (Laguerre right-hand side)
  void enqueue_chunk();       // a chunk of iterations + async copy of the scalars + event
  int  poll(bool block);      // 1: all systems finished, 0: running, <0: pending work not finished (non-blocking)
  int  finish_status() const; // LAG_OK / LAG_ENOTCONV / LAG_ENUMERIC from the host mirror
  int  solve_blocking();
  void copy_result(double *x_out);
  void report(int *iters, double *relres) const;

 private:
  void pcg_iteration();
  void pcg_chunk(int iters);  // iters PCG iterations, launched one kernel at a time
  void pcg_while();           // iterate until every system stops, as one graph launch
  void pcg_loop_condition(unsigned long long handle);  // the WHILE node's condition kernel
  void mirror_state();        // async copy of the scalars and the plans' error words + event
  void gmres_begin_cycle(bool first);
  void gmres_step();
  void gmres_end_cycle();
};

}  // namespace lag

// ------------------------------------------------------------------------------ shot
struct lag_shot {
  lag_ctx *ctx = nullptr;
  lag_grid grid{};
  lag_laguerre lag{};
  lag_solver solver{};
  lag_wavelet wavelet{};
  bool elastic = false;
  int nsrc = 0, nrcv = 0, nt = 0, ncomp = 1;
  cudaStream_t stream = nullptr;
  lag_medium *medium = nullptr;
  lag_precond *p1 = nullptr, *p2 = nullptr;
  lag::KrylovWork wk;
  lag::DevBuf hist;       // T, S accumulators [nsrc][ncomp][nz][nx] each
  lag::DevBuf tables;     // fm [n] | tab [n][nt] | t [nt] | rrcv [n][nsrc][ncomp][nrcv] | traces
  lag::DevBuf idx;        // src_idx [nsrc] | rcv_idx [nrcv]
  lag::DevBuf fm_scratch;
  std::vector<double> cm, chat;   // c_m, c^_m
  int m = 0;              // harmonics finished
  int phase = 0;          // 0: next harmonic not started, 1: iterating
  bool failed = false;
  int last_status = LAG_OK;
  std::vector<int> iters;        // [nsrc][n_harm]
  std::vector<double> relres;    // [nsrc][n_harm]
  long long total_iters = 0;
  double t_start = 0.0, t_busy = 0.0;
  size_t device_bytes = 0;
  ~lag_shot();
  double *fm() const { return tables.as<double>(); }
  double *tab() const { return fm() + lag.n_harm; }
  double *tout() const { return tab() + (size_t)lag.n_harm * nt; }
  double *rrcv() const { return tout() + nt; }
  double *traces() const { return rrcv() + (size_t)lag.n_harm * nsrc * ncomp * nrcv; }
  int pump(bool block);   // 1 done, 0 in progress
};
