// Serving loop: continuous batching of shots.
//
// Requests are admitted in arrival order when their estimated device memory fits the context's
// HBM budget next to the requests already running (and fewer than max_active run).  Each admitted
// request is a shot with its own CUDA stream; the scheduler thread advances every running shot by
// one chunk of Krylov iterations whenever its previous chunk has finished, so the work of
// different requests overlaps on the device and a new request starts while others are mid-way.
// A shot's arithmetic never depends on the other shots (no shared reductions), so a request gives
// the same result alone and in the mix.
#include <cstring>
#include <deque>

#include "solver.h"

using namespace lag;

lag_shot *shot_new(lag_ctx *ctx, const lag_grid &g, const double *c, const double *vs, const double *rho,
                   const lag_laguerre &lag, const lag_solver &s, const lag_wavelet &w, int nsrc, const lag_point *src,
                   int nrcv, const lag_point *rcv, int nt, const double *t_out);

namespace {

struct Request {
  uint64_t ticket = 0;
  lag_request req{};
  std::vector<double> c, vs, rho, t_out, traces;
  std::vector<lag_point> src, rcv;
  size_t est_bytes = 0;
  lag_shot *shot = nullptr;
  bool cancel = false, done = false;
  int status = LAG_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
  long long iters = 0;
  size_t device_bytes = 0;
  int harmonics = 0;
  std::string error;
};

// device memory of a shot, estimated from its sizes (vectors, history, coefficients, plans, tables)
size_t estimate_bytes(const lag_request &r) {
  const size_t nx = r.grid.nx, nz = r.grid.nz, n = nx * nz;
  const size_t ncomp = r.kind == 1 ? 2 : 1;
  const size_t nsrc = r.nsrc;
  const size_t nvec = r.kind == 1 ? 3 + 2 * (size_t)r.solver.restart_k + 1 : 7;
  size_t b = (nvec + 2) * n * ncomp * nsrc * 8;                 // Krylov vectors + T, S
  b += (r.kind == 1 ? 12 : 6) * n * 8;                           // operator coefficients, rho h^2
  const size_t nplans = r.kind == 1 ? 2 : 1;
  const size_t ku = (nx + 1) / 2;
  b += 2 * ku * ku * 12 + ku * ku * 8 * 2;                        // DST halves (+ tensor-core copies)
  b += nplans * (5 * 3 * ((nz + 31) / 32 + 1) * nx + nx * 32 * 18) * 12;  // tridiagonal factors
  b += n * ncomp * nsrc * 8;                                     // preconditioner scratch
  b += nplans * (2 * 9 * (nz * nsrc + 256) * (ku + 64) * 2 + 152 * 128 * 128 * 8);  // exact-slice A slices, stream-K parts
  b += ((size_t)r.lag.n_harm * (r.nt + 1 + nsrc * ncomp * r.nrcv) + (size_t)r.nt * (1 + nsrc * ncomp * r.nrcv)) * 8;
  b += (size_t)r.lag.n_harm * 16 * 8 * 40;                       // source-coefficient scratch (transient)
  return b + (4u << 20);
}

}  // namespace

struct Server {
  lag_ctx *ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  int max_active = 8;
  uint64_t next = 1;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  size_t reserved = 0;  // estimated bytes of the running requests

  void finish(const std::shared_ptr<Request> &r, int status) {
    r->status = status;
    r->t_done = now_seconds() - ctx->t_created;
    if (r->shot) {
      r->iters = r->shot->total_iters;
      r->harmonics = r->shot->m;
      r->device_bytes = r->shot->device_bytes;
      lag_shot_destroy(r->shot);
      r->shot = nullptr;
    }
    r->done = true;
  }

  void run() {
    cudaSetDevice(ctx->device);
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
        if (active.empty() && queue.empty()) cv.wait_for(lk, std::chrono::milliseconds(20));
        if (stop) break;
      }
      admit();
      bool progressed = false;
      for (size_t i = 0; i < active.size();) {
        auto r = active[i];
        bool remove = false;
        if (r->cancel) {
          std::lock_guard<std::mutex> lk(mu);
          finish(r, LAG_ECANCELED);
          remove = true;
        } else {
          try {
            const int d = r->shot->pump(false);
            if (d == 1) {
              progressed = true;
              int st = r->shot->failed ? r->shot->last_status : r->shot->last_status;
              if (st == LAG_OK || st == LAG_ENOTCONV) {
                const int rows = r->req.nsrc * r->shot->ncomp * r->req.nrcv;
                r->traces.assign((size_t)rows * r->req.nt, 0.0);
                if (rows > 0 && r->req.nt > 0) {
                  const int rc = lag_shot_traces(r->shot, r->traces.data());
                  if (rc != LAG_OK) st = rc;
                }
              }
              std::lock_guard<std::mutex> lk(mu);
              finish(r, st);
              remove = true;
            }
          } catch (const Error &e) {
            std::lock_guard<std::mutex> lk(mu);
            r->error = e.what();
            finish(r, e.status);
            remove = true;
          } catch (const std::exception &e) {
            std::lock_guard<std::mutex> lk(mu);
            r->error = e.what();
            finish(r, LAG_ECUDA);
            remove = true;
          }
        }
        if (remove) {
          std::lock_guard<std::mutex> lk(mu);
          reserved -= r->est_bytes;
          active.erase(active.begin() + i);
          progressed = true;
        } else {
          ++i;
        }
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    // stop: cancel what is left
    std::lock_guard<std::mutex> lk(mu);
    for (auto &r : active) finish(r, LAG_ECANCELED);
    active.clear();
    for (auto &r : queue) finish(r, LAG_ECANCELED);
    queue.clear();
  }

  void admit() {
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (queue.empty() || (int)active.size() >= max_active) return;
        r = queue.front();
        if (r->cancel) {
          queue.pop_front();
          finish(r, LAG_ECANCELED);
          continue;
        }
        if (ctx->budget != 0) {
          if (r->est_bytes > ctx->budget) {  // can never fit
            queue.pop_front();
            r->error = "request needs more device memory than the HBM budget";
            finish(r, LAG_ENOMEM);
            continue;
          }
          if (reserved + r->est_bytes > ctx->budget) return;  // wait for running requests to finish
        }
        queue.pop_front();
        reserved += r->est_bytes;
      }
      try {
        const lag_request &q = r->req;
        r->shot = shot_new(ctx, q.grid, r->c.data(), q.kind == 1 ? r->vs.data() : nullptr, r->rho.data(), q.lag,
                           q.solver, q.wavelet, q.nsrc, r->src.data(), q.nrcv, r->rcv.data(), q.nt, r->t_out.data());
        r->t_admit = now_seconds() - ctx->t_created;
        std::lock_guard<std::mutex> lk(mu);
        active.push_back(r);
      } catch (const Error &e) {
        std::lock_guard<std::mutex> lk(mu);
        reserved -= r->est_bytes;
        r->error = e.what();
        finish(r, e.status);
      } catch (const std::exception &e) {
        std::lock_guard<std::mutex> lk(mu);
        reserved -= r->est_bytes;
        r->error = e.what();
        finish(r, LAG_ECUDA);
      }
    }
  }
};

void server_destroy(lag_ctx *ctx) {
  if (!ctx || !ctx->server) return;
  Server *s = ctx->server;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  delete s;
  ctx->server = nullptr;
}

extern "C" {

int lag_serve_start(lag_ctx *ctx, int max_active) {
  if (!ctx || max_active < 1) return LAG_EINVAL;
  if (ctx->server) return LAG_OK;
  Server *s = new Server();
  s->ctx = ctx;
  s->max_active = max_active;
  ctx->server = s;
  s->th = std::thread([s] { s->run(); });
  return LAG_OK;
}

int lag_serve_stop(lag_ctx *ctx) {
  if (!ctx) return LAG_EINVAL;
  server_destroy(ctx);
  return LAG_OK;
}

int lag_serve_submit(lag_ctx *ctx, const lag_request *q, uint64_t *ticket) {
  if (!ctx || !q || !ticket) return LAG_EINVAL;
  if (!ctx->server) {
    const int rc = lag_serve_start(ctx, 8);
    if (rc != LAG_OK) return rc;
  }
  if ((q->kind != 0 && q->kind != 1) || q->grid.nx < 1 || q->grid.nz < 1 || !q->c_host || !q->rho_host ||
      (q->kind == 1 && !q->vs_host) || q->nsrc < 1 || !q->src || q->nrcv < 0 || q->nt < 0 || q->lag.n_harm < 1)
    return LAG_EINVAL;
  auto r = std::make_shared<Request>();
  const size_t n = (size_t)q->grid.nx * q->grid.nz;
  r->req = *q;
  r->c.assign(q->c_host, q->c_host + n);
  r->rho.assign(q->rho_host, q->rho_host + n);
  if (q->kind == 1) r->vs.assign(q->vs_host, q->vs_host + n);
  r->src.assign(q->src, q->src + q->nsrc);
  if (q->nrcv > 0) r->rcv.assign(q->rcv, q->rcv + q->nrcv);
  if (q->nt > 0) r->t_out.assign(q->t_out_host, q->t_out_host + q->nt);
  r->req.c_host = r->req.vs_host = r->req.rho_host = nullptr;
  r->req.src = nullptr;
  r->req.rcv = nullptr;
  r->req.t_out_host = nullptr;
  r->est_bytes = estimate_bytes(*q);
  Server *s = ctx->server;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next++;
    r->t_submit = now_seconds() - ctx->t_created;
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return LAG_OK;
}

int lag_serve_poll(lag_ctx *ctx, uint64_t ticket, lag_result *out) {
  if (!ctx || !ctx->server || !out) return LAG_EINVAL;
  Server *s = ctx->server;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return LAG_EINVAL;
    r = it->second;
    if (!r->done) return LAG_EAGAIN;
    s->all.erase(it);
  }
  out->status = r->status;
  out->t_submit = r->t_submit;
  out->t_admit = r->t_admit;
  out->t_done = r->t_done;
  out->total_iters = r->iters;
  out->device_bytes = r->device_bytes;
  out->harmonics_done = r->harmonics;
  if (out->traces_host && !r->traces.empty())
    std::memcpy(out->traces_host, r->traces.data(), r->traces.size() * sizeof(double));
  if (!r->error.empty()) ctx->last_error = r->error;
  return LAG_OK;
}

int lag_serve_cancel(lag_ctx *ctx, uint64_t ticket) {
  if (!ctx || !ctx->server) return LAG_EINVAL;
  Server *s = ctx->server;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return LAG_EINVAL;
  it->second->cancel = true;
  return LAG_OK;
}

}  // extern "C"
