// Checkpoint / restore of a shot, and the bounded-wait self-test.
//
// The state of a shot after harmonic m is: m, the two history sums T, S of every source (they
// carry everything the later right-hand sides of Eq. 9 need), the receiver values of harmonics
// 0..m-1 and the per-harmonic statistics.  A checkpoint copies that to host memory; restoring it
// into a new shot built from the same inputs continues the series with identical arithmetic.
#include <cstring>

#include "solver.h"

using namespace lag;

namespace {

struct CkptHeader {
  uint64_t magic;
  int32_t nx, nz, nsrc, ncomp, nrcv, n_harm, m, last_status;
  int64_t total_iters;
};
constexpr uint64_t kMagic = 0x4c41475741564531ull;  // "LAGWAVE1"

size_t ckpt_bytes(const lag_shot *sh) {
  const size_t hist = 2 * sh->wk.n * sh->nsrc * sizeof(double);
  const size_t rr = (size_t)sh->lag.n_harm * sh->nsrc * sh->ncomp * sh->nrcv * sizeof(double);
  const size_t stats = (size_t)sh->nsrc * sh->lag.n_harm * (sizeof(int) + sizeof(double));
  return sizeof(CkptHeader) + hist + rr + stats;
}

// wait on an mbarrier that nothing arrives on, for at most `limit` polls; 1 = timed out
__global__ void wait_timeout_kernel(long long limit, int *status) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (long long i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(0)
        : "memory");
    if (ok) {
      *status = 0;
      return;
    }
    __nanosleep(1000);
  }
  *status = 1;
}

}  // namespace

extern "C" {

size_t lag_shot_checkpoint_size(const lag_shot *sh) { return sh ? ckpt_bytes(sh) : 0; }

int lag_shot_checkpoint(lag_shot *sh, void *host_buf, size_t bytes) {
  if (!sh || !host_buf || bytes < ckpt_bytes(sh)) return LAG_EINVAL;
  try {
    LAG_CUDA_CHECK(cudaSetDevice(sh->ctx->device));
    LAG_CUDA_CHECK(cudaStreamSynchronize(sh->stream));
    if (sh->phase != 0) throw Error(LAG_EINVAL, "checkpoint between harmonics only");
    if (sh->failed) throw Error(LAG_EINVAL, "the shot has failed; there is nothing to resume");
    uint8_t *o = static_cast<uint8_t *>(host_buf);
    CkptHeader h{kMagic, sh->grid.nx, sh->grid.nz, sh->nsrc, sh->ncomp, sh->nrcv, sh->lag.n_harm, sh->m, sh->last_status,
                 sh->total_iters};
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const size_t hist = 2 * sh->wk.n * sh->nsrc * sizeof(double);
    LAG_CUDA_CHECK(cudaMemcpy(o, sh->hist.ptr, hist, cudaMemcpyDeviceToHost));
    o += hist;
    const size_t rr = (size_t)sh->lag.n_harm * sh->nsrc * sh->ncomp * sh->nrcv * sizeof(double);
    if (rr) LAG_CUDA_CHECK(cudaMemcpy(o, sh->rrcv(), rr, cudaMemcpyDeviceToHost));
    o += rr;
    std::memcpy(o, sh->iters.data(), sh->iters.size() * sizeof(int));
    o += sh->iters.size() * sizeof(int);
    std::memcpy(o, sh->relres.data(), sh->relres.size() * sizeof(double));
    return LAG_OK;
  } catch (const Error &e) {
    sh->ctx->last_error = e.what();
    return e.status;
  }
}

int lag_shot_restore(lag_shot *sh, const void *host_buf, size_t bytes) {
  if (!sh || !host_buf || bytes < sizeof(CkptHeader)) return LAG_EINVAL;
  try {
    LAG_CUDA_CHECK(cudaSetDevice(sh->ctx->device));
    LAG_CUDA_CHECK(cudaStreamSynchronize(sh->stream));
    const uint8_t *i = static_cast<const uint8_t *>(host_buf);
    CkptHeader h;
    std::memcpy(&h, i, sizeof(h));
    i += sizeof(h);
    if (h.magic != kMagic || h.nx != sh->grid.nx || h.nz != sh->grid.nz || h.nsrc != sh->nsrc ||
        h.ncomp != sh->ncomp || h.nrcv != sh->nrcv || h.n_harm != sh->lag.n_harm || h.m < 0 || h.m > h.n_harm ||
        bytes < ckpt_bytes(sh))
      throw Error(LAG_EINVAL, "checkpoint does not match this shot");
    const size_t hist = 2 * sh->wk.n * sh->nsrc * sizeof(double);
    LAG_CUDA_CHECK(cudaMemcpy(sh->hist.ptr, i, hist, cudaMemcpyHostToDevice));
    i += hist;
    const size_t rr = (size_t)sh->lag.n_harm * sh->nsrc * sh->ncomp * sh->nrcv * sizeof(double);
    if (rr) LAG_CUDA_CHECK(cudaMemcpy(sh->rrcv(), i, rr, cudaMemcpyHostToDevice));
    i += rr;
    std::memcpy(sh->iters.data(), i, sh->iters.size() * sizeof(int));
    i += sh->iters.size() * sizeof(int);
    std::memcpy(sh->relres.data(), i, sh->relres.size() * sizeof(double));
    sh->m = h.m;
    sh->phase = 0;
    sh->total_iters = h.total_iters;
    sh->last_status = h.last_status;
    sh->failed = false;
    return LAG_OK;
  } catch (const Error &e) {
    sh->ctx->last_error = e.what();
    return e.status;
  }
}

int lag_selftest_wait_timeout(lag_ctx *ctx, long long polls) {
  if (!ctx || polls < 1) return LAG_EINVAL;
  try {
    LAG_CUDA_CHECK(cudaSetDevice(ctx->device));
    DevBuf st;
    st.alloc(ctx, sizeof(int), true);
    wait_timeout_kernel<<<1, 32, 0, ctx->stream>>>(polls, st.as<int>());
    count_launch();
    LAG_LAUNCH_CHECK();
    int h = -1;
    LAG_CUDA_CHECK(cudaMemcpyAsync(&h, st.ptr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LAG_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    if (h == 1) {
      ctx->last_error = "bounded device wait gave up (self-test: nothing arrives on the barrier)";
      return LAG_ETIMEDOUT;
    }
    return h == 0 ? LAG_OK : LAG_ECUDA;
  } catch (const Error &e) {
    ctx->last_error = e.what();
    return e.status;
  }
}

}  // extern "C"
