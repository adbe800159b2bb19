// Per-kernel-class timing: when enabled, every launch of a profiled kernel class is bracketed by
// two CUDA events recorded on the stream it is launched on; lag_profile_read sums the elapsed
// times per class.  Off by default (no events are recorded).
#include <mutex>

#include "internal.h"

namespace lag {

namespace {
struct Rec {
  int cls;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  LAG_CUDA_CHECK(cudaEventCreate(&e));
  return e;
}
}  // namespace

bool profiling_on() { return g_on; }

const char *kclass_name(int c) {
  static const char *names[NK_CLASSES] = {"dst_f64", "dst_f32_fwd", "dst_f32_inv", "dst_tc_fwd", "dst_tc_inv",
                                          "tri_f64", "tri_f32", "stencil_acoustic", "stencil_elastic",
                                          "krylov_vector", "laguerre", "gmres", "setup"};
  return (c >= 0 && c < NK_CLASSES) ? names[c] : "?";
}

ProfScope::ProfScope(int c, cudaStream_t st) : cls(c), s(st) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  a = take_event();
  LAG_CUDA_CHECK(cudaEventRecord(a, s));
  active = true;
}

ProfScope::~ProfScope() {
  if (!active) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, s);
  g_recs.push_back(Rec{cls, a, b});
}

}  // namespace lag

using namespace lag;

extern "C" {

int lag_profile_enable(lag_ctx *ctx, int on) {
  if (!ctx) return LAG_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_on = on != 0;
  return LAG_OK;
}

int lag_profile_read(lag_ctx *ctx, int nclasses, long long *counts, double *ms) {
  if (!ctx || nclasses < 0) return LAG_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int c = 0; c < nclasses; ++c) {
    if (counts) counts[c] = 0;
    if (ms) ms[c] = 0.0;
  }
  for (auto &r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return LAG_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return LAG_ECUDA;
    if (r.cls < nclasses) {
      if (counts) counts[r.cls] += 1;
      if (ms) ms[r.cls] += t;
    }
  }
  return LAG_OK;
}

const char *lag_profile_class_name(int c) { return kclass_name(c); }
int lag_profile_num_classes(void) { return NK_CLASSES; }

}  // extern "C"
