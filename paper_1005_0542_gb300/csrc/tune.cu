// Autotuner of a preconditioner plan: partition count and mode tile of the tridiagonal solve and,
// on mixed plans, the number of bf16 products of the tensor-core DST.  Each candidate is timed with CUDA events on
// the context's stream over a few applies to nrhs seeded right-hand sides; a product count is kept
// only if its result stays within 2e-2 (relative L2) of the 3-product split, i.e. the
// preconditioner remains the same operator up to bf16 rounding.
#include <cmath>
#include <vector>

#include "internal.h"

namespace lag {

__global__ void tune_fill_kernel(double *x, size_t n, unsigned seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)(i * 2654435761u) ^ seed;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    x[i] = (double)h / 4294967296.0 - 0.5;
  }
}

__global__ void tune_diff_kernel(const double *a, const double *b, size_t n, double *out) {
  double d = 0.0, s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double e = a[i] - b[i];
    d = fma(e, e, d);
    s = fma(b[i], b[i], s);
  }
  d = warp_sum(d);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, d);
    atomicAdd(out + 1, s);
  }
}

static float time_applies(lag_precond *p, const double *r, double *z, int nrhs, int reps) {
  cudaStream_t s = p->ctx->stream;
  cudaEvent_t a, b;
  LAG_CUDA_CHECK(cudaEventCreate(&a));
  LAG_CUDA_CHECK(cudaEventCreate(&b));
  p->apply(r, z, nrhs, nullptr, s);  // warm-up (and scratch growth)
  LAG_CUDA_CHECK(cudaEventRecord(a, s));
  for (int i = 0; i < reps; ++i) p->apply(r, z, nrhs, nullptr, s);
  LAG_CUDA_CHECK(cudaEventRecord(b, s));
  LAG_CUDA_CHECK(cudaEventSynchronize(b));
  float ms = 0.f;
  LAG_CUDA_CHECK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

void precond_rebuild_tri(lag_precond *p, int want_P, int want_mt, cudaStream_t s) {
  TriFactors t64;
  t64.nx = p->grid.nx;
  t64.nz = p->grid.nz;
  const bool gen = p->zrows.ptr != nullptr;
  tri_choose_layout(t64, 8, want_P, p->prec == LAG_FP64 ? want_mt : 0, gen);
  tri_build_factors(t64, p->tri_store, p->coef(), p->grid.dx, p->grid.dz, s, 0);
  p->tri64 = t64;
  if (p->prec == LAG_MIXED) {
    TriFactors t32;
    t32.nx = p->grid.nx;
    t32.nz = p->grid.nz;
    tri_choose_layout(t32, 4, want_P, want_mt, gen);
    if (p->use_tc) {
      TriFactors tp = t64;
      DevBuf tmp;
      tmp.ctx = p->ctx;
      tri_build_factors(tp, tmp, p->coef(), p->grid.dx, p->grid.dz, s, p->dst.ku);
      tri_make_f32(tp, t32, p->tri32_store, s);
      LAG_CUDA_CHECK(cudaStreamSynchronize(s));
    } else {
      tri_make_f32(t64, t32, p->tri32_store, s);
    }
    p->tri32 = t32;
  }
  LAG_CUDA_CHECK(cudaStreamSynchronize(s));
}

}  // namespace lag

using namespace lag;

extern "C" int lag_precond_autotune(lag_precond *p, int nrhs, int *partitions_out, int *mt_out, int *products_out,
                                    double *ms_out) {
  if (!p || nrhs < 1) return LAG_EINVAL;
  try {
    LAG_CUDA_CHECK(cudaSetDevice(p->ctx->device));
    cudaStream_t s = p->ctx->stream;
    const size_t n = (size_t)nrhs * p->grid.nx * p->grid.nz;
    DevBuf buf;
    buf.alloc(p->ctx, (3 * n + 2) * sizeof(double));
    double *r = buf.as<double>(), *z = r + n, *zref = z + n, *acc = zref + n;
    tune_fill_kernel<<<1024, 256, 0, s>>>(r, n, 0x1005u);
    count_launch();
    LAG_LAUNCH_CHECK();
    const int reps = 3;
    // 1. partition count x mode tile of the register kernel (float32 8 / 16 / 32 modes per CTA,
    //    float64 4 / 8; a layout that falls back to the shared-memory kernel ignores the tile)
    const bool f64 = p->prec == LAG_FP64;
    const std::vector<int> tiles = f64 ? std::vector<int>{4, 8} : std::vector<int>{8, 16, 32};
    float best = 1e30f;
    int bestWant = 32, bestMt = 0;
    for (int want : {8, 16, 32}) {
      for (int mt : tiles) {
        precond_rebuild_tri(p, want, mt, s);
        const TriFactors &t = f64 ? p->tri64 : p->tri32;
        if (t.reg && t.mt != mt) continue;  // tile not available at this partition length
        if (!t.reg && mt != tiles[0]) continue;  // the shared-memory kernel: time once per count
        const float ms = time_applies(p, r, z, nrhs, reps);
        if (ms < best) {
          best = ms;
          bestWant = want;
          bestMt = mt;
        }
      }
    }
    precond_rebuild_tri(p, bestWant, bestMt, s);
    const int bestP = f64 ? p->tri64.P : p->tri32.P;
    if (mt_out) *mt_out = f64 ? p->tri64.mt : p->tri32.mt;
    // 2. bf16 products of the tensor-core DST (quality-checked against the split)
    int bestK = p->use_tc ? p->dst.tc_products : 3;
    if (p->use_tc) {
      p->dst.tc_products = 3;
      p->apply(r, zref, nrhs, nullptr, s);
      best = time_applies(p, r, z, nrhs, reps);
      bestK = 3;
      for (int k : {2, 1}) {
        p->dst.tc_products = k;
        const float ms = time_applies(p, r, z, nrhs, reps);
        LAG_CUDA_CHECK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
        tune_diff_kernel<<<512, 256, 0, s>>>(z, zref, n, acc);
        count_launch();
        LAG_LAUNCH_CHECK();
        double h[2];
        LAG_CUDA_CHECK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
        LAG_CUDA_CHECK(cudaStreamSynchronize(s));
        const double relerr = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
        if (relerr < 2e-2 && ms < best) {
          best = ms;
          bestK = k;
        }
      }
      p->dst.tc_products = bestK;
    }
    if (partitions_out) *partitions_out = bestP;
    if (products_out) *products_out = bestK;
    if (ms_out) *ms_out = best;
    return LAG_OK;
  } catch (const Error &e) {
    p->ctx->last_error = e.what();
    return e.status;
  } catch (const std::exception &e) {
    p->ctx->last_error = e.what();
    return LAG_ECUDA;
  }
}
