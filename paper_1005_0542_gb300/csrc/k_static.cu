// Preconditioner apply that allocates nothing (for callers that cannot allocate device memory).
//
// lag_precond_apply keeps its intermediate spectrum in a buffer the plan allocates (and grows)
// with cudaMalloc.  Some callers cannot let a library allocate at call time: a host framework
// that owns all device memory through its own allocator and forbids others, or a real-time loop
// that must not block in cudaMalloc / cudaFree (cudaFree synchronises the device).  For them,
// lag_precond_apply_static runs the three steps (DST-I along x, partitioned tridiagonal solve
// along z, DST-I back; cylindrical plans: DCT-II along z, systems along r, inverse DCT-II) with the
// spectrum in the file-scope device array below, whose size is
// fixed when the library is loaded; the DST runs on the FP64 SIMT pipes (the tensor-core float64
// DST keeps its operand slices in plan scratch that lag_precond_apply allocates on demand).  The plan itself is created beforehand (lag_precond_create
// allocates its factors once).
#include <mutex>

#include "internal.h"

namespace {

// 2^21 float64 values = 16 MiB, held on every GPU that loads the library until the process exits
constexpr size_t kStaticSpectrumPoints = (size_t)1 << 21;
static __device__ __align__(256) double g_static_spectrum[kStaticSpectrumPoints];

std::mutex g_sym_mu;
double *g_sym_ptr[64] = {nullptr};  // device address of g_static_spectrum, per device

}  // namespace

using namespace lag;

extern "C" {

size_t lag_precond_static_capacity(void) { return kStaticSpectrumPoints; }

int lag_precond_apply_static(lag_precond *p, const double *r, double *z, int nrhs) {
  if (!p || nrhs < 0 || (nrhs > 0 && (!r || !z))) return LAG_EINVAL;
  lag_ctx *ctx = p->ctx;
  if (p->prec != LAG_FP64) {
    ctx->last_error = "lag_precond_apply_static: only float64 (LAG_FP64) plans are supported";
    return LAG_EINVAL;
  }
  const size_t points = (size_t)nrhs * p->grid.nz * p->grid.nx;
  if (points > kStaticSpectrumPoints) {
    ctx->last_error = "lag_precond_apply_static: nrhs * nz * nx = " + std::to_string(points) +
                      " exceeds the static capacity of " + std::to_string(kStaticSpectrumPoints) + " values";
    return LAG_EINVAL;
  }
  if (nrhs == 0) return LAG_OK;
  try {
    LAG_CUDA_CHECK(cudaSetDevice(ctx->device));
    if (ctx->device < 0 || ctx->device >= 64) throw Error(LAG_EINVAL, "device index out of range");
    double *spec = nullptr;
    {
      // once per device, with that device current: the host-side symbol is only a stand-in, the
      // kernels need the array's device address
      std::lock_guard<std::mutex> lk(g_sym_mu);
      if (g_sym_ptr[ctx->device] == nullptr) {
        void *addr = nullptr;
        LAG_CUDA_CHECK(cudaGetSymbolAddress(&addr, g_static_spectrum));
        g_sym_ptr[ctx->device] = static_cast<double *>(addr);
      }
      spec = g_sym_ptr[ctx->device];
    }
    // every value of the spectrum the kernels read is written first in the same call: nothing in
    // the array has to start at zero
    const int rows = nrhs * p->grid.nz;
    dst_apply_f64_simt(p->dst, r, spec, rows, p->grid.nz, nullptr, ctx->stream);
    tri_solve_f64(p->tri64, spec, spec, nrhs, nullptr, ctx->stream);
    dst_inverse_f64_simt(p->dst, spec, z, rows, p->grid.nz, nullptr, ctx->stream);
    return LAG_OK;
  } catch (const Error &e) {
    ctx->last_error = e.what();
    return e.status;
  } catch (const std::exception &e) {
    ctx->last_error = e.what();
    return LAG_ECUDA;
  }
}

}  // extern "C"
