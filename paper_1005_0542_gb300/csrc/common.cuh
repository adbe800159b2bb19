// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>

namespace lag {

// ------------------------------------------------------------------ errors
// Host code throws lag::Error; the C ABI layer converts it to a status code.
struct Error : public std::runtime_error {
  int status;
  Error(int s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define LAG_CUDA_CHECK(call)                                                                  \
  do {                                                                                        \
    cudaError_t e__ = (call);                                                                 \
    if (e__ != cudaSuccess)                                                                   \
      throw ::lag::Error(-5, std::string(#call) + ": " + cudaGetErrorString(e__) + " (" +     \
                                 __FILE__ + ":" + std::to_string(__LINE__) + ")");            \
  } while (0)

#define LAG_LAUNCH_CHECK() LAG_CUDA_CHECK(cudaGetLastError())

// One-time set-up that belongs to a device (kernel attributes, constant memory): runs f once per
// device, on the device current at the call, under a mutex (several host threads may make the first
// calls).  f throws on failure and is then retried by the next call.
struct PerDeviceOnce {
  std::mutex mu;
  uint64_t done[4] = {0, 0, 0, 0};  // one bit per device ordinal (256 devices)
  template <typename F>
  void run(F &&f) {
    int dev = 0;
    LAG_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) throw Error(-5, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    const uint64_t bit = 1ull << (dev & 63);
    if (done[dev >> 6] & bit) return;
    f();
    done[dev >> 6] |= bit;
  }
};

// Count of the library's kernel launches (process-wide, for launch accounting).
// While a thread captures a CUDA graph its launches are not counted (the graph's kernel nodes
// are counted at every replay instead).
extern unsigned long long g_launches;
extern thread_local bool g_capturing;
inline void count_launch(int n = 1) {
  if (!g_capturing) __atomic_add_fetch(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED);
}

// ------------------------------------------------------------------ Krylov scalars
// One record per right-hand side, resident on the device.  Kernels read alpha/beta from here
// and skip a right-hand side whose `state` is not 0, so no host round trip is needed between
// the steps of an iteration.
struct KrylovScalars {
  double bb;      // ||b||^2
  double rz;      // (r, z) of the current iterate
  double pq;      // (p, q)
  double rr;      // (r, r)
  double zq;      // (z, q)      (Polak-Ribiere beta)
  double alpha;
  double beta;
  double tol2;    // tol^2
  int state;      // ST_* below
  int iters;
  int jdone;      // GMRES: steps taken in the open cycle
  int reorth;     // GMRES: 1 if this step's second Gram-Schmidt pass runs (set by the first pass)
};
static_assert(sizeof(KrylovScalars) == 80, "layout");

// Residual scaling of the float32 / bf16 preconditioner pipelines inside PCG: the right-hand side of
// system b enters them multiplied by 2^-e, e = the binary exponent of ||r_b|| (KrylovScalars::rr),
// and the float64 output is multiplied by 2^e again.  Power-of-two scaling is exact; it keeps
// residuals that are tiny in absolute terms (a weak source, a late iterate) away from float32
// underflow, the preconditioner being linear.
// ilogb(sqrt(rr)) = floor(ilogb(rr) / 2) for every positive finite rr (a correctly rounded square
// root of a double below 2^(2k+2) stays below 2^(k+1)), from the bits: no float64 square root
__device__ __forceinline__ int residual_exponent(const KrylovScalars *sc, int b) {
  const double rr = sc[b].rr;
  if (!(rr > 0.0) || !isfinite(rr)) return 0;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(rr);
  const int E = (int)(bits >> 52);  // sign clear: rr > 0
  const int lb = E ? E - 1023 : (63 - __clzll((long long)(bits & 0xfffffffffffffull))) - 1074;
  return lb >> 1;  // arithmetic shift: floor
}

// x * 2^e by an add to the exponent field (integer ops: the FP64 pipe of this part is narrow).
// Zero stays zero, Inf / NaN pass through, results below the normal range become signed zero and
// above it signed Inf; subnormal inputs count as zero.
__device__ __forceinline__ double scale_pow2(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  const long long sign = b & (long long)0x8000000000000000ull;
  if (ex == 0x7ff) return x;
  if (ex == 0) return __longlong_as_double(sign);
  const int ne = ex + e;
  if (ne <= 0) return __longlong_as_double(sign);
  if (ne >= 0x7ff) return __longlong_as_double(sign | 0x7ff0000000000000ll);
  return __longlong_as_double(b + ((long long)e << 52));
}

// (double) f * 2^e with scale_pow2's rules, from the float's bits (integer ops: conversions between
// float and double run on the narrow FP64 pipe of this part)
__device__ __forceinline__ double widen_pow2(float f, int e) {
  const uint32_t fb = __float_as_uint(f);
  const uint32_t fe = (fb >> 23) & 0xffu, fm = fb & 0x7fffffu;
  const long long sign = (long long)(fb >> 31) << 63;
  if (fe == 0xffu) return __longlong_as_double(sign | 0x7ff0000000000000ll | ((long long)fm << 29));  // Inf / NaN
  int ne;
  long long mant;
  if (fe == 0u) {  // zero, or a float subnormal: a normal double with its leading one at bit p of fm
    if (fm == 0u) return __longlong_as_double(sign);
    const int p = 31 - __clz((int)fm);
    ne = p + 874 + e;  // 2^(p - 149), double bias 1023
    mant = ((long long)fm << (52 - p)) & 0xfffffffffffffll;
  } else {
    ne = (int)fe + 896 + e;  // float bias 127, double bias 1023
    mant = (long long)fm << 29;
  }
  if (ne <= 0) return __longlong_as_double(sign);
  if (ne >= 0x7ff) return __longlong_as_double(sign | 0x7ff0000000000000ll);
  return __longlong_as_double(sign | ((long long)ne << 52) | mant);
}

// (float) scale_pow2(x, e) from the double's bits: round to nearest even, float subnormals and
// overflow to Inf included (integer ops, as above)
__device__ __forceinline__ float narrow_pow2(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned long long M = b & 0xfffffffffffffull;
  if (E == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (M ? 0x400000u | (uint32_t)(M >> 29) : 0u));
  const int ne = E + e;
  if (E == 0 || ne <= 0) return __uint_as_float(sign);  // scale_pow2 flushes double subnormals
  const int u = ne - 1023;
  if (ne >= 0x7ff || u > 127) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long m = M | (1ull << 52);
  if (u >= -126) {  // a normal float: keep 24 bits; a carry into bit 24 raises the exponent (to Inf at most)
    uint32_t r = (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1fffffffull);
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
    return __uint_as_float(sign | (((uint32_t)(u + 126) << 23) + r));
  }
  const int s = -u - 97;  // a float subnormal: the mantissa in units of 2^-149
  if (s > 54) return __uint_as_float(sign);
  const unsigned long long r0 = m >> s, rem = m & ((1ull << s) - 1ull), half = 1ull << (s - 1);
  const uint32_t r = (uint32_t)r0 + ((rem > half || (rem == half && (r0 & 1ull))) ? 1u : 0u);
  return __uint_as_float(sign | r);
}

// ST_MET (GMRES only): the residual estimate met the tolerance inside an open cycle; the true
// residual at the next cycle start turns it into ST_CONV or back into ST_RUN.
enum { ST_RUN = 0, ST_CONV = 1, ST_NAN = 2, ST_STOP = 3, ST_MET = 4 };

// Scratch for deterministic two-stage reductions: per rhs a slot of `nblk` partial sums and a
// completion counter.  The last block to finish sums the partials in index order.
struct Reduce {
  double *part;        // [nrhs][rstride]: value i of block b at i * nblk + b
  unsigned int *count; // [nrhs]  (must start at zero; reset by the last block)
  int nblk;            // block capacity per value
  int rstride;         // doubles per rhs (values capacity * nblk)
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV values per thread; result valid in thread 0.  blockDim.x multiple of 32, <= 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh /* [32*NV] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i * 32 + warp] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = lane < nw ? sh[i * 32 + lane] : 0.0;
      v[i] = warp_sum(t);
    }
  }
}

// After thread 0 of a block has its NV block partials, publish them into red.part for `rhs`
// and return true in thread 0 of the last block of that rhs, with the totals in `tot`
// (summed in block-index order: deterministic).  Call from every thread.
template <int NV>
__device__ __forceinline__ bool publish_partials(const Reduce &red, int rhs, int blk, int nblk,
                                                 const double (&v)[NV], double (&tot)[NV]) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    double *p = red.part + (size_t)rhs * red.rstride;
#pragma unroll
    for (int i = 0; i < NV; ++i) p[i * red.nblk + blk] = v[i];
    __threadfence();
    unsigned int prev = atomicAdd(red.count + rhs, 1u);
    is_last = (prev == (unsigned int)(nblk - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  // the last block: every thread helps sum the partials in a fixed order
  __threadfence();
  const double *p = red.part + (size_t)rhs * red.rstride;
  __shared__ double sh[32 * NV];
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    acc[i] = 0.0;
    // fixed partition: thread t sums blocks t, t + blockDim, ... in order
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc[i] += __ldcg(p + i * red.nblk + b);
  }
  block_sum<NV>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = acc[i];
    red.count[rhs] = 0u;  // ready for the next use
  }
  return threadIdx.x == 0;
}

}  // namespace lag
